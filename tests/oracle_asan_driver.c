/*
 * Host memory-safety run of the oracle: built by test_oracle_sanitizers.py
 * together with oracle/gbsz_oracle.c under AddressSanitizer and UBSan, it
 * compresses and decompresses small seeded fields of every mode (1D/2D/3D/4D,
 * per-block, orders 1-3, radii 2..32768, chunks 64..65536, non-finite values)
 * and decodes single-bit and byte corruptions of the archives.  It checks
 * only that the oracle keeps within its buffers and that valid archives come
 * back within the bound; the sanitizers report everything else and make the
 * process fail.  Prints "ok <cases>" at the end.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../oracle/gbsz_oracle.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;

/* splitmix64: the input generator only */
static uint64_t next_u64(void)
{
    uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unit(void) { return (double)(next_u64() >> 11) / 9007199254740992.0; }

static void fill(float *x, uint64_t n, int kind)
{
    double w = 0.0;
    for (uint64_t i = 0; i < n; i++) {
        w += (unit() - 0.5) * 0.02;
        double v = kind == 0 ? w : kind == 1 ? sin(0.01 * (double)i) + 0.001 * unit() : unit() * 2.0 - 1.0;
        if (unit() < 0.01) v = unit() * 4.0 - 2.0;
        x[i] = (float)v;
    }
    if (kind == 2 && n > 8) {
        x[1] = NAN;
        x[3] = INFINITY;
        x[5] = 3e38f;
    }
}

static int run_case(uint32_t ndim, const uint64_t dims[4], double eb, uint32_t radius, uint32_t chunk,
                    uint32_t lblock, uint32_t order, int kind)
{
    gbsz_ref_params p;
    memset(&p, 0, sizeof(p));
    p.ndim = ndim;
    uint64_t n = 1;
    for (int i = 0; i < 4; i++) {
        p.dims[i] = i < (int)ndim ? dims[i] : 1;
        n *= p.dims[i];
    }
    p.eb = eb;
    p.eb_mode = REF_EB_REL;
    p.radius = radius;
    p.chunk = chunk;
    p.lorenzo_block = lblock;
    p.lorenzo_order = order;
    float *x = (float *)malloc(n * sizeof(float));
    float *y = (float *)malloc(n * sizeof(float));
    fill(x, n, kind);
    const size_t cap = gbsz_ref_compress_bound(&p);
    uint8_t *a = (uint8_t *)malloc(cap);
    size_t bytes = 0;
    int st = gbsz_ref_compress(x, &p, a, cap, &bytes);
    if (st != REF_OK) {
        fprintf(stderr, "compress failed %d\n", st);
        return 1;
    }
    /* the archive exactly: a copy of its own size, so any read past it is caught */
    uint8_t *exact = (uint8_t *)malloc(bytes);
    memcpy(exact, a, bytes);
    st = gbsz_ref_decompress(exact, bytes, y, n);
    if (st != REF_OK) {
        fprintf(stderr, "decompress failed %d\n", st);
        return 1;
    }
    float sc[3];
    gbsz_ref_error_bound(x, n, REF_EB_REL, eb, sc);
    for (uint64_t i = 0; i < n; i++) {
        if (isfinite(x[i]) && fabs((double)x[i] - (double)y[i]) > (double)sc[0]) {
            fprintf(stderr, "bound exceeded at %llu\n", (unsigned long long)i);
            return 1;
        }
    }
    /* corruptions: single bits anywhere, and whole bytes, decoded from exact-size copies */
    for (int t = 0; t < 48; t++) {
        memcpy(exact, a, bytes);
        const size_t pos = (size_t)(next_u64() % bytes);
        if (t % 3 == 0) exact[pos] = (uint8_t)next_u64();
        else exact[pos] ^= (uint8_t)(1u << (next_u64() % 8));
        (void)gbsz_ref_decompress(exact, bytes, y, n);
    }
    /* and truncations */
    for (size_t cut = 1; cut < bytes && cut < 64; cut += 7) (void)gbsz_ref_decompress(exact, bytes - cut, y, n);
    free(exact);
    free(a);
    free(x);
    free(y);
    return 0;
}

int main(void)
{
    int cases = 0, fails = 0;
    const uint64_t d1[4] = {20011, 1, 1, 1}, d2[4] = {181, 97, 1, 1}, d3[4] = {23, 19, 17, 1}, d4[4] = {9, 7, 6, 5};
    const uint64_t tiny[4] = {1, 1, 1, 1}, tiny3[4] = {2, 3, 5, 1};
    struct {
        uint32_t ndim;
        const uint64_t *dims;
        double eb;
        uint32_t radius, chunk, lblock, order;
        int kind;
    } cs[] = {
        {1, d1, 1e-4, 512, 64, 0, 1, 0},   {1, d1, 1e-4, 512, 4096, 0, 1, 0},  {1, d1, 1e-6, 32768, 1024, 0, 1, 0},
        {1, d1, 1e-3, 2, 256, 0, 1, 2},    {1, d1, 1e-4, 512, 65536, 0, 1, 0}, {1, d1, 1e-4, 512, 256, 1, 1, 0},
        {1, d1, 1e-3, 512, 256, 0, 2, 0},  {1, d1, 1e-3, 64, 128, 0, 3, 1},    {2, d2, 1e-4, 512, 512, 0, 1, 1},
        {2, d2, 1e-3, 512, 64, 1, 1, 2},   {2, d2, 1e-3, 512, 256, 0, 3, 1},   {3, d3, 1e-4, 512, 2048, 0, 1, 1},
        {3, d3, 1e-5, 32768, 4096, 0, 1, 0}, {3, d3, 1e-3, 512, 256, 1, 1, 2}, {3, d3, 1e-3, 512, 256, 0, 2, 1},
        {4, d4, 1e-4, 512, 64, 0, 1, 1},   {1, tiny, 1e-3, 512, 64, 0, 1, 0},  {3, tiny3, 1e-3, 2, 64, 0, 1, 2},
    };
    for (size_t i = 0; i < sizeof(cs) / sizeof(cs[0]); i++) {
        cases++;
        if (run_case(cs[i].ndim, cs[i].dims, cs[i].eb, cs[i].radius, cs[i].chunk, cs[i].lblock, cs[i].order,
                     cs[i].kind)) {
            fprintf(stderr, "case %zu failed\n", i);
            fails++;
        }
    }
    if (fails) return 1;
    printf("ok %d\n", cases);
    return 0;
}
