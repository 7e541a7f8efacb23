// k_recon.cu -- S8: reversed dual-quantization (Algorithm 2, decompression;
// Sec. 3.3).
//
// The paper reconstructs cascadingly per chunk.  Since the order-1 Lorenzo
// residual is the d-dimensional first difference of the prequantized
// integers, reconstruction is the d-dimensional inclusive prefix sum of the
// residuals (modulo 2^32), computed here without any inter-CTA waiting:
//   1. outlier scatter: the residual of every code-0 point goes to a per-point
//      scratch array (indices checked: ascending, in range, code 0);
//   2. faces: each tile computes its local prefix sum L and publishes, for
//      every non-empty subset A of the dimensions, L taken at the tile's last
//      coordinate along A as a function of the other coordinates (1D: the
//      tile total; 2D: last column, last row, total; 3D: 3 faces, 3 edges,
//      total);
//   3. carries: inclusive scans of each published array along the tile grid
//      dimensions in A;
//   4. values: S = L + sum over A of the scanned array of the tile that
//      precedes this one along every dimension of A, at this point's other
//      coordinates; d' = fl(2eb * fl((float)S)); then verbatim exceptions.
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>
#include <cstring>
#include <type_traits>

namespace gbsz {

namespace {

struct Geo {
    uint32_t ndim;
    uint64_t n[3];      // field extents
    uint32_t T[3];      // tile extents
    uint32_t nt[3];     // tiles per dimension
    uint64_t ntiles;
    uint64_t size[8];   // entries per tile of the array of subset A
    uint64_t off[8];    // start of the array of subset A in the carry scratch
};

constexpr int k1Threads = 256;                // 8 warps, each on its own tiles
constexpr int k1PerThread = 16;
constexpr int k1Tile = 32 * k1PerThread;      // 512 points: one warp
static_assert(k1Tile == (int)kRecon1DTile, "decoder tile sums and 1D tiles must agree");
constexpr int k2TX = 128, k2TY = 32, k2Threads = 256;
constexpr int k3TX = 32, k3TY = 16, k3TZ = 16, k3Threads = 512;

Geo make_geo(uint32_t ndim, const uint64_t dims[3])
{
    Geo g{};
    g.ndim = ndim;
    for (int d = 0; d < 3; d++) g.n[d] = d < (int)ndim ? dims[d] : 1;
    if (ndim == 1) {
        g.T[0] = k1Tile; g.T[1] = 1; g.T[2] = 1;
    } else if (ndim == 2) {
        g.T[0] = k2TX; g.T[1] = k2TY; g.T[2] = 1;
    } else {
        g.T[0] = k3TX; g.T[1] = k3TY; g.T[2] = k3TZ;
    }
    g.ntiles = 1;
    for (int d = 0; d < 3; d++) {
        g.nt[d] = (uint32_t)((g.n[d] + g.T[d] - 1) / g.T[d]);
        g.ntiles *= g.nt[d];
    }
    uint64_t off = 0;
    for (int A = 1; A < 8; A++) {
        bool used = true;
        for (int d = 0; d < 3; d++)
            if ((A >> d) & 1) used &= d < (int)ndim;
        uint64_t s = 1;
        for (int d = 0; d < (int)ndim; d++)
            if (!((A >> d) & 1)) s *= g.T[d];
        g.size[A] = used ? s : 0;
        g.off[A] = off;
        off += used ? s * g.ntiles : 0;
    }
    g.off[0] = off;  // total entries
    return g;
}

__device__ __forceinline__ uint32_t delta_of(const ReconArgs &a, uint64_t i)
{
    const uint32_t c = a.codes[i];
    return c ? c - a.radius : (uint32_t)a.dscr[i];
}

// ---------------------------------------------------------------------------
// 1. outliers

__device__ __forceinline__ void scatter_outliers_body(const ReconArgs &a, uint64_t n, VGrid vg)
{
    const uint8_t *o = a.archive + a.off_outl;
    for (uint64_t t = (uint64_t)vg.bid * blockDim.x + threadIdx.x; t < a.m;
         t += (uint64_t)vg.nb * blockDim.x) {
        const uint32_t idx = *reinterpret_cast<const uint32_t *>(o + 8 * t);
        const int32_t d = *reinterpret_cast<const int32_t *>(o + 8 * t + 4);
        bool ok = idx < n;
        if (t > 0) ok &= idx > *reinterpret_cast<const uint32_t *>(o + 8 * (t - 1));
        if (ok && a.codes) ok &= a.codes[idx] == 0;  // no codes: the fused 1D decoder kept them on chip
        if (ok) {
            a.dscr[idx] = d;
        } else {
            atomicOr(&a.ctl->error, DERR_CORRUPT);
        }
    }
}

__global__ void k_scatter_outliers(const __grid_constant__ ReconArgs a, uint64_t n)
{
    scatter_outliers_body(a, n, vgrid_self());
}

// 1D: the outlier residuals go to the tile sums (added to the in-cap sums
// the decoder left there), and every 512-point tile g learns where its
// outliers start in the index-ordered list: start[g] = first outlier with
// idx >= 512 g, for g = 0 .. ntiles (start[ntiles] = m).  Consecutive
// outliers mostly share a tile, so a warp adds each run of equal tiles with
// one atomic.
constexpr uint32_t kGroup1D = kRecon1DTile;

__device__ __forceinline__ void outlier_tiles_1d_body(const ReconArgs &a, uint64_t n, uint64_t ngroups, uint32_t *start,
                                                      VGrid vg)
{
    const uint8_t *o = a.archive + a.off_outl;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)vg.nb * blockDim.x;
    // whole warps stay in the loop so the shuffles see every lane
    const uint64_t tmax = (a.m + 31) & ~31ull;
    for (uint64_t t = (uint64_t)vg.bid * blockDim.x + threadIdx.x; t < tmax; t += stride) {
        const bool live = t < a.m;
        uint32_t idx = 0, d = 0;
        bool ok = true;
        int64_t gprev = -1;
        if (live) {
            idx = *reinterpret_cast<const uint32_t *>(o + 8 * t);
            d = *reinterpret_cast<const uint32_t *>(o + 8 * t + 4);
            ok = idx < n;
            if (t > 0) {
                const uint32_t pidx = *reinterpret_cast<const uint32_t *>(o + 8 * (t - 1));
                ok &= idx > pidx;
                gprev = (int64_t)(pidx / kGroup1D);
            }
        }
        const uint64_t T = ok ? idx / kRecon1DTile : 0;
        if (live && !ok) atomicOr(&a.ctl->error, DERR_CORRUPT);
        // runs of equal tiles inside the warp (the list is sorted)
        const uint64_t key = live && ok ? T : ~0ull;
        const uint64_t kprev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool head = lane == 0 || kprev != key;
        uint32_t sum = live && ok ? d : 0u;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const unsigned below = heads & (0xffffffffu >> (31 - lane));
        const uint32_t seg0 = 31 - __clz(below);  // first lane of this lane's run
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, sum, off);
            if (lane >= (uint32_t)off && lane - off >= seg0) sum += v;
        }
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u) || t + 1 >= a.m;
        if (live && ok && tail && GBSZ_CHECK(T < a.faces_cap, a.ctl)) atomicAdd(&a.faces[T], sum);
        if (live && ok) {
            const uint64_t G = idx / kGroup1D;
            for (int64_t u = gprev + 1; u <= (int64_t)G; u++)
                if (GBSZ_CHECK((uint64_t)u <= ngroups, a.ctl)) start[u] = (uint32_t)t;
            if (t + 1 == a.m)
                for (uint64_t u = G + 1; u <= ngroups; u++) start[u] = (uint32_t)a.m;
        }
    }
}

__global__ void k_outlier_tiles_1d(const __grid_constant__ ReconArgs a, uint64_t n, uint64_t ngroups, uint32_t *start)
{
    outlier_tiles_1d_body(a, n, ngroups, start, vgrid_self());
}

__device__ __forceinline__ void patch_exceptions_body(const ReconArgs &a, uint64_t n, VGrid vg)
{
    const uint8_t *e = a.archive + a.off_exc;
    for (uint64_t t = (uint64_t)vg.bid * blockDim.x + threadIdx.x; t < a.e;
         t += (uint64_t)vg.nb * blockDim.x) {
        const uint32_t idx = *reinterpret_cast<const uint32_t *>(e + 8 * t);
        const uint32_t raw = *reinterpret_cast<const uint32_t *>(e + 8 * t + 4);
        bool ok = idx < n;
        if (t > 0) ok &= idx > *reinterpret_cast<const uint32_t *>(e + 8 * (t - 1));
        if (ok && a.codes) ok &= a.codes[idx] == 0;  // no codes: the fused 1D decoder kept them on chip
        if (ok) reinterpret_cast<uint32_t *>(a.out)[idx] = raw;
        else atomicOr(&a.ctl->error, DERR_CORRUPT);
    }
}

__global__ void k_patch_exceptions(const __grid_constant__ ReconArgs a, uint64_t n)
{
    patch_exceptions_body(a, n, vgrid_self());
}

// ---------------------------------------------------------------------------
// 1D tiles: 4096 points, 16 consecutive per thread, block scan of totals

// One 512-point tile per warp iteration, with no block-level synchronisation.
// A tile's outliers are the run start[t] .. start[t+1] of the index-ordered
// list; the first 32 of them are loaded one per lane, and a warp scan of the
// lanes' code-0 counts tells each lane which entries its code-0 points take,
// in order (fetched by shuffles; runs longer than 32 read the rest from
// global memory).  Every entry's index must be its point's and the counts
// must match the run.  Residuals are code - R, or the outlier's residual for
// code 0; their sum within the tile is a thread run plus a warp scan, and the
// tile's carry F[t] completes the prefix.  The codes of the next two tiles
// are in flight (cp.async into a per-warp ring in shared memory), and the
// next tile's outlier entries and carry and the run bounds of the tile after
// it are loaded before this tile is processed.

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kValStages = 3;  // tiles of codes per warp in shared memory: this one and two ahead

__device__ __forceinline__ void values_1d_body(const ReconArgs &a, const Geo &g, const uint32_t *F, const uint32_t *start,
                                               VGrid vg)
{
    __shared__ uint32_t s_od[k1Threads * 17];  // outlier residuals by (thread, point); stride 17 spreads banks
    // codes of the next tiles, copied by each lane for itself (32 bytes per
    // lane per tile) with cp.async, two tiles ahead of the one in use
    __shared__ uint4 s_code[k1Threads / 32][kValStages][64];
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint64_t n = g.n[0];
    const float ebx2 = a.ebx2;
    const uint32_t R = a.radius;
    const uint32_t lane = threadIdx.x & 31;
    const uint2 *ol = reinterpret_cast<const uint2 *>(a.archive + a.off_outl);
    uint32_t *od = s_od + threadIdx.x * 17;
    const uint64_t nwarps = (uint64_t)vg.nb * (k1Threads / 32);
    bool bad = false;
    auto bounds = [&](uint64_t t, uint32_t &lo, uint32_t &hi) {
        lo = hi = 0;
        if (a.m && t < g.ntiles) {
            lo = start[t];
            hi = start[t + 1];
        }
    };
    uint4(*ring)[64] = s_code[threadIdx.x >> 5];
    // one commit group per tile, empty past the end, so the group count stays uniform
    auto issue = [&](uint64_t t, int stage) {
        const uint64_t s0 = t * k1Tile + (uint64_t)lane * 16;
        if (t < g.ntiles && s0 + 16 <= n) {
            cp_async16(&ring[stage][2 * lane], a.codes + s0);
            cp_async16(&ring[stage][2 * lane + 1], a.codes + s0 + 8);
        }
        cp_async_commit();
    };
    auto entry = [&](uint32_t lo, uint32_t hi) {
        uint2 en = make_uint2(0xFFFFFFFFu, 0u);
        if (lo + lane < hi) en = ol[lo + lane];
        return en;
    };
    uint64_t tile = (uint64_t)vg.bid * (k1Threads / 32) + (threadIdx.x >> 5);
    uint32_t lo, hi, lo1, hi1;
    bounds(tile, lo, hi);
    bounds(tile + nwarps, lo1, hi1);
    for (int k = 0; k < kValStages - 1; k++) issue(tile + (uint64_t)k * nwarps, k);
    uint2 en = entry(lo, hi);
    int stage = 0;
    // per-block mode: no carries (every 32-point block restarts from 0)
    const bool blocked = a.lblock != 0;
    uint32_t carry = tile < g.ntiles && !blocked ? F[tile] : 0u;
    for (; tile < g.ntiles; tile += nwarps) {
        const uint64_t s0 = tile * k1Tile + (uint64_t)lane * 16;
        uint32_t c[16];
        cp_async_wait<kValStages - 2>();  // this tile's group has landed
        if (s0 + 16 <= n) {
            const uint4 w0 = ring[stage][2 * lane], w1 = ring[stage][2 * lane + 1];
            const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int j = 0; j < 16; j++) c[j] = (w[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++) c[j] = s0 + j < n ? a.codes[s0 + j] : R;  // past the end: residual 0
        }
        const uint32_t clo = lo, chi = hi, ccarry = carry;
        const uint2 cen = en;
        // the tile two ahead into the slot just read; next tile's outliers
        const uint64_t tn = tile + nwarps;
        issue(tile + (uint64_t)(kValStages - 1) * nwarps, (stage + kValStages - 1) % kValStages);
        stage = (stage + 1) % kValStages;
        en = entry(lo1, hi1);
        lo = lo1;
        hi = hi1;
        bounds(tn + nwarps, lo1, hi1);
        if (tn < g.ntiles && !blocked) carry = F[tn];

        uint32_t d[16], zm = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) {
            d[j] = c[j] - R;
            zm |= (c[j] == 0 ? 1u : 0u) << j;
        }
        const uint32_t zc = __popc(zm);
        const uint32_t zinc = warp_incl_scan(zc);
        if (lane == 31 && (uint64_t)clo + zinc != chi) bad = true;  // a tile holds exactly its outliers
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, zc);
        uint32_t r = zinc - zc;  // this lane's first entry within the run
        uint32_t m = zm;
        for (uint32_t k = 0; k < kmax; k++, r++) {
            const uint32_t ix = __shfl_sync(0xffffffffu, cen.x, r & 31);
            const uint32_t dv = __shfl_sync(0xffffffffu, cen.y, r & 31);
            if (k < zc) {
                const uint32_t j = __ffs(m) - 1;
                m &= m - 1;
                uint2 e = make_uint2(ix, dv);
                if (r >= 32) e = (uint64_t)clo + r < chi ? ol[clo + r] : make_uint2(0xFFFFFFFFu, 0u);
                if (e.x != s0 + j) bad = true;
                od[j] = e.x == s0 + j ? e.y : 0u;
            }
        }
        if (zm) {
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (c[j] == 0) d[j] = od[j];
        }
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < 16; j++) s += d[j];
        uint32_t run;
        if (blocked) {
            // a 32-point block is two lanes: the odd lane continues the even one
            const uint32_t sprev = __shfl_up_sync(0xffffffffu, s, 1);
            run = (lane & 1u) ? sprev : 0u;
        } else {
            run = ccarry + warp_incl_scan(s) - s;
        }
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            run += d[j];
            v[j] = recon_value((int32_t)run, ebx2);
        }
        if (a.anchors) {
            // anchored archive: the integer before each chunk is its anchor
            // (chunks are multiples of 16 points, so only a run's last point
            // can precede one)
            if (s0 + 16 < n && ((s0 + 16) & (a.chunk - 1)) == 0 && a.anchors[(s0 + 16) / a.chunk] != run) bad = true;
            if (s0 == 0 && a.anchors[0] != 0u) bad = true;
        }
        if (s0 + 16 <= n) {
            float4 *o = reinterpret_cast<float4 *>(a.out + s0);
#pragma unroll
            for (int j = 0; j < 4; j++) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (s0 + j < n) a.out[s0 + j] = v[j];
        }
    }
    cp_async_wait<0>();
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
}

__global__ void __launch_bounds__(k1Threads) k_values_1d(const __grid_constant__ ReconArgs a, const __grid_constant__ Geo g,
                                                         const uint32_t *F, const uint32_t *start)
{
    values_1d_body(a, g, F, start, vgrid_self());
}

// ---------------------------------------------------------------------------
// Per-block mode, 2D / 3D: every B^D block is reconstructed on its own as a
// d-dimensional inclusive prefix sum of its residuals (zero padding around
// the block), one thread per point, sums along x, then y, then z in shared
// memory.

template <int D>
__device__ __forceinline__ void values_blocked_body(const ReconArgs &a, const Geo &g, VGrid vg)
{
    constexpr uint32_t B = lorenzo_block_extent(D);
    constexpr uint32_t NB = D == 2 ? B * B : B * B * B;
    __shared__ uint32_t s0[NB], s1[NB];
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint32_t t = threadIdx.x;
    const uint32_t lx = t % B, ly = (t / B) % B, lz = D == 3 ? t / (B * B) : 0u;
    const uint64_t nbx = (g.n[0] + B - 1) / B, nby = (g.n[1] + B - 1) / B;
    const uint64_t nbz = D == 3 ? (g.n[2] + B - 1) / B : 1;
    const uint64_t nblocks = nbx * nby * nbz;
    for (uint64_t blk = vg.bid; blk < nblocks; blk += vg.nb) {
        const uint64_t gx = (blk % nbx) * B + lx, gy = ((blk / nbx) % nby) * B + ly;
        const uint64_t gz = D == 3 ? (blk / (nbx * nby)) * B + lz : 0;
        const bool in = gx < g.n[0] && gy < g.n[1] && gz < g.n[2];
        const uint64_t idx = (gz * g.n[1] + gy) * g.n[0] + gx;
        s0[t] = in ? delta_of(a, idx) : 0u;
        __syncthreads();
        uint32_t v = 0;  // along x
        for (uint32_t k = 0; k <= lx; k++) v += s0[t - lx + k];
        s1[t] = v;
        __syncthreads();
        v = 0;  // along y
        for (uint32_t k = 0; k <= ly; k++) v += s1[t - (ly - k) * B];
        if (D == 3) {
            s0[t] = v;
            __syncthreads();
            v = 0;  // along z
            for (uint32_t k = 0; k <= lz; k++) v += s0[t - (lz - k) * B * B];
        }
        if (in) a.out[idx] = recon_value((int32_t)v, a.ebx2);
        __syncthreads();  // s0 / s1 are reused by the next block
    }
}

template <int D>
__global__ void __launch_bounds__(D == 2 ? 256 : 512) k_values_blocked(const __grid_constant__ ReconArgs a,
                                                                       const __grid_constant__ Geo g)
{
    values_blocked_body<D>(a, g, vgrid_self());
}

// ---------------------------------------------------------------------------
// 2D / 3D tiles through shared memory

// Tile geometry known at compile time.  Thread t's j-th point is l = t + j*NT:
// with NT a multiple of TX its x is t % TX for every j, and its row index
// (y + TY z inside the tile) is t / TX + j * NT / TX.  Point indices fit in 32
// bits (n < 2^32).
template <int TX, int TY, int TZ, int NT>
struct TileGeo {
    static constexpr int NE = TX * TY * TZ, PER = NE / NT, RPJ = NT / TX;
    static_assert(NE % NT == 0 && NT % TX == 0, "whole rows per thread step");
    static constexpr int D = TZ > 1 ? 3 : 2;
    static constexpr int NA = D == 3 ? 7 : 3;  // nonempty subsets of the dimensions
    // entries of subset A's array per tile, and where it starts in the staged carries
    __host__ __device__ static constexpr int size(int A)
    {
        return ((A & 1) ? 1 : TX) * ((A & 2) ? 1 : TY) * ((A & 4) ? 1 : TZ);
    }
    __host__ __device__ static constexpr int base(int A)
    {
        int b = 0;  // a loop, not recursion: it must inline into the kernels
        for (int B = 1; B < A; B++) b += size(B);
        return b;
    }
    // index of point (x, y, z) in subset A's array: the coordinates not in A
    __host__ __device__ static constexpr int comp(int A, int x, int y, int z)
    {
        return ((A & 1) ? 0 : x) + ((A & 2) ? 0 : y * ((A & 1) ? 1 : TX)) +
               ((A & 4) ? 0 : z * ((A & 1) ? 1 : TX) * ((A & 2) ? 1 : TY));
    }
    // Column layout (3D tiles of 32-wide rows with one thread per (x, y)):
    // thread t owns the z-column (t % TX, t / TX) and scans it in registers;
    // the staged tile's rows are padded to TX + 1 words, so that scans along
    // y (a thread per (x, z) line) and along x (HPR threads per row) hit 32
    // different banks.
    static constexpr bool COL = D == 3 && TX == 32 && NT == TX * TY && TX * TZ <= NT;
    static constexpr int RS = COL ? TX + 1 : TX;  // words per staged row
    static constexpr int SMW = TY * TZ * RS;
    __host__ __device__ static constexpr int sidx(int x, int y, int z) { return (z * TY + y) * RS + x; }
};

// tile coordinates of a tile index (tile counts fit in 32 bits: n < 2^32)
__device__ __forceinline__ void tile_coords(const Geo &g, uint32_t tile, uint32_t tc[3])
{
    const uint32_t nt0 = g.nt[0], nt1 = g.nt[1];
    const uint32_t r = tile / nt0;
    tc[0] = tile - r * nt0;
    tc[1] = r % nt1;
    tc[2] = r / nt1;
}

// Tile-local inclusive 3D prefix sum of the residuals in the column layout:
// z in registers, then y and x through the padded staging array.
template <int TX, int TY, int TZ, int NT>
__device__ void tile_prefix_col(const ReconArgs &a, const Geo &g, const uint32_t tc[3], uint32_t *sm)
{
    using TG = TileGeo<TX, TY, TZ, NT>;
    static_assert(TG::COL, "column layout");
    const uint32_t n0 = (uint32_t)g.n[0], n1 = (uint32_t)g.n[1], n2 = (uint32_t)g.n[2];
    const int x = threadIdx.x % TX, y = threadIdx.x / TX;
    const uint32_t gx = tc[0] * TX + x, gy = tc[1] * TY + y, gz0 = tc[2] * TZ;
    const bool inxy = gx < n0 && gy < n1;
    const uint32_t plane = n0 * n1;
    const uint32_t base = (gz0 * n1 + gy) * n0 + gx;  // only dereferenced in range
    uint32_t code[TZ];
#pragma unroll
    for (int z = 0; z < TZ; z++)
        code[z] = inxy && gz0 + z < n2 ? (uint32_t)a.codes[base + z * plane] : a.radius;  // outside: residual 0
    uint32_t run = 0;
#pragma unroll
    for (int z = 0; z < TZ; z++) {
        uint32_t v = code[z] - a.radius;
        if (code[z] == 0) v = (uint32_t)a.dscr[base + z * plane];
        run += v;
        sm[TG::sidx(x, y, z)] = run;
    }
    __syncthreads();
    // along y: a thread per (x, z) line
    for (int line = threadIdx.x; line < TX * TZ; line += NT) {
        const int lx = line % TX, lz = line / TX;
        uint32_t r = 0;
#pragma unroll
        for (int yy = 0; yy < TY; yy++) {
            const int i = TG::sidx(lx, yy, lz);
            r += sm[i];
            sm[i] = r;
        }
    }
    __syncthreads();
    // along x: HPR threads per row (adjacent lanes), SEG points each, then
    // the segment totals scanned across the HPR lanes
    constexpr int ROWS = TY * TZ, HPR = NT / ROWS, SEG = TX / HPR;
    static_assert(NT % ROWS == 0 && HPR >= 1 && HPR <= 32 && TX % HPR == 0, "row split");
    {
        const int row = threadIdx.x / HPR, seg = threadIdx.x % HPR;
        uint32_t *p = sm + row * TG::RS + seg * SEG;
        uint32_t v[SEG];
        uint32_t r = 0;
#pragma unroll
        for (int i = 0; i < SEG; i++) {
            r += p[i];
            v[i] = r;
        }
        uint32_t incl = r;
#pragma unroll
        for (int o = 1; o < HPR; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o, HPR);
            if (seg >= o) incl += t;
        }
        const uint32_t excl = incl - r;
#pragma unroll
        for (int i = 0; i < SEG; i++) p[i] = v[i] + excl;
    }
    __syncthreads();
}

// Tile-local inclusive prefix sum in the row layout (2D tiles): thread t's
// j-th point is l = t + j * NT; rows scanned by warps, columns by threads.
template <int TX, int TY, int TZ, int NT>
__device__ void tile_prefix_rows(const ReconArgs &a, const Geo &g, const uint32_t tc[3], uint32_t *sm)
{
    using TG = TileGeo<TX, TY, TZ, NT>;
    static_assert(TG::RS == TX, "row-major staging");
    const uint32_t tx = tc[0], ty = tc[1], tz = tc[2];
    const uint32_t n0 = (uint32_t)g.n[0], n1 = (uint32_t)g.n[1], n2 = (uint32_t)g.n[2];
    const uint32_t gx = tx * TX + threadIdx.x % TX;
    const uint32_t r0 = threadIdx.x / TX;
    // all of the thread's codes are loaded before any is used, so the loads
    // overlap; the few outliers' residuals follow
    uint32_t code[TG::PER];
#pragma unroll
    for (int j = 0; j < TG::PER; j++) {
        const uint32_t r = r0 + j * TG::RPJ, gy = ty * TY + r % TY, gz = tz * TZ + r / TY;
        const bool in = gx < n0 && gy < n1 && gz < n2;
        code[j] = in ? (uint32_t)a.codes[(gz * n1 + gy) * n0 + gx] : a.radius;  // outside: residual 0
    }
#pragma unroll
    for (int j = 0; j < TG::PER; j++) {
        uint32_t v = code[j] - a.radius;
        if (code[j] == 0) {
            const uint32_t r = r0 + j * TG::RPJ, gy = ty * TY + r % TY, gz = tz * TZ + r / TY;
            v = (uint32_t)a.dscr[(gz * n1 + gy) * n0 + gx];
        }
        sm[threadIdx.x + j * NT] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int line = warp; line < TY * TZ; line += NT / 32) {
        uint32_t carry = 0;
#pragma unroll
        for (int seg = 0; seg < TX / 32; seg++) {
            const int idx = line * TX + seg * 32 + lane;
            const uint32_t v = warp_incl_scan(sm[idx]) + carry;
            sm[idx] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    if (TY > 1) {
        for (int line = threadIdx.x; line < TX * TZ; line += NT) {
            const int x = line % TX, z = line / TX;
            uint32_t run = 0;
#pragma unroll
            for (int y = 0; y < TY; y++) {
                const int idx = (z * TY + y) * TX + x;
                run += sm[idx];
                sm[idx] = run;
            }
        }
        __syncthreads();
    }
    if (TZ > 1) {
        for (int line = threadIdx.x; line < TX * TY; line += NT) {
            uint32_t run = 0;
#pragma unroll
            for (int z = 0; z < TZ; z++) {
                const int idx = z * TX * TY + line;
                run += sm[idx];
                sm[idx] = run;
            }
        }
        __syncthreads();
    }
}

template <int TX, int TY, int TZ, int NT>
__device__ __forceinline__ void tile_prefix(const ReconArgs &a, const Geo &g, const uint32_t tc[3], uint32_t *sm)
{
    if constexpr (TileGeo<TX, TY, TZ, NT>::COL) tile_prefix_col<TX, TY, TZ, NT>(a, g, tc, sm);
    else tile_prefix_rows<TX, TY, TZ, NT>(a, g, tc, sm);
}

template <int TX, int TY, int TZ, int NT>
__device__ __forceinline__ void faces_body(const ReconArgs &a, const Geo &g, uint32_t *F, VGrid vg)
{
    using TG = TileGeo<TX, TY, TZ, NT>;
    __shared__ uint32_t sm[TG::SMW];
    if (a.ctl->error & DERR_CORRUPT) return;
    for (uint32_t tile = vg.bid; tile < (uint32_t)g.ntiles; tile += vg.nb) {
        uint32_t tc[3];
        tile_coords(g, tile, tc);
        tile_prefix<TX, TY, TZ, NT>(a, g, tc, sm);
        for (int A = 1; A <= TG::NA; A++) {
            const int sz = TG::size(A);
            uint32_t *dst = F + g.off[A] + tile * (uint64_t)sz;
            for (int ci = threadIdx.x; ci < sz; ci += NT) {
                // complement coordinates from ci, A coordinates at the last index
                int r = ci, x = TX - 1, y = TY - 1, z = TZ - 1;
                if (!(A & 1)) { x = r % TX; r /= TX; }
                if (!(A & 2)) { y = r % TY; r /= TY; }
                if (!(A & 4)) { z = r; }
                if (GBSZ_CHECK(g.off[A] + tile * (uint64_t)sz + ci < a.faces_cap, a.ctl)) dst[ci] = sm[TG::sidx(x, y, z)];
            }
        }
        __syncthreads();
    }
}

template <int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 3 : 6) k_faces(const __grid_constant__ ReconArgs a,
                                                              const __grid_constant__ Geo g, uint32_t *F)
{
    faces_body<TX, TY, TZ, NT>(a, g, F, vgrid_self());
}

template <int TX, int TY, int TZ, int NT>
__device__ __forceinline__ void values_body(const ReconArgs &a, const Geo &g, const uint32_t *F, VGrid vg)
{
    using TG = TileGeo<TX, TY, TZ, NT>;
    __shared__ uint32_t sm[TG::SMW];
    __shared__ uint32_t carry[TG::base(TG::NA) + TG::size(TG::NA)];
    if (a.ctl->error & DERR_CORRUPT) return;
    const float ebx2 = a.ebx2;
    for (uint32_t tile = vg.bid; tile < (uint32_t)g.ntiles; tile += vg.nb) {
        uint32_t tc[3];
        tile_coords(g, tile, tc);
        // stage the carries of every subset: each subset's array has at most
        // NT entries, so a thread loads one entry of each, all loads at once
        uint32_t cv[TG::NA + 1];
#pragma unroll
        for (int A = 1; A <= TG::NA; A++) {
            static_assert(TG::size(1) <= NT && TG::size(2) <= NT && (TG::D == 2 || TG::size(4) <= NT),
                          "one carry entry per thread and subset");
            cv[A] = 0;
            bool has = true;
            uint32_t pt[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                pt[d] = tc[d];
                if ((A >> d) & 1) {
                    has &= tc[d] > 0;
                    pt[d] = tc[d] - 1;
                }
            }
            const uint64_t ptile = ((uint64_t)pt[2] * g.nt[1] + pt[1]) * g.nt[0] + pt[0];
            if (has && (int)threadIdx.x < TG::size(A) &&
                GBSZ_CHECK(g.off[A] + ptile * (uint64_t)TG::size(A) + threadIdx.x < a.faces_cap, a.ctl))
                cv[A] = F[g.off[A] + ptile * (uint64_t)TG::size(A) + threadIdx.x];
        }
#pragma unroll
        for (int A = 1; A <= TG::NA; A++)
            if ((int)threadIdx.x < TG::size(A)) carry[TG::base(A) + threadIdx.x] = cv[A];
        tile_prefix<TX, TY, TZ, NT>(a, g, tc, sm);
        const uint32_t n0 = (uint32_t)g.n[0], n1 = (uint32_t)g.n[1], n2 = (uint32_t)g.n[2];
        const uint32_t x0 = tc[0] * TX, y0 = tc[1] * TY, z0 = tc[2] * TZ;
        if constexpr (TG::COL) {
            // the thread's own column: x, y fixed, z = 0 .. TZ-1
            const int x = threadIdx.x % TX, y = threadIdx.x / TX;
            const uint32_t gx = x0 + x, gy = y0 + y;
            const uint32_t plane = n0 * n1, base = (z0 * n1 + gy) * n0 + gx;
            if (gx < n0 && gy < n1) {
#pragma unroll
                for (int z = 0; z < TZ; z++) {
                    uint32_t s = sm[TG::sidx(x, y, z)];
#pragma unroll
                    for (int A = 1; A <= TG::NA; A++) s += carry[TG::base(A) + TG::comp(A, x, y, z)];
                    if (z0 + z < n2 && GBSZ_CHECK((uint64_t)base + (uint64_t)z * plane < (uint64_t)plane * n2, a.ctl))
                        a.out[base + z * plane] = recon_value((int32_t)s, ebx2);
                }
            }
        } else {
            for (int l = threadIdx.x; l < TX * TY * TZ; l += NT) {
                const int x = l % TX, y = (l / TX) % TY, z = l / (TX * TY);
                const uint32_t gx = x0 + x, gy = y0 + y, gz = z0 + z;
                if (gx < n0 && gy < n1 && gz < n2) {
                    uint32_t s = sm[TG::sidx(x, y, z)];
#pragma unroll
                    for (int A = 1; A <= TG::NA; A++) s += carry[TG::base(A) + TG::comp(A, x, y, z)];
                    if (GBSZ_CHECK(((uint64_t)gz * n1 + gy) * n0 + gx < (uint64_t)n0 * n1 * n2, a.ctl))
                        a.out[(gz * n1 + gy) * n0 + gx] = recon_value((int32_t)s, ebx2);
                }
            }
        }
        __syncthreads();
    }
}

template <int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 4 : 8) k_values(const __grid_constant__ ReconArgs a,
                                                              const __grid_constant__ Geo g, const uint32_t *F)
{
    values_body<TX, TY, TZ, NT>(a, g, F, vgrid_self());
}

// ---------------------------------------------------------------------------
// 3. inclusive scans of a subset's array along one tile-grid dimension

__device__ __forceinline__ uint64_t line_base(const Geo &g, int A, int d, uint64_t line, uint64_t &stride)
{
    const uint64_t sz = g.size[A];
    const uint64_t ci = line % sz;
    uint64_t r = line / sz;
    uint64_t c[3] = {0, 0, 0};
    for (int e = 0; e < 3; e++) {
        if (e == d) continue;
        c[e] = r % g.nt[e];
        r /= g.nt[e];
    }
    const uint64_t tile = (c[2] * g.nt[1] + c[1]) * g.nt[0] + c[0];
    stride = sz * (d == 0 ? 1 : d == 1 ? g.nt[0] : (uint64_t)g.nt[0] * g.nt[1]);
    return g.off[A] + tile * sz + ci;
}

// one warp per line, 32 entries at a time: for few lines, where a thread per
// line would leave most of the GPU idle behind one long serial chain
__device__ __forceinline__ void scan_lines_warp_body(const Geo &g, int A, int d, uint64_t nlines, uint32_t *F, VGrid vg)
{
    const uint32_t lane = threadIdx.x & 31, len = g.nt[d];
    const uint64_t nw = ((uint64_t)vg.nb * blockDim.x) >> 5;
    for (uint64_t line = ((uint64_t)vg.bid * blockDim.x + threadIdx.x) >> 5; line < nlines; line += nw) {
        uint64_t stride;
        const uint64_t p0 = line_base(g, A, d, line, stride);
        uint32_t carry = 0;
        for (uint32_t i0 = 0; i0 < len; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t v = i < len ? F[p0 + i * stride] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= (uint32_t)o) v += u;
            }
            v += carry;
            if (i < len) F[p0 + i * stride] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// one CTA per long line
__global__ void __launch_bounds__(1024) k_scan_lines_cta(Geo g, int A, int d, uint32_t *F)
{
    __shared__ uint32_t sh[33];
    uint64_t stride;
    const uint64_t p0 = line_base(g, A, d, blockIdx.x, stride);
    const uint32_t len = g.nt[d], T = blockDim.x, t = threadIdx.x;
    const uint32_t per = (len + T - 1) / T;
    const uint32_t lo = min(len, t * per), hi = min(len, lo + per);
    uint32_t s = 0;
    for (uint32_t i = lo; i < hi; i++) s += F[p0 + i * stride];
    uint32_t tot;
    uint32_t run = block_excl_scan(s, sh, &tot);
    for (uint32_t i = lo; i < hi; i++) {
        run += F[p0 + i * stride];
        F[p0 + i * stride] = run;
    }
}

// One pass along tile-grid dimension d over every subset that contains d
// (subsets are separate arrays, and each subset's dimensions are scanned in
// increasing order, pass by pass): lines numbered across the subsets.
struct LinePass {
    Geo g;
    uint32_t *F;
    int d, na;
    int A[4];
    uint64_t first[5];  // lines before subset i; first[na] = all lines
};

__device__ __forceinline__ uint64_t pass_line(const LinePass &p, uint64_t line, uint64_t &stride)
{
    int i = 0;
    while (i + 1 < p.na && line >= p.first[i + 1]) i++;
    return line_base(p.g, p.A[i], p.d, line - p.first[i], stride);
}

// a warp per line (few lines)
__global__ void __launch_bounds__(256) k_scan_pass_warp(const __grid_constant__ LinePass p)
{
    const uint32_t lane = threadIdx.x & 31, len = p.g.nt[p.d];
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5, nlines = p.first[p.na];
    for (uint64_t line = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; line < nlines; line += nw) {
        uint64_t stride;
        const uint64_t p0 = pass_line(p, line, stride);
        uint32_t carry = 0;
        for (uint32_t i0 = 0; i0 < len; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t v = i < len ? p.F[p0 + i * stride] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= (uint32_t)o) v += u;
            }
            v += carry;
            if (i < len) p.F[p0 + i * stride] = v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// a thread per line (many lines)
__global__ void __launch_bounds__(256) k_scan_pass(const __grid_constant__ LinePass p)
{
    const uint64_t line = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= p.first[p.na]) return;
    uint64_t stride;
    uint64_t q = pass_line(p, line, stride);
    uint32_t run = 0;
    for (uint32_t i = 0; i < p.g.nt[p.d]; i++, q += stride) {
        run += p.F[q];
        p.F[q] = run;
    }
}

// in-place exclusive scan of the 1D tile sums (modulo 2^32)
struct TileOp {
    using T = uint32_t;
    uint32_t *v;
    __device__ T load(uint64_t i) const { return v[i]; }
    __device__ void store(uint64_t i, T x) const { v[i] = x; }
    __device__ void total(T) const {}
};

// ---------------------------------------------------------------------------
// Order n > 1: the residual is prod_j (1 - S_j)^n q, so q comes back from n
// inclusive prefix sums along every dimension, modulo 2^32.  The residuals
// are expanded into an int32 array (code - R; outliers scattered on top),
// then every sum is a pass of its own: a 1D field as one device-wide scan,
// rows along x in 2D/3D one warp per row, and columns along y or z in
// 32-point segments (segment totals, a carry scan down every column, then
// the segments again), adjacent threads on adjacent columns.

__global__ void k_residuals(ReconArgs a, uint64_t n)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t c = a.codes[i];
        a.dscr[i] = c ? (int32_t)(c - a.radius) : 0;  // outliers are written by the scatter
    }
}

struct InclusiveOp {  // in-place inclusive scan through the exclusive-scan kernels
    using T = uint32_t;
    uint32_t *v;
    __device__ T load(uint64_t i) const { return v[i]; }
    __device__ void store(uint64_t i, T excl) const { v[i] += excl; }
    __device__ void total(T) const {}
};

__global__ void __launch_bounds__(256) k_scan_rows(uint32_t *v, uint64_t nx, uint64_t nrows)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows; r += nw) {
        uint32_t *row = v + r * nx;
        uint32_t carry = 0;
        for (uint64_t x0 = 0; x0 < nx; x0 += 32) {
            const uint64_t x = x0 + lane;
            uint32_t t = x < nx ? row[x] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= (uint32_t)o) t += u;
            }
            t += carry;
            if (x < nx) row[x] = t;
            carry = __shfl_sync(0xffffffffu, t, 31);
        }
    }
}

constexpr uint32_t kSeg = 32;

// Column geometry: element k of column (o, i) at o * len * s + k * s + i.
struct Cols {
    uint64_t s, len, outer, nseg;
};

__global__ void k_seg_sums(const uint32_t *v, Cols c, uint32_t *tmp)
{
    const uint64_t total = c.outer * c.nseg * c.s, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t i = t % c.s, rest = t / c.s, g = rest % c.nseg, o = rest / c.nseg;
        const uint64_t k0 = g * kSeg, k1 = min(c.len, k0 + kSeg);
        const uint32_t *col = v + o * c.len * c.s + i;
        uint32_t sum = 0;
        for (uint64_t k = k0; k < k1; k++) sum += col[k * c.s];
        tmp[t] = sum;
    }
}

__global__ void k_seg_carry(Cols c, uint32_t *tmp)
{
    const uint64_t total = c.outer * c.s, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t i = t % c.s, o = t / c.s;
        uint32_t *col = tmp + o * c.nseg * c.s + i;
        uint32_t run = 0;
        for (uint64_t g = 0; g < c.nseg; g++) {
            const uint32_t x = col[g * c.s];
            col[g * c.s] = run;
            run += x;
        }
    }
}

__global__ void k_seg_apply(uint32_t *v, Cols c, const uint32_t *tmp)
{
    const uint64_t total = c.outer * c.nseg * c.s, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t i = t % c.s, rest = t / c.s, g = rest % c.nseg, o = rest / c.nseg;
        const uint64_t k0 = g * kSeg, k1 = min(c.len, k0 + kSeg);
        uint32_t *col = v + o * c.len * c.s + i;
        uint32_t run = tmp[t];
        for (uint64_t k = k0; k < k1; k++) {
            run += col[k * c.s];
            col[k * c.s] = run;
        }
    }
}

__global__ void k_dequant(ReconArgs a, uint64_t n)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        a.out[i] = recon_value(a.dscr[i], a.ebx2);
}

int launch_reconstruct_order(const ReconArgs &a, const Geo &g, uint64_t n, cudaStream_t st)
{
    int nl = 0;
    auto grid_for = [&](uint64_t work) {
        return (int)std::max<uint64_t>(1, std::min<uint64_t>((work + 255) / 256, (uint64_t)a.num_sms * 16));
    };
    uint32_t *v = reinterpret_cast<uint32_t *>(a.dscr);
    uint32_t *tmp = v + ((n + 3) & ~3ull);  // the second half of the per-point scratch
    k_residuals<<<grid_for(n), 256, 0, st>>>(a, n);
    nl++;
    if (a.m) {
        k_scatter_outliers<<<grid_for(a.m), 256, 0, st>>>(a, n);
        nl++;
    }
    for (uint32_t pass = 0; pass < a.order; pass++) {
        for (uint32_t d = 0; d < g.ndim; d++) {
            if (g.n[d] < 2) continue;
            if (d == 0 && g.ndim == 1) {
                nl += launch_scan(InclusiveOp{v}, n, a.scan_partial, a.ctl, st);
            } else if (d == 0) {
                const uint64_t rows = n / g.n[0];
                k_scan_rows<<<grid_for(rows * 32), 256, 0, st>>>(v, g.n[0], rows);
                nl++;
            } else {
                Cols c;
                c.s = d == 1 ? g.n[0] : g.n[0] * g.n[1];
                c.len = g.n[d];
                c.outer = n / (c.s * c.len);
                c.nseg = (c.len + kSeg - 1) / kSeg;
                k_seg_sums<<<grid_for(c.outer * c.nseg * c.s), 256, 0, st>>>(v, c, tmp);
                k_seg_carry<<<grid_for(c.outer * c.s), 256, 0, st>>>(c, tmp);
                k_seg_apply<<<grid_for(c.outer * c.nseg * c.s), 256, 0, st>>>(v, c, tmp);
                nl += 3;
            }
        }
    }
    k_dequant<<<grid_for(n), 256, 0, st>>>(a, n);
    nl++;
    if (a.e) {
        k_patch_exceptions<<<grid_for(a.e), 256, 0, st>>>(a, n);
        nl++;
    }
    return nl;
}

// ---------------------------------------------------------------------------
// Grouped reconstruction: every stage of many fields in one launch per
// kernel (variant), each field owning a range of the grid's blocks.

struct RItem {
    ReconArgs a;
    Geo g;
    uint64_t n;
};
struct LineItem {
    Geo g;
    uint32_t *F;
    uint64_t nlines;
    int A, d;
};

__global__ void k_scatter_outliers_group(const RItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    scatter_outliers_body(it.a, it.n, vg);
}

__global__ void k_outlier_tiles_1d_group(const RItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    outlier_tiles_1d_body(it.a, it.n, it.g.ntiles, reinterpret_cast<uint32_t *>(it.a.dscr), vg);
}

__global__ void k_patch_exceptions_group(const RItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    patch_exceptions_body(it.a, it.n, vg);
}

__global__ void __launch_bounds__(k1Threads) k_values_1d_group(const RItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    values_1d_body(it.a, it.g, it.a.faces, reinterpret_cast<const uint32_t *>(it.a.dscr), vg);
}

template <int D>
__global__ void __launch_bounds__(D == 2 ? 256 : 512) k_values_blocked_group(const RItem *items, const uint32_t *first,
                                                                            uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    values_blocked_body<D>(it.a, it.g, vg);
}

template <int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 3 : 6) k_faces_group(const RItem *items, const uint32_t *first,
                                                                      uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    faces_body<TX, TY, TZ, NT>(it.a, it.g, it.a.faces, vg);
}

template <int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 4 : 8) k_values_group(const RItem *items, const uint32_t *first,
                                                                       uint32_t ni)
{
    VGrid vg;
    const RItem &it = items[group_item(first, ni, vg)];
    values_body<TX, TY, TZ, NT>(it.a, it.g, it.a.faces, vg);
}

__global__ void __launch_bounds__(256) k_scan_lines_group(const LineItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const LineItem &it = items[group_item(first, ni, vg)];
    scan_lines_warp_body(it.g, it.A, it.d, it.nlines, it.F, vg);
}

// appends an array to the plan (16-byte aligned); returns its offset
template <typename T> uint64_t plan_put(std::vector<uint8_t> &plan, const std::vector<T> &v)
{
    const uint64_t off = (plan.size() + 15) & ~uint64_t(15);
    plan.resize(off + sizeof(T) * v.size());
    if (!v.empty()) std::memcpy(plan.data() + off, v.data(), sizeof(T) * v.size());
    return off;
}

// one grouped launch: items and their blocks
template <typename T> struct GroupList {
    std::vector<T> items;
    std::vector<uint32_t> first{0};
    void add(const T &it, uint64_t blocks)
    {
        items.push_back(it);
        first.push_back(first.back() + (uint32_t)std::max<uint64_t>(1, blocks));
    }
    bool empty() const { return items.empty(); }
};

}  // namespace

void plan_reconstruct_group(const ReconArgs *ra, uint32_t count, std::vector<uint8_t> &plan,
                            std::vector<GroupLaunch> &launches)
{
    GroupList<RItem> tiles1d, scatter, exc, val1d, blk2, blk3, faces2, faces3, val2, val3;
    GroupList<ScanItem<TileOp>> tscan;
    // one launch per tile-grid dimension: every field's subsets containing it
    // (subsets are separate arrays; each is scanned along its dimensions in
    // increasing order, launch by launch)
    std::vector<GroupList<LineItem>> lines(3);
    for (uint32_t f = 0; f < count; f++) {
        const ReconArgs &a = ra[f];
        const Geo g = make_geo(a.ndim, a.dims);
        const uint64_t n = g.n[0] * g.n[1] * g.n[2];
        const uint64_t sms = (uint64_t)a.num_sms;
        const RItem it{a, g, n};
        if (a.m) {
            const uint64_t grid = std::min<uint64_t>((a.m + 255) / 256, sms * 16);
            (g.ndim == 1 ? tiles1d : scatter).add(it, grid);
        }
        const uint64_t gridt = std::min<uint64_t>(g.ntiles, sms * 8);
        if (a.lblock && g.ndim > 1) {
            const uint32_t B = lorenzo_block_extent(g.ndim);
            uint64_t nb = 1;
            for (uint32_t d = 0; d < g.ndim; d++) nb *= (g.n[d] + B - 1) / B;
            (g.ndim == 2 ? blk2 : blk3).add(it, std::min<uint64_t>(nb, sms * 8));
        } else {
            if (g.ndim == 1) {
                if (!a.lblock)
                    tscan.add(ScanItem<TileOp>{TileOp{a.faces}, g.ntiles, a.scan_partial}, scan_blocks(g.ntiles));
            } else {
                (g.ndim == 2 ? faces2 : faces3).add(it, gridt);
                for (int A = 1; A < 8; A++) {
                    if (!g.size[A]) continue;
                    for (int d = 0; d < (int)g.ndim; d++) {
                        if (!((A >> d) & 1) || g.nt[d] < 2) continue;
                        const uint64_t nlines = g.size[A] * (g.ntiles / g.nt[d]);
                        lines[d].add(LineItem{g, a.faces, nlines, A, d}, std::min<uint64_t>((nlines + 7) / 8, sms * 8));
                    }
                }
            }
            if (g.ndim == 1) {
                const uint64_t blocks = (g.ntiles + k1Threads / 32 - 1) / (k1Threads / 32);
                val1d.add(it, std::min<uint64_t>(blocks, sms * 4));
            } else {
                (g.ndim == 2 ? val2 : val3).add(it, gridt);
            }
        }
        if (a.e) exc.add(it, std::min<uint64_t>((a.e + 255) / 256, sms * 16));
    }
    // launches in stage order; each closure reads its arrays at the plan's device address
    auto emit = [&](auto &list, auto launch) {
        if (list.empty()) return;
        const uint64_t oi = plan_put(plan, list.items), of = plan_put(plan, list.first);
        const uint32_t ni = (uint32_t)list.items.size(), blocks = list.first.back();
        using Item = typename std::remove_reference<decltype(list.items[0])>::type;
        launches.push_back([=](const uint8_t *dev, cudaStream_t st) {
            launch(reinterpret_cast<const Item *>(dev + oi), reinterpret_cast<const uint32_t *>(dev + of), ni, blocks,
                   st);
            return 1;
        });
    };
    emit(tiles1d, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_outlier_tiles_1d_group<<<b, 256, 0, st>>>(i, f, ni);
    });
    emit(scatter, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_scatter_outliers_group<<<b, 256, 0, st>>>(i, f, ni);
    });
    if (!tscan.empty()) {
        const uint64_t oi = plan_put(plan, tscan.items), of = plan_put(plan, tscan.first);
        const uint32_t ni = (uint32_t)tscan.items.size(), blocks = tscan.first.back();
        launches.push_back([=](const uint8_t *dev, cudaStream_t st) {
            return launch_scan_group(reinterpret_cast<const ScanItem<TileOp> *>(dev + oi),
                                     reinterpret_cast<const uint32_t *>(dev + of), ni, blocks, st);
        });
    }
    emit(faces2, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_faces_group<k2TX, k2TY, 1, k2Threads><<<b, k2Threads, 0, st>>>(i, f, ni);
    });
    emit(faces3, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_faces_group<k3TX, k3TY, k3TZ, k3Threads><<<b, k3Threads, 0, st>>>(i, f, ni);
    });
    for (auto &l : lines)
        emit(l, [](const LineItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
            k_scan_lines_group<<<b, 256, 0, st>>>(i, f, ni);
        });
    emit(val1d, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_values_1d_group<<<b, k1Threads, 0, st>>>(i, f, ni);
    });
    emit(val2, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_values_group<k2TX, k2TY, 1, k2Threads><<<b, k2Threads, 0, st>>>(i, f, ni);
    });
    emit(val3, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_values_group<k3TX, k3TY, k3TZ, k3Threads><<<b, k3Threads, 0, st>>>(i, f, ni);
    });
    emit(blk2, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_values_blocked_group<2><<<b, 256, 0, st>>>(i, f, ni);
    });
    emit(blk3, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_values_blocked_group<3><<<b, 512, 0, st>>>(i, f, ni);
    });
    emit(exc, [](const RItem *i, const uint32_t *f, uint32_t ni, uint32_t b, cudaStream_t st) {
        k_patch_exceptions_group<<<b, 256, 0, st>>>(i, f, ni);
    });
}

uint64_t recon_faces_entries(uint32_t ndim, const uint64_t dims[3])
{
    return make_geo(ndim, dims).off[0];
}

void launch_reconstruct(const ReconArgs &a, cudaStream_t st, int *launches)
{
    const Geo g = make_geo(a.ndim, a.dims);
    const uint64_t n = g.n[0] * g.n[1] * g.n[2];
    if (a.order > 1) {
        const int nlo = launch_reconstruct_order(a, g, n, st);
        if (launches) *launches += nlo;
        return;
    }
    int nl = 0;
    uint32_t *start1d = reinterpret_cast<uint32_t *>(a.dscr);  // 1D: per-tile outlier starts
    const uint64_t ngroups = g.ntiles;
    if (a.m) {
        const int grid = (int)std::min<uint64_t>((a.m + 255) / 256, (uint64_t)a.num_sms * 16);
        if (g.ndim == 1) k_outlier_tiles_1d<<<grid, 256, 0, st>>>(a, n, ngroups, start1d);
        else k_scatter_outliers<<<grid, 256, 0, st>>>(a, n);
        nl++;
    }
    const int gridt = (int)std::min<uint64_t>(g.ntiles, (uint64_t)a.num_sms * 8);
    if (a.lblock && g.ndim > 1) {
        // per-block mode: block-local prefix sums, no carries
        const uint32_t B = lorenzo_block_extent(g.ndim);
        uint64_t nb = 1;
        for (uint32_t d = 0; d < g.ndim; d++) nb *= (g.n[d] + B - 1) / B;
        const int gridb = (int)std::min<uint64_t>(nb, (uint64_t)a.num_sms * 8);
        if (g.ndim == 2) k_values_blocked<2><<<gridb, 256, 0, st>>>(a, g);
        else k_values_blocked<3><<<gridb, 512, 0, st>>>(a, g);
        nl++;
    } else {
        if (g.ndim == 1) {
            // tile sums were accumulated by the decoder and the outlier pass
            if (!a.lblock) nl += launch_scan(TileOp{a.faces}, g.ntiles, a.scan_partial, a.ctl, st);
        } else if (g.ndim == 2) {
            k_faces<k2TX, k2TY, 1, k2Threads><<<gridt, k2Threads, 0, st>>>(a, g, a.faces);
            nl++;
        } else {
            k_faces<k3TX, k3TY, k3TZ, k3Threads><<<gridt, k3Threads, 0, st>>>(a, g, a.faces);
            nl++;
        }
        // carry scans: one launch per tile-grid dimension over every subset
        // containing it (a CTA per line when lines are very long)
        for (int d = 0; d < (int)g.ndim && g.ndim > 1; d++) {
            if (g.nt[d] < 2) continue;
            LinePass p{};
            p.g = g;
            p.F = a.faces;
            p.d = d;
            uint64_t nlines = 0;
            for (int A = 1; A < 8; A++) {
                if (!g.size[A] || !((A >> d) & 1)) continue;
                const uint64_t nA = g.size[A] * (g.ntiles / g.nt[d]);
                if (g.nt[d] > 2048) {
                    k_scan_lines_cta<<<(unsigned)nA, 1024, 0, st>>>(g, A, d, a.faces);
                    nl++;
                    continue;
                }
                p.A[p.na] = A;
                p.first[p.na] = nlines;
                p.na++;
                nlines += nA;
            }
            if (p.na == 0) continue;
            p.first[p.na] = nlines;
            if (nlines < (uint64_t)a.num_sms * 256) {
                const uint64_t blocks = (nlines + 7) / 8;  // eight warps per block
                k_scan_pass_warp<<<(unsigned)std::min<uint64_t>(blocks, (uint64_t)a.num_sms * 8), 256, 0, st>>>(p);
            } else {
                k_scan_pass<<<(unsigned)((nlines + 255) / 256), 256, 0, st>>>(p);
            }
            nl++;
        }
        if (g.ndim == 1) {
            // persistent: as many blocks as fit at once
            const uint64_t blocks = (g.ntiles + k1Threads / 32 - 1) / (k1Threads / 32);
            const int grid1 = (int)std::min<uint64_t>(blocks, (uint64_t)a.num_sms * 4);
            k_values_1d<<<grid1, k1Threads, 0, st>>>(a, g, a.faces, start1d);
        } else if (g.ndim == 2) {
            k_values<k2TX, k2TY, 1, k2Threads><<<gridt, k2Threads, 0, st>>>(a, g, a.faces);
        } else {
            k_values<k3TX, k3TY, k3TZ, k3Threads><<<gridt, k3Threads, 0, st>>>(a, g, a.faces);
        }
        nl++;
    }
    nl += launch_exceptions(a, st);
    if (launches) *launches += nl;
}

int launch_exceptions(const ReconArgs &a, cudaStream_t st)
{
    if (!a.e) return 0;
    const Geo g = make_geo(a.ndim, a.dims);
    const uint64_t n = g.n[0] * g.n[1] * g.n[2];
    const int grid = (int)std::min<uint64_t>((a.e + 255) / 256, (uint64_t)a.num_sms * 16);
    k_patch_exceptions<<<grid, 256, 0, st>>>(a, n);
    return 1;
}

}  // namespace gbsz
