// k_quant.cu -- S0 (error bound from the value range) and S1-S3 (prequant,
// Lorenzo prediction, postquant with outliers, fused code histogram).
//
// Paper: Sec. 3.1 (chunking, dual-quantization, Algorithm 2), Lorenzo
// predictor with binomial coefficients (order 1), Sec. 3.2.1 (histogram),
// valrel footnote of Sec. 3.2.2.
//
// Unlike the paper's per-block zero padding, one predictor covers the whole
// field: every tile computes the prequantized integers of a one-point halo on
// its low side itself, so tiles are independent and the output does not
// depend on the tile shape.
#include "common.cuh"

#include <algorithm>

namespace gbsz {

namespace {

// ---------------------------------------------------------------------------
// S0

__device__ __forceinline__ uint32_t ordered_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float key_to_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// eb = rel * (max - min) over finite values (valrel), or the absolute bound;
// 2eb as a float product; 1/(2eb) rounded from double.
__device__ void finalize_eb(Control *ctl, double eb, uint32_t mode, uint32_t kmax, uint32_t kmin_inv)
{
    float e;
    if (mode == 1 && kmax != 0) {
        const float hi = key_to_float(kmax), lo = key_to_float(~kmin_inv);
        const double range = __dsub_rn((double)hi, (double)lo);
        e = range == 0.0 ? __double2float_rn(eb) : __double2float_rn(__dmul_rn(eb, range));
    } else {
        e = __double2float_rn(eb);
    }
    const float e2 = __fmul_rn(e, 2.0f);
    const float inv = __double2float_rn(__ddiv_rn(1.0, (double)e2));
    const bool ok = e > 0.0f && isfinite(e) && isfinite(e2) && isfinite(inv) && inv > 0.0f;
    ctl->eb = e;
    ctl->ebx2 = e2;
    ctl->inv2eb = inv;
    if (!ok) atomicOr(&ctl->error, DERR_EB);
}

// max and min over the finite values: v * 0 + v is v when v is finite and NaN
// for +-Inf and NaN, which fmaxf / fminf ignore (three operations a value).
// A zero may come back as either zero; the range max - min, and so the bound,
// is the same.
__device__ __forceinline__ void mm_update(float v, float &mx, float &mn)
{
    const float w = __fmaf_rn(v, 0.0f, v);
    mx = fmaxf(mx, w);
    mn = fminf(mn, w);
}

template <bool VEC>
__device__ __forceinline__ void minmax_body(const float *__restrict__ x, uint64_t n, Control *ctl, double eb,
                                            uint32_t mode, VGrid vg)
{
    float mx = -INFINITY, mn = INFINITY;
    const uint64_t tid = (uint64_t)vg.bid * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)vg.nb * blockDim.x;
    if (VEC) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const uint64_t n4 = n / 4;
        uint64_t i = tid;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = x4[i + u * stride];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                mm_update(v[u].x, mx, mn);
                mm_update(v[u].y, mx, mn);
                mm_update(v[u].z, mx, mn);
                mm_update(v[u].w, mx, mn);
            }
        }
        for (; i < n4; i += stride) {
            const float4 v = x4[i];
            mm_update(v.x, mx, mn);
            mm_update(v.y, mx, mn);
            mm_update(v.z, mx, mn);
            mm_update(v.w, mx, mn);
        }
        for (uint64_t j = n4 * 4 + tid; j < n; j += stride) mm_update(x[j], mx, mn);
    } else {
        for (uint64_t j = tid; j < n; j += stride) mm_update(x[j], mx, mn);
    }
    // order-preserving keys for the reductions across the grid (0: no finite value)
    uint32_t kmax = mx > -INFINITY ? ordered_key(mx) : 0u, kmin = mn < INFINITY ? ~ordered_key(mn) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        kmin = max(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    }
    __shared__ uint32_t s_max[8], s_min[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_max[warp] = kmax;
        s_min[warp] = kmin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            kmax = max(kmax, s_max[w]);
            kmin = max(kmin, s_min[w]);
        }
        if (kmax) atomicMax(&ctl->max_key, kmax);
        if (kmin) atomicMax(&ctl->min_key_inv, kmin);
        __threadfence();
        s_last = atomicAdd(&ctl->s0_done, 1u) == vg.nb - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const uint32_t km = atomicAdd(&ctl->max_key, 0u);
        const uint32_t kn = atomicAdd(&ctl->min_key_inv, 0u);
        finalize_eb(ctl, eb, mode, km, kn);
    }
}

// 8 blocks per SM resident (at most 32 registers): the grid is 8 blocks per SM
template <bool VEC>
__global__ void __launch_bounds__(256, 8) k_minmax(const float *__restrict__ x, uint64_t n, Control *ctl, double eb,
                                                   uint32_t mode)
{
    minmax_body<VEC>(x, n, ctl, eb, mode, vgrid_self());
}

__global__ void k_eb_abs(Control *ctl, double eb) { finalize_eb(ctl, eb, 0, 0, 0); }

// grouped S0: an absolute bound takes one block (no reduction)
template <bool VEC>
__global__ void __launch_bounds__(256, 8) k_minmax_group(const MinmaxItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const MinmaxItem &m = items[group_item(first, ni, vg)];
    if (m.mode == 0) {
        if (threadIdx.x == 0) finalize_eb(m.ctl, m.eb, 0, 0, 0);
        return;
    }
    minmax_body<VEC>(m.x, m.n, m.ctl, m.eb, m.mode, vg);
}

// ---------------------------------------------------------------------------
// S1-S3 shared pieces

// Histogram: full 2R bins in shared memory when 2R <= kWinBins, else a
// window of kWinBins bins centred on R with global atomics outside it.  The
// centre code R (in the order-n kernel also R-1 and R+1) is counted in
// registers first and reduced per warp at the end.
constexpr uint32_t kWinBins = 8192;

struct HistState {
    uint32_t *sh;   // shared bins
    uint32_t lo;    // first bin held in shared memory
    uint32_t nsh;   // bins held in shared memory
    uint32_t R;
    uint32_t c_lo, c_mid, c_hi;
    uint32_t n_out, n_exc;
    Control *ctl;
};

__device__ __forceinline__ void hist_add(HistState &h, uint32_t code, uint32_t *ghist)
{
    if (code == h.R) {
        h.c_mid++;
    } else if (code == h.R - 1) {
        h.c_lo++;
    } else if (code == h.R + 1) {
        h.c_hi++;
    } else {
        const uint32_t b = code - h.lo;
        if (b < h.nsh) atomicAdd(&h.sh[b], 1u);
        else if (GBSZ_CHECK(code < 2 * h.R, h.ctl)) atomicAdd(&ghist[code], 1u);
    }
}

__device__ __forceinline__ void hist_init(HistState &h, uint32_t *sh, uint32_t R, Control *ctl)
{
    h.ctl = ctl;
    h.sh = sh;
    h.R = R;
    const uint32_t nbins = 2 * R;
    if (nbins <= kWinBins) {
        h.lo = 0;
        h.nsh = nbins;
    } else {
        h.lo = R - kWinBins / 2;
        h.nsh = kWinBins;
    }
    h.c_lo = h.c_mid = h.c_hi = 0;
    h.n_out = h.n_exc = 0;
    for (uint32_t i = threadIdx.x; i < h.nsh; i += blockDim.x) sh[i] = 0;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out_from_bin0: the block's outliers are its shared bin-0 count (every bin
// in shared memory) rather than the per-thread n_out
__device__ void hist_flush(HistState &h, uint32_t *ghist, Control *ctl, bool out_from_bin0 = false)
{
    const uint32_t lo = warp_sum(h.c_lo), mid = warp_sum(h.c_mid), hi = warp_sum(h.c_hi);
    const uint32_t no = warp_sum(h.n_out), ne = warp_sum(h.n_exc);
    __syncthreads();  // every shared atomic of the block has landed
    if ((threadIdx.x & 31) == 0) {
        if (lo) atomicAdd(&h.sh[h.R - 1 - h.lo], lo);
        if (mid) atomicAdd(&h.sh[h.R - h.lo], mid);
        if (hi) atomicAdd(&h.sh[h.R + 1 - h.lo], hi);
        if (no) atomicAdd(&ctl->n_out, (unsigned long long)no);
        if (ne) atomicAdd(&ctl->n_exc, (unsigned long long)ne);
    }
    __syncthreads();
    if (out_from_bin0 && threadIdx.x == 0 && h.sh[0]) atomicAdd(&ctl->n_out, (unsigned long long)h.sh[0]);
    for (uint32_t i = threadIdx.x; i < h.nsh; i += blockDim.x) {
        const uint32_t v = h.sh[i];
        if (v) atomicAdd(&ghist[h.lo + i], v);
    }
}

// emit one point: code, outlier residual, histogram
__device__ __forceinline__ uint32_t emit_point(HistState &h, const QuantArgs &a, uint64_t idx,
                                               uint32_t delta, bool exc)
{
    const uint32_t code = postquant(delta, exc, (int32_t)h.R);
    const bool in = GBSZ_CHECK(idx < npoints(a), a.ctl);
    if (code == 0) {
        if (in) a.dscr[idx] = make_int2((int32_t)delta, exc ? 1 : 0);
        h.n_out++;
    }
    if (exc && in) atomicAdd(&a.unit_exc[idx >> a.unit_shift], 1u);
    h.n_exc += exc;
    hist_add(h, code, a.hist);
    return code;
}

// ---------------------------------------------------------------------------
// 1D: 256 threads, tile of 4096 points, 16 consecutive points per thread
// (four 16-byte loads issued together, two 16-byte code stores).  Each lane
// prequantizes the point before its run itself (one extra point per 16) so
// no lane waits on another.  Point indices fit in 32 bits (n < 2^32).

constexpr int kQ1Threads = 256;
constexpr int kQ1Per = 16;
constexpr int kQ1Tile = kQ1Threads * kQ1Per;

// code for residual d; in cap iff -R < d < R, tested as one unsigned compare
__device__ __forceinline__ uint32_t code_of(uint32_t d, bool exc, uint32_t R)
{
    return (!exc && d + (R - 1) < 2 * R - 1) ? d + R : 0u;
}

// One point of the 1D, 2D and 3D kernels, without branches.  The centre
// code R is counted in a register (added to the thread's count every tile);
// other codes go to the shared bins with a predicated atomic.  (Counting R-1
// and R+1 in registers too, as packed 8-bit fields, cost more instructions
// than their shared atomics: 1D 0.344 -> 0.352 ms at 2^28, 3D 0.463 -> 0.482
// ms at 512^3.)  With every bin
// in shared memory (WIN), the block's outlier count is its bin-0 count, so
// it is not counted here.
template <bool WIN>
__device__ __forceinline__ uint32_t point_1d(HistState &h, const QuantArgs &a, uint32_t idx, uint32_t d, bool exc,
                                             uint32_t &pk)
{
    const uint32_t code = code_of(d, exc, h.R);
    const bool central = code == h.R;
    pk += central ? 1u : 0u;
    if (WIN) {
        // predicated shared-memory add: no branch around it
        const uint32_t addr = (uint32_t)__cvta_generic_to_shared(h.sh + code);
        const bool add = !central && GBSZ_CHECK(code < h.nsh, a.ctl);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.u32 p, %0, 0;\n\t"
            "@p red.shared.add.u32 [%1], 1;\n\t}" ::"r"((uint32_t)add),
            "r"(addr)
            : "memory");
    } else if (!central) {
        const uint32_t b = code - h.lo;
        if (b < h.nsh) atomicAdd(&h.sh[b], 1u);
        else if (GBSZ_CHECK(code < 2 * h.R, a.ctl)) atomicAdd(&a.hist[code], 1u);
        h.n_out += code == 0;
    }
    if (code == 0 && GBSZ_CHECK(idx < npoints(a), a.ctl)) a.dscr[idx] = make_int2((int32_t)d, exc ? 1 : 0);
    h.n_exc += exc;
    return code;
}

__device__ __forceinline__ void unpack_central(HistState &h, uint32_t &pk)
{
    h.c_mid += pk;
    pk = 0;
}

template <bool VEC, bool WIN>
__device__ __forceinline__ void dualquant_1d_body(const QuantArgs &a, uint32_t ntiles, VGrid vg)
{
    extern __shared__ uint32_t sh_hist[];
    HistState h;
    hist_init(h, sh_hist, a.radius, a.ctl);
    __syncthreads();
    if (a.ctl->error & DERR_EB) return;
    const EbScalars sc = load_scalars(a.ctl);
    const uint32_t n = (uint32_t)a.dims[0];
    for (uint32_t tile = vg.bid; tile < ntiles; tile += vg.nb) {
        const uint32_t e0 = tile * kQ1Tile + threadIdx.x * kQ1Per;
        float v[kQ1Per];
        float vp = 0.0f;
        const bool full = VEC && (uint64_t)e0 + kQ1Per <= n;
        if (full) {
            const float4 *p = reinterpret_cast<const float4 *>(a.x + e0);
#pragma unroll
            for (int j = 0; j < kQ1Per / 4; j++) {
                const float4 f = p[j];
                v[4 * j] = f.x;
                v[4 * j + 1] = f.y;
                v[4 * j + 2] = f.z;
                v[4 * j + 3] = f.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kQ1Per; j++) v[j] = e0 + j < n ? a.x[e0 + j] : 0.0f;
        }
        // the point before the run predicts its first point, unless that one
        // starts a block of the per-block mode (its neighbour is padding)
        const bool has_prev = e0 > 0 && e0 <= n && !(a.lblock && e0 % lorenzo_block_extent(1) == 0);
        if (has_prev) vp = a.x[e0 - 1];
        bool dummy;
        uint32_t qprev = has_prev ? (uint32_t)prequant(vp, sc, dummy) : 0u;
        uint32_t code[kQ1Per];
        uint32_t pk = 0;
        const uint32_t exc0 = h.n_exc;  // this run's exceptions go to its encoder unit below
        if (full) {
            // the prequant fast path for all 16 points; the few it cannot
            // decide (near a rounding tie, huge, non-finite) are redone with
            // the full watchdog in a branch the warp rarely takes
            uint32_t q[kQ1Per], slow = 0, excm = 0;
#pragma unroll
            for (int j = 0; j < kQ1Per; j++) {
                bool ok;
                q[j] = (uint32_t)prequant_fast(v[j], sc, ok);
                slow |= (ok ? 0u : 1u) << j;
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < kQ1Per; j++) {
                    if (slow & (1u << j)) {
                        bool exc;
                        q[j] = (uint32_t)prequant_full(v[j], sc, exc);
                        excm |= (exc ? 1u : 0u) << j;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kQ1Per; j++) {
                code[j] = point_1d<WIN>(h, a, e0 + j, q[j] - qprev, (excm >> j) & 1u, pk);
                qprev = q[j];
            }
            // chunks are multiples of the run: only a run's last point can precede a chunk
            if (a.anchors && ((e0 + kQ1Per) & (a.chunk - 1)) == 0 && e0 + kQ1Per < n &&
                GBSZ_CHECK((e0 + kQ1Per) / a.chunk < (n + a.chunk - 1) / a.chunk, a.ctl))
                a.anchors[(e0 + kQ1Per) / a.chunk] = qprev;
            if (a.anchors && e0 == 0) a.anchors[0] = 0u;
            uint4 *o = reinterpret_cast<uint4 *>(a.codes + e0);
            if (GBSZ_CHECK(e0 + kQ1Per <= n, a.ctl)) {
            o[0] = make_uint4(code[0] | (code[1] << 16), code[2] | (code[3] << 16), code[4] | (code[5] << 16),
                              code[6] | (code[7] << 16));
            o[1] = make_uint4(code[8] | (code[9] << 16), code[10] | (code[11] << 16), code[12] | (code[13] << 16),
                              code[14] | (code[15] << 16));
            }
        } else {
#pragma unroll
            for (int j = 0; j < kQ1Per; j++) {
                bool exc;
                const uint32_t q = (uint32_t)prequant(v[j], sc, exc);
                if (e0 + j < n) a.codes[e0 + j] = (uint16_t)point_1d<WIN>(h, a, e0 + j, q - qprev, exc, pk);
                qprev = q;
                const uint64_t nxt = (uint64_t)e0 + j + 1;
                if (a.anchors && nxt < n && (nxt & (a.chunk - 1)) == 0 &&
                    GBSZ_CHECK(nxt / a.chunk < ((uint64_t)n + a.chunk - 1) / a.chunk, a.ctl))
                    a.anchors[nxt / a.chunk] = q;
            }
            if (a.anchors && e0 == 0) a.anchors[0] = 0u;
        }
        unpack_central(h, pk);
        // the 16 points of a run lie in one encoder unit (units are 2^k >= 2048 points)
        if (h.n_exc != exc0 && GBSZ_CHECK(e0 < n, a.ctl)) atomicAdd(&a.unit_exc[e0 >> a.unit_shift], h.n_exc - exc0);
    }
    if (WIN) h.n_out = 0;  // taken from bin 0 below
    hist_flush(h, a.hist, a.ctl, WIN);
}

// four blocks per SM resident (at most 64 registers)
template <bool VEC, bool WIN>
__global__ void __launch_bounds__(kQ1Threads, 4) k_dualquant_1d(const __grid_constant__ QuantArgs a, uint32_t ntiles)
{
    dualquant_1d_body<VEC, WIN>(a, ntiles, vgrid_self());
}

// ---------------------------------------------------------------------------
// 2D: 128 threads; tile 512 (x) x ty (y, 8 unless set) swept row by row.  Each thread holds
// 4 points of a row (x = x0 + tid + 128 j).  Three row buffers of prequantized
// integers in shared memory (slot 0 = the halo column x0 - 1); the next row's
// floats are prefetched into registers while the current row is processed.

constexpr int kQ2Threads = 128;
constexpr int kQ2TX = 512;
constexpr int kQ2TY = 8;

template <bool WIN>
__device__ __forceinline__ void dualquant_2d_body(const QuantArgs &a, uint32_t ntx, uint32_t nty, uint32_t ty,
                                                  VGrid vg)
{
    extern __shared__ uint32_t sh_hist[];
    __shared__ int32_t rows[3][kQ2TX + 1];
    HistState h;
    hist_init(h, sh_hist, a.radius, a.ctl);
    __syncthreads();
    if (a.ctl->error & DERR_EB) return;
    const EbScalars sc = load_scalars(a.ctl);
    // point indices fit in 32 bits (n < 2^32)
    const uint32_t nx = (uint32_t)a.dims[0], ny = (uint32_t)a.dims[1];
    const uint32_t ntiles = ntx * nty;
    constexpr uint32_t B2 = lorenzo_block_extent(2);
    int buf = 0;
    for (uint32_t tile = vg.bid; tile < ntiles; tile += vg.nb) {
        const uint32_t x0 = (tile % ntx) * kQ2TX;
        const int y0 = (int)((tile / ntx) * ty);
        const int y1 = (int)min(ny, (uint32_t)y0 + ty);
        // per-block mode: neighbours across a block edge are padding (0)
        uint32_t mL[4];
        bool inx[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t x = x0 + threadIdx.x + 128u * j;
            mL[j] = (a.lblock && x % B2 == 0) ? 0u : ~0u;
            inx[j] = x < nx;
        }
        float cur[4], nxt[4], hcur = 0.0f, hnxt = 0.0f;
        auto load_row = [&](int y, float *v, float &hv) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t x = x0 + threadIdx.x + 128u * j;
                v[j] = (y >= 0 && inx[j]) ? a.x[(uint32_t)y * nx + x] : 0.0f;
            }
            if (threadIdx.x == 0) hv = (y >= 0 && x0 > 0) ? a.x[(uint32_t)y * nx + x0 - 1] : 0.0f;
        };
        load_row(y0 - 1, cur, hcur);
        for (int y = y0 - 1; y < y1; y++) {
            if (y + 1 < y1) load_row(y + 1, nxt, hnxt);
            // the prequant fast path for the row's points; the few it cannot
            // decide take the full watchdog in a branch the warp rarely enters
            int32_t q[4];
            bool ex[4];
            uint32_t slow = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                q[j] = 0;
                ex[j] = false;
                if (y >= 0 && inx[j]) {
                    bool ok;
                    q[j] = prequant_fast(cur[j], sc, ok);
                    slow |= (ok ? 0u : 1u) << j;
                }
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (slow & (1u << j)) q[j] = prequant_full(cur[j], sc, ex[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) rows[buf][1 + threadIdx.x + 128 * j] = q[j];
            if (threadIdx.x == 0) {
                bool dummy;
                rows[buf][0] = (y >= 0 && x0 > 0) ? prequant(hcur, sc, dummy) : 0;
            }
            __syncthreads();
            if (y >= y0) {
                const int prev = buf == 0 ? 2 : buf - 1;
                const uint32_t mU = (a.lblock && (uint32_t)y % B2 == 0) ? 0u : ~0u;
                uint32_t pk = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const uint32_t lx = threadIdx.x + 128u * j;
                    if (inx[j]) {
                        const uint32_t d = (uint32_t)q[j] - ((uint32_t)rows[buf][lx] & mL[j]) -
                                           ((uint32_t)rows[prev][lx + 1] & mU) +
                                           ((uint32_t)rows[prev][lx] & mL[j] & mU);
                        const uint32_t idx = (uint32_t)y * nx + x0 + lx;
                        const uint32_t cd = point_1d<WIN>(h, a, idx, d, ex[j], pk);
                        if (GBSZ_CHECK(idx < npoints(a), a.ctl)) {
                            a.codes[idx] = (uint16_t)cd;
                            if (ex[j]) atomicAdd(&a.unit_exc[idx >> a.unit_shift], 1u);
                        }
                    }
                }
                unpack_central(h, pk);
            }
            buf = buf == 2 ? 0 : buf + 1;
#pragma unroll
            for (int j = 0; j < 4; j++) cur[j] = nxt[j];
            hcur = hnxt;
        }
    }
    if (WIN) h.n_out = 0;  // taken from bin 0 below
    hist_flush(h, a.hist, a.ctl, WIN);
}

template <bool WIN>
__global__ void __launch_bounds__(kQ2Threads) k_dualquant_2d(const __grid_constant__ QuantArgs a, uint32_t ntx,
                                                             uint32_t nty, uint32_t ty)
{
    dualquant_2d_body<WIN>(a, ntx, nty, ty, vgrid_self());
}

// ---------------------------------------------------------------------------
// 3D: 256 threads; tile 32 (x) x 32 (y) swept along z over tz planes.  Thread
// (lx = tid % 32, ly = tid / 32 + 8 j) holds 4 points of a plane.  Threads
// 0..64 also prequantize one halo point each: the column x0 - 1 for
// y0-1..y0+31 and the row y0 - 1 for x0..x0+31.  The 3D Lorenzo residual is
// taken as its separable form: the z-difference r = q(z) - q(z-1) of each
// point comes from the thread's own previous integer (a register), and the
// residual is the 2D Lorenzo stencil of r in the plane,
//   d = r(x,y) - r(x-1,y) - r(x,y-1) + r(x-1,y-1),
// which expands to the eight-term stencil exactly (modulo 2^32), masks of
// the per-block mode included.  Two plane buffers of r, one barrier a plane.

constexpr int kQ3Threads = 256;
constexpr int kQ3T = 32;

template <bool WIN>
__device__ __forceinline__ void dualquant_3d_body(const QuantArgs &a, uint32_t ntx, uint32_t nty, uint32_t ntz,
                                                  uint32_t tz, VGrid vg)
{
    extern __shared__ uint32_t sh_hist[];
    __shared__ uint32_t rp[2][kQ3T + 1][kQ3T + 1];
    HistState h;
    hist_init(h, sh_hist, a.radius, a.ctl);
    __syncthreads();
    if (a.ctl->error & DERR_EB) return;
    const EbScalars sc = load_scalars(a.ctl);
    // point indices fit in 32 bits (n < 2^32)
    const uint32_t nx = (uint32_t)a.dims[0], ny = (uint32_t)a.dims[1], nz = (uint32_t)a.dims[2];
    const uint32_t ntiles = ntx * nty * ntz;
    const int lx = threadIdx.x & 31, ly0 = threadIdx.x >> 5;
    constexpr uint32_t B3 = lorenzo_block_extent(3);
    // halo point of this thread (if any), as plane-local coordinates (+1 offset)
    int hx = -2, hy = -2;
    if (threadIdx.x < 33) {
        hx = -1;
        hy = (int)threadIdx.x - 1;
    } else if (threadIdx.x < 65) {
        hx = (int)threadIdx.x - 33;
        hy = -1;
    }
    int buf = 0;
    for (uint32_t tile = vg.bid; tile < ntiles; tile += vg.nb) {
        const uint32_t x0 = (tile % ntx) * kQ3T, y0 = ((tile / ntx) % nty) * kQ3T;
        const int z0 = (int)((tile / (ntx * nty)) * tz), z1 = (int)min(nz, (uint32_t)z0 + tz);
        const uint32_t gx = x0 + lx;
        const int ghx = (int)x0 + hx, ghy = (int)y0 + hy;
        const bool has_halo = hx > -2;
        const bool halo_in = has_halo && ghx >= 0 && ghy >= 0 && (uint32_t)ghx < nx && (uint32_t)ghy < ny;
        // per-block mode: neighbours across a block face are padding (0)
        const uint32_t mL = (a.lblock && gx % B3 == 0) ? 0u : ~0u;
        uint32_t mU[4];
        bool inpt[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t gy = y0 + ly0 + 8 * j;
            mU[j] = (a.lblock && gy % B3 == 0) ? 0u : ~0u;
            inpt[j] = gx < nx && gy < ny;
        }
        float cur[4], nxt[4], hcur = 0.0f, hnxt = 0.0f;
        auto load_plane = [&](int z, float *v, float &hv) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t gy = y0 + ly0 + 8 * j;
                v[j] = (z >= 0 && inpt[j]) ? a.x[((uint32_t)z * ny + gy) * nx + gx] : 0.0f;
            }
            hv = (z >= 0 && halo_in) ? a.x[((uint32_t)z * ny + (uint32_t)ghy) * nx + (uint32_t)ghx] : 0.0f;
        };
        load_plane(z0 - 1, cur, hcur);
        uint32_t qprev[4] = {0u, 0u, 0u, 0u}, hprev = 0u;  // integers of the plane before (0 outside)
        for (int z = z0 - 1; z < z1; z++) {
            if (z + 1 < z1) load_plane(z + 1, nxt, hnxt);
            // the prequant fast path for the plane's points and the halo
            // point; the few it cannot decide take the full watchdog in a
            // branch the warp rarely enters
            uint32_t q[4], hq = 0u, slow = 0;
            bool ex[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                q[j] = 0u;
                ex[j] = false;
                if (z >= 0 && inpt[j]) {
                    bool ok;
                    q[j] = (uint32_t)prequant_fast(cur[j], sc, ok);
                    slow |= (ok ? 0u : 1u) << j;
                }
            }
            if (z >= 0 && halo_in) {
                bool ok;
                hq = (uint32_t)prequant_fast(hcur, sc, ok);
                slow |= (ok ? 0u : 1u) << 4;
            }
            if (slow) {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (slow & (1u << j)) q[j] = (uint32_t)prequant_full(cur[j], sc, ex[j]);
                if (slow & 16u) {
                    bool dummy;
                    hq = (uint32_t)prequant_full(hcur, sc, dummy);
                }
            }
            if (z >= z0) {
                const uint32_t mB = (a.lblock && (uint32_t)z % B3 == 0) ? 0u : ~0u;
                uint32_t(*c)[kQ3T + 1] = rp[buf];
                uint32_t r[4];
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    r[j] = q[j] - (qprev[j] & mB);
                    c[ly0 + 8 * j + 1][lx + 1] = r[j];
                }
                if (has_halo) c[hy + 1][hx + 1] = hq - (hprev & mB);
                __syncthreads();
                const int X = lx + 1;
                uint32_t pk = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int Y = ly0 + 8 * j + 1;
                    if (inpt[j]) {
                        const uint32_t d = r[j] - (c[Y][X - 1] & mL) - (c[Y - 1][X] & mU[j]) +
                                           (c[Y - 1][X - 1] & mL & mU[j]);
                        const uint32_t idx = ((uint32_t)z * ny + (y0 + Y - 1)) * nx + gx;
                        const uint32_t cd = point_1d<WIN>(h, a, idx, d, ex[j], pk);
                        if (GBSZ_CHECK(idx < npoints(a), a.ctl)) {
                            a.codes[idx] = (uint16_t)cd;
                            if (ex[j]) atomicAdd(&a.unit_exc[idx >> a.unit_shift], 1u);
                        }
                    }
                }
                unpack_central(h, pk);
                buf ^= 1;
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                qprev[j] = q[j];
                cur[j] = nxt[j];
            }
            hprev = hq;
            hcur = hnxt;
        }
    }
    if (WIN) h.n_out = 0;  // taken from bin 0 below
    hist_flush(h, a.hist, a.ctl, WIN);
}

template <bool WIN>
__global__ void __launch_bounds__(kQ3Threads, 5) k_dualquant_3d(const __grid_constant__ QuantArgs a, uint32_t ntx,
                                                             uint32_t nty, uint32_t ntz, uint32_t tz)
{
    dualquant_3d_body<WIN>(a, ntx, nty, ntz, tz, vgrid_self());
}

// grouped S1-S3: one launch per kernel variant over every field of the
// variant (D = 1, 2, 3; VEC for D = 1)
template <int D, bool VEC, bool WIN>
__global__ void __launch_bounds__(D == 1 ? kQ1Threads : D == 2 ? kQ2Threads : kQ3Threads, D == 1 ? 3 : 1)
    k_dualquant_group(const QuantItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const QuantItem &q = items[group_item(first, ni, vg)];
    if (D == 1) dualquant_1d_body<VEC, WIN>(q.a, q.t[0], vg);
    else if (D == 2) dualquant_2d_body<WIN>(q.a, q.t[0], q.t[1], q.t[2], vg);
    else dualquant_3d_body<WIN>(q.a, q.t[0], q.t[1], q.t[2], q.t[3], vg);
}

// ---------------------------------------------------------------------------
// Order n > 1 (Lorenzo predictor with binomial coefficients, Sec. 3.1.2).
// The prequantized integers go to a scratch copy first, exceptions to a bit
// mask; a second kernel evaluates the stencil of all (n+1)^d - 1 earlier
// neighbours of every point from that copy, with zeros outside the field.
// The neighbour k steps back weighs -prod_j (-1)^k_j C(n, k_j): the
// expansion of 1 - prod_j (1 - S_j)^n, so the residual is the n-th
// difference along every dimension.  One thread per point; the neighbours
// are re-read through L1/L2.

__global__ void __launch_bounds__(256) k_prequant_int(QuantArgs a, uint64_t n)
{
    if (a.ctl->error & DERR_EB) return;
    const EbScalars sc = load_scalars(a.ctl);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        bool ex;
        a.qint[i] = prequant(a.x[i], sc, ex);
        if (ex) atomicOr(&a.excm[i >> 5], 1u << (i & 31));
    }
}

__host__ __device__ constexpr uint32_t binom_c(uint32_t n, uint32_t k)
{
    return k == 0 ? 1u : binom_c(n, k - 1) * (n - k + 1) / k;
}

template <int D, int ORDER>
__global__ void __launch_bounds__(256) k_lorenzo_order(QuantArgs a, uint32_t n)
{
    extern __shared__ uint32_t sh_hist[];
    HistState h;
    hist_init(h, sh_hist, a.radius, a.ctl);
    __syncthreads();
    if (a.ctl->error & DERR_EB) return;
    const uint32_t nx = (uint32_t)a.dims[0], ny = D >= 2 ? (uint32_t)a.dims[1] : 1u;
    const uint32_t sz = nx * ny;  // below 2^32 as n is
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i64 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i64 < n; i64 += stride) {
        const uint32_t i = (uint32_t)i64;
        const uint32_t x = i % nx, r = i / nx;
        const uint32_t y = D >= 2 ? r % ny : 0u, z = D >= 3 ? r / ny : 0u;
        uint32_t p = 0;
#pragma unroll
        for (int kz = 0; kz <= (D >= 3 ? ORDER : 0); kz++)
#pragma unroll
            for (int ky = 0; ky <= (D >= 2 ? ORDER : 0); ky++)
#pragma unroll
                for (int kx = 0; kx <= ORDER; kx++) {
                    if (kx + ky + kz == 0) continue;
                    if ((uint32_t)kx > x || (uint32_t)ky > y || (uint32_t)kz > z) continue;
                    const uint32_t c = binom_c(ORDER, kx) * binom_c(ORDER, ky) * binom_c(ORDER, kz);
                    const uint32_t v = (uint32_t)a.qint[i - kx - ky * nx - kz * sz] * c;
                    p = ((kx + ky + kz) & 1) ? p + v : p - v;
                }
        const bool ex = (a.excm[i >> 5] >> (i & 31)) & 1u;
        a.codes[i] = (uint16_t)emit_point(h, a, i, (uint32_t)a.qint[i] - p, ex);
    }
    hist_flush(h, a.hist, a.ctl);
}

template <int D>
void launch_order(const QuantArgs &a, uint32_t n, int grid, size_t hist_bytes, cudaStream_t st)
{
    if (a.order == 2) k_lorenzo_order<D, 2><<<grid, 256, hist_bytes, st>>>(a, n);
    else k_lorenzo_order<D, 3><<<grid, 256, hist_bytes, st>>>(a, n);
}

}  // namespace

void launch_minmax_eb(const float *x, uint64_t n, Control *ctl, double eb, uint32_t mode, int num_sms,
                      cudaStream_t st)
{
    if (mode == 0) {
        k_eb_abs<<<1, 1, 0, st>>>(ctl, eb);
        return;
    }
    const uint64_t need = (n / 4 + 255) / 256;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms * 8));
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0)
        k_minmax<true><<<grid, 256, 0, st>>>(x, n, ctl, eb, mode);
    else
        k_minmax<false><<<grid, 256, 0, st>>>(x, n, ctl, eb, mode);
}

uint32_t minmax_blocks(uint64_t n, uint32_t mode, int num_sms)
{
    if (mode == 0) return 1;
    const uint64_t need = (n / 4 + 255) / 256;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms * 8));
}

void launch_minmax_group(const MinmaxItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks, bool vec,
                         cudaStream_t st)
{
    if (vec) k_minmax_group<true><<<blocks, 256, 0, st>>>(items, first, ni);
    else k_minmax_group<false><<<blocks, 256, 0, st>>>(items, first, ni);
}

// 2D tiles: t = {tiles along x, tiles along y, rows per tile}
static void tiles_2d(const QuantArgs &a, uint32_t t[4])
{
    const uint32_t ty = a.slab ? a.slab : (uint32_t)kQ2TY;
    t[0] = (uint32_t)((a.dims[0] + kQ2TX - 1) / kQ2TX);
    t[1] = (uint32_t)((a.dims[1] + ty - 1) / ty);
    t[2] = ty;
    t[3] = 0;
}

// 3D tiles: t = {tiles along x, y, z, planes per tile}; by default the
// planes halve from the whole depth until there are 8 tiles per SM (or 4 planes)
static void tiles_3d(const QuantArgs &a, uint32_t t[4])
{
    const uint32_t ntx = (uint32_t)((a.dims[0] + kQ3T - 1) / kQ3T);
    const uint32_t nty = (uint32_t)((a.dims[1] + kQ3T - 1) / kQ3T);
    const uint64_t nz = a.dims[2];
    uint64_t tz = nz;
    if (a.slab) {
        tz = std::min<uint64_t>(a.slab, nz);
    } else {
        while (tz > 4 && (uint64_t)ntx * nty * ((nz + tz - 1) / tz) < (uint64_t)a.num_sms * 8) tz = (tz + 1) / 2;
    }
    t[0] = ntx;
    t[1] = nty;
    t[2] = (uint32_t)((nz + tz - 1) / tz);
    t[3] = (uint32_t)tz;
}

uint32_t dualquant_plan(const QuantArgs &a, uint32_t t[4], int *variant, size_t *smem)
{
    const uint32_t nbins = 2 * a.radius;
    const bool win = nbins <= kWinBins;
    *smem = sizeof(uint32_t) * std::min<uint32_t>(nbins, kWinBins);
    t[0] = t[1] = t[2] = t[3] = 0;
    if (a.ndim == 1) {
        const uint64_t n = a.dims[0];
        t[0] = (uint32_t)((n + kQ1Tile - 1) / kQ1Tile);
        const bool vec = (reinterpret_cast<uintptr_t>(a.x) & 15) == 0;
        *variant = 4 + (vec ? 2 : 0) + (win ? 1 : 0);
        return (uint32_t)std::min<uint64_t>(t[0], (uint64_t)a.num_sms * 8);
    }
    if (a.ndim == 2) {
        tiles_2d(a, t);
        *variant = 8 + (win ? 1 : 0);
        return (uint32_t)std::min<uint64_t>((uint64_t)t[0] * t[1], (uint64_t)a.num_sms * 12);
    }
    tiles_3d(a, t);
    *variant = 12 + (win ? 1 : 0);
    return (uint32_t)std::min<uint64_t>((uint64_t)t[0] * t[1] * t[2], (uint64_t)a.num_sms * 8);
}

void launch_dualquant_group(int variant, const QuantItem *items, const uint32_t *first, uint32_t ni,
                            uint32_t blocks, size_t smem, cudaStream_t st)
{
    switch (variant) {
    case 4: k_dualquant_group<1, false, false><<<blocks, kQ1Threads, smem, st>>>(items, first, ni); break;
    case 5: k_dualquant_group<1, false, true><<<blocks, kQ1Threads, smem, st>>>(items, first, ni); break;
    case 6: k_dualquant_group<1, true, false><<<blocks, kQ1Threads, smem, st>>>(items, first, ni); break;
    case 7: k_dualquant_group<1, true, true><<<blocks, kQ1Threads, smem, st>>>(items, first, ni); break;
    case 8: k_dualquant_group<2, false, false><<<blocks, kQ2Threads, smem, st>>>(items, first, ni); break;
    case 9: k_dualquant_group<2, false, true><<<blocks, kQ2Threads, smem, st>>>(items, first, ni); break;
    case 12: k_dualquant_group<3, false, false><<<blocks, kQ3Threads, smem, st>>>(items, first, ni); break;
    case 13: k_dualquant_group<3, false, true><<<blocks, kQ3Threads, smem, st>>>(items, first, ni); break;
    default: break;
    }
}

int launch_dualquant(const QuantArgs &a, cudaStream_t st)
{
    const uint32_t nbins = 2 * a.radius;
    const size_t hist_bytes = sizeof(uint32_t) * std::min<uint32_t>(nbins, kWinBins);
    if (a.order > 1) {
        const uint64_t n = a.dims[0] * a.dims[1] * a.dims[2];
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)a.num_sms * 8));
        k_prequant_int<<<grid, 256, 0, st>>>(a, n);
        if (a.ndim == 1) launch_order<1>(a, (uint32_t)n, grid, hist_bytes, st);
        else if (a.ndim == 2) launch_order<2>(a, (uint32_t)n, grid, hist_bytes, st);
        else launch_order<3>(a, (uint32_t)n, grid, hist_bytes, st);
        return 2;
    }
    if (a.ndim == 1) {
        const uint64_t n = a.dims[0];
        const uint32_t ntiles = (uint32_t)((n + kQ1Tile - 1) / kQ1Tile);
        const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)a.num_sms * 8);
        const bool vec = (reinterpret_cast<uintptr_t>(a.x) & 15) == 0, win = nbins <= kWinBins;
        if (vec && win) k_dualquant_1d<true, true><<<grid, kQ1Threads, hist_bytes, st>>>(a, ntiles);
        else if (vec) k_dualquant_1d<true, false><<<grid, kQ1Threads, hist_bytes, st>>>(a, ntiles);
        else if (win) k_dualquant_1d<false, true><<<grid, kQ1Threads, hist_bytes, st>>>(a, ntiles);
        else k_dualquant_1d<false, false><<<grid, kQ1Threads, hist_bytes, st>>>(a, ntiles);
    } else if (a.ndim == 2) {
        uint32_t t[4];
        tiles_2d(a, t);
        const uint64_t ntiles = (uint64_t)t[0] * t[1];
        const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)a.num_sms * 12);
        if (nbins <= kWinBins) k_dualquant_2d<true><<<grid, kQ2Threads, hist_bytes, st>>>(a, t[0], t[1], t[2]);
        else k_dualquant_2d<false><<<grid, kQ2Threads, hist_bytes, st>>>(a, t[0], t[1], t[2]);
    } else {
        uint32_t t[4];
        tiles_3d(a, t);
        const uint64_t ntiles = (uint64_t)t[0] * t[1] * t[2];
        const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)a.num_sms * 8);
        if (nbins <= kWinBins) k_dualquant_3d<true><<<grid, kQ3Threads, hist_bytes, st>>>(a, t[0], t[1], t[2], t[3]);
        else k_dualquant_3d<false><<<grid, kQ3Threads, hist_bytes, st>>>(a, t[0], t[1], t[2], t[3]);
    }
    return 1;
}

}  // namespace gbsz
