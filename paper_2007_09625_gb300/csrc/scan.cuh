// scan.cuh -- device-wide exclusive prefix sums (chunk word offsets, encoder
// unit offsets, 1D tile carries, the outlier residuals' prefix).  A single
// call is one kernel: every block scans a tile of kScanBlock entries, takes
// the tiles before it from a decoupled look-back (tiles are taken in order
// from a ticket, so a block waits only on tiles held by blocks already
// running; the wait gives up after 1 s and reports a timeout) and writes its
// results.  Grouped batches use three coalesced kernels per scan instead
// (block reduce -> scan of block totals -> block scan plus carry), with no
// inter-CTA waiting.
#pragma once

#include "common.cuh"

namespace gbsz {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 8;
constexpr uint64_t kScanBlock = (uint64_t)kScanThreads * kScanPer;

__device__ __forceinline__ uint32_t block_excl_scan_t(uint32_t v, void *sh, uint32_t *tot)
{
    return block_excl_scan(v, static_cast<uint32_t *>(sh), tot);
}
__device__ __forceinline__ unsigned long long block_excl_scan_t(unsigned long long v, void *sh,
                                                                unsigned long long *tot)
{
    return block_excl_scan64(v, static_cast<unsigned long long *>(sh), tot);
}

__device__ __forceinline__ ulonglong2 operator+(ulonglong2 a, ulonglong2 b)
{
    return make_ulonglong2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ ulonglong2 &operator+=(ulonglong2 &a, ulonglong2 b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}
// pair scan: two 64-bit scans sharing the synchronisation (sh: 66 entries)
__device__ __forceinline__ ulonglong2 block_excl_scan_t(ulonglong2 v, void *sh, ulonglong2 *tot)
{
    unsigned long long *s = static_cast<unsigned long long *>(sh);
    unsigned long long tx, ty;
    const unsigned long long ex = block_excl_scan64(v.x, s, &tx);
    const unsigned long long ey = block_excl_scan64(v.y, s + 33, &ty);
    *tot = make_ulonglong2(tx, ty);
    return make_ulonglong2(ex, ey);
}

template <typename T> __device__ __forceinline__ T scan_zero() { return T(0); }
template <> __device__ __forceinline__ ulonglong2 scan_zero<ulonglong2>() { return make_ulonglong2(0, 0); }

// Op provides: using T; T load(uint64_t i) const; void store(uint64_t i, T v) const;
// void check(uint64_t i) const (optional validation, may be empty)
template <typename Op>
__device__ __forceinline__ void scan_reduce_body(const Op &op, uint64_t n, typename Op::T *partial, uint32_t bid)
{
    using T = typename Op::T;
    __shared__ unsigned long long sh[66];
    const uint64_t base = bid * kScanBlock + (uint64_t)threadIdx.x * kScanPer;
    T s = scan_zero<T>();
#pragma unroll
    for (int j = 0; j < kScanPer; j++)
        if (base + j < n) s += op.load(base + j);
    T tot;
    block_excl_scan_t(s, sh, &tot);
    if (threadIdx.x == 0) partial[bid] = tot;
}

template <typename Op>
__device__ __forceinline__ void scan_top_body(const Op &op, uint64_t nb, typename Op::T *partial)
{
    using T = typename Op::T;
    __shared__ unsigned long long sh[66];
    const uint64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = min(nb, threadIdx.x * per), hi = min(nb, lo + per);
    T s = scan_zero<T>();
    for (uint64_t i = lo; i < hi; i++) s += partial[i];
    T tot;
    T run = block_excl_scan_t(s, sh, &tot);
    for (uint64_t i = lo; i < hi; i++) {
        const T v = partial[i];
        partial[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) op.total(tot);
}

template <typename Op>
__device__ __forceinline__ void scan_apply_body(const Op &op, uint64_t n, const typename Op::T *partial, uint32_t bid)
{
    using T = typename Op::T;
    __shared__ unsigned long long sh[66];
    const uint64_t base = bid * kScanBlock + (uint64_t)threadIdx.x * kScanPer;
    T v[kScanPer];
    T s = scan_zero<T>();
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        v[j] = base + j < n ? op.load(base + j) : scan_zero<T>();
        s += v[j];
    }
    T tot;
    T run = block_excl_scan_t(s, sh, &tot) + partial[bid];
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        if (base + j < n) op.store(base + j, run);
        run += v[j];
    }
}

// The single-pass scan's state in the partial scratch: a ticket word, one
// flag per tile (0 none, 1 its total, 2 the total of every tile up to it),
// then the tiles' totals and inclusive totals.
__host__ __device__ inline uint64_t scan_flag_bytes(uint64_t nb) { return 16 + ((4 * nb + 15) & ~15ull); }

template <typename T> __device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <> __device__ __forceinline__ ulonglong2 warp_sum_t<ulonglong2>(ulonglong2 v)
{
    return make_ulonglong2(warp_sum_t(v.x), warp_sum_t(v.y));
}

__device__ __forceinline__ unsigned long long scan_now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kScanWaitNs = 1000000000ull;

template <typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(Op op, uint64_t n, typename Op::T *partial, uint32_t nb,
                                                               Control *ctl)
{
    using T = typename Op::T;
    __shared__ unsigned long long sh[66];
    __shared__ uint32_t s_tile;
    __shared__ T s_pre;
    uint8_t *b8 = reinterpret_cast<uint8_t *>(partial);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(b8);
    volatile uint32_t *flag = reinterpret_cast<volatile uint32_t *>(b8 + 16);
    T *agg = reinterpret_cast<T *>(b8 + scan_flag_bytes(nb));
    T *inc = agg + nb;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t base = tile * kScanBlock + (uint64_t)threadIdx.x * kScanPer;
    T v[kScanPer];
    T s = scan_zero<T>();
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        v[j] = base + j < n ? op.load(base + j) : scan_zero<T>();
        s += v[j];
    }
    T tot;
    const T local = block_excl_scan_t(s, sh, &tot);
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        T pre = scan_zero<T>();
        if (tile == 0) {
            if (lane == 0) {
                inc[0] = tot;
                __threadfence();
                flag[0] = 2;
            }
        } else {
            if (lane == 0) {
                agg[tile] = tot;
                __threadfence();
                flag[tile] = 1;
            }
            int64_t b = (int64_t)tile - 1;
            const unsigned long long t0 = scan_now_ns();
            bool late = false;
            for (;;) {
                const int64_t idx = b - (int64_t)lane;
                const uint32_t fl = idx >= 0 ? flag[idx] : 2u;
                const unsigned incm = __ballot_sync(0xffffffffu, fl == 2);
                const unsigned notyet = __ballot_sync(0xffffffffu, fl == 0);
                const uint32_t fi = incm ? __ffs(incm) - 1 : 31u;
                const unsigned need = fi == 31 ? 0xffffffffu : ((2u << fi) - 1u);
                if (notyet & need) {
                    // the same decision in every lane: the votes need the whole warp
                    if (__any_sync(0xffffffffu, scan_now_ns() - t0 > kScanWaitNs)) {
                        late = true;
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                __threadfence();
                T val = scan_zero<T>();
                if (lane <= fi && idx >= 0) val = fl == 2 ? __ldcg(inc + idx) : __ldcg(agg + idx);
                pre += warp_sum_t(val);
                if (incm) break;
                b -= 32;
            }
            if (lane == 0) {
                inc[tile] = pre + tot;
                __threadfence();
                flag[tile] = 2;
                if (late) atomicOr(&ctl->error, DERR_TIMEOUT);
            }
        }
        if (lane == 0) s_pre = pre;
    }
    __syncthreads();
    const T pre = s_pre;
    T run = local + pre;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        if (base + j < n) op.store(base + j, run);
        run += v[j];
    }
    if (tile == nb - 1 && threadIdx.x == 0) op.total(pre + tot);
}

// partial: scratch of at least scan_partials(n) entries of Op::T; ctl gets
// the timeout bit if a look-back wait gives up.  Returns kernels launched.
template <typename Op>
inline int launch_scan(const Op &op, uint64_t n, typename Op::T *partial, Control *ctl, cudaStream_t st)
{
    if (n == 0) return 0;
    const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    cudaMemsetAsync(partial, 0, scan_flag_bytes(nb), st);
    k_scan_onepass<Op><<<(unsigned)nb, kScanThreads, 0, st>>>(op, n, partial, (uint32_t)nb, ctl);
    return 1;
}

// Grouped: the scans of many fields in three launches.  Item provides
// using Op; Op op() const; uint64_t n; typename Op::T *partial.  Item i owns
// ceil(n / kScanBlock) blocks of the reduce and apply grids (first[]) and
// block i of the top grid.
template <typename Item>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce_group(const Item *items, const uint32_t *first,
                                                                   uint32_t ni)
{
    VGrid vg;
    const Item &it = items[group_item(first, ni, vg)];
    scan_reduce_body(it.op(), it.n, it.partial, vg.bid);
}

template <typename Item>
__global__ void __launch_bounds__(kScanThreads) k_scan_top_group(const Item *items)
{
    const Item &it = items[blockIdx.x];
    scan_top_body(it.op(), (it.n + kScanBlock - 1) / kScanBlock, it.partial);
}

template <typename Item>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply_group(const Item *items, const uint32_t *first,
                                                                  uint32_t ni)
{
    VGrid vg;
    const Item &it = items[group_item(first, ni, vg)];
    scan_apply_body(it.op(), it.n, it.partial, vg.bid);
}

// blocks = first[ni] (every item with n >= 1); returns kernels launched
template <typename Item>
inline int launch_scan_group(const Item *items, const uint32_t *first, uint32_t ni, uint32_t blocks, cudaStream_t st)
{
    if (ni == 0 || blocks == 0) return 0;
    k_scan_reduce_group<Item><<<blocks, kScanThreads, 0, st>>>(items, first, ni);
    k_scan_top_group<Item><<<ni, kScanThreads, 0, st>>>(items);
    k_scan_apply_group<Item><<<blocks, kScanThreads, 0, st>>>(items, first, ni);
    return 3;
}

inline uint64_t scan_blocks(uint64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

// entries of T (4 bytes or more) the scratch of a scan of n entries needs:
// the single pass's ticket, flags, totals and inclusive totals, or the three
// kernels' block totals
inline uint64_t scan_partials(uint64_t n) { return 3 * ((n + kScanBlock - 1) / kScanBlock) + 8; }

}  // namespace gbsz
