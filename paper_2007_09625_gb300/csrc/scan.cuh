// scan.cuh -- device-wide exclusive prefix sum in three coalesced kernels
// (block reduce -> scan of block totals -> block scan plus carry), used for
// chunk word offsets and 1D tile carries.  No inter-CTA waiting.
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

template <typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(Op op, uint64_t n, typename Op::T *partial)
{
    scan_reduce_body(op, n, partial, blockIdx.x);
}

template <typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_top(Op op, uint64_t nb, typename Op::T *partial)
{
    scan_top_body(op, nb, partial);
}

template <typename Op>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(Op op, uint64_t n, const typename Op::T *partial)
{
    scan_apply_body(op, n, partial, blockIdx.x);
}

// partial: scratch of at least ceil(n / kScanBlock) entries
template <typename Op>
inline int launch_scan(const Op &op, uint64_t n, typename Op::T *partial, cudaStream_t st)
{
    if (n == 0) return 0;
    const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_reduce<Op><<<(unsigned)nb, kScanThreads, 0, st>>>(op, n, partial);
    k_scan_top<Op><<<1, kScanThreads, 0, st>>>(op, nb, partial);
    k_scan_apply<Op><<<(unsigned)nb, kScanThreads, 0, st>>>(op, n, partial);
    return 3;
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

inline uint64_t scan_partials(uint64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

}  // namespace gbsz
