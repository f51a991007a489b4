// prims.cuh -- device-wide building blocks written for this library:
// block/warp scans, an exclusive scan over functor-generated int64 values,
// a stable LSD radix sort of (uint64 key, int32 value) pairs, and reductions.
#pragma once

#include "common.cuh"

namespace sclap {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---------------------------------------------------------------- block scan

// Exclusive scan of one value per thread over the block; returns the thread's
// exclusive prefix and writes the block total to *total (all threads).
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total, T *smem /* >= NT/32 + 1 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) smem[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = (lane < NT / 32) ? smem[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < NT / 32) smem[lane] = wi - w;  // exclusive warp offsets
        if (lane == NT / 32 - 1) smem[NT / 32] = wi;
    }
    __syncthreads();
    T res = smem[warp] + inc - x;
    *total = smem[NT / 32];
    __syncthreads();
    return res;
}

// Appends the non-negative values x of the calling warp's lanes to list
// (count in *cnt), lane order within the warp: one atomic per warp.  Every
// lane of the warp must call it.
template <typename T>
__device__ __forceinline__ void warp_append(T *list, int *cnt, int x) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, x >= 0);
    if (!m) return;
    const int first = __ffs(m) - 1;
    int base = 0;
    if (lane == first) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, first);
    if (x >= 0) list[base + __popc(m & ((1u << lane) - 1))] = (T)x;
}

// ---------------------------------------------------------------- device-wide exclusive scan

template <typename F>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(F f, int64_t n, int64_t *sums) {
    __shared__ int64_t sm[kScanThreads / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + (int64_t)j * kScanThreads + threadIdx.x;
        if (i < n) acc += (int64_t)f(i);
    }
    int64_t tot;
    block_exclusive_scan<kScanThreads>(acc, &tot, sm);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Blocked layout: thread t owns items [t*kScanItems, (t+1)*kScanItems) of the tile.
template <typename F>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_apply(F f, int64_t n, const int64_t *offs, int64_t *out, int64_t *total) {
    __shared__ int64_t sm[kScanThreads / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + j;
        v[j] = i < n ? (int64_t)f(i) : 0;
        acc += v[j];
    }
    int64_t tot;
    int64_t pre = block_exclusive_scan<kScanThreads>(acc, &tot, sm) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        int64_t i = base + j;
        if (i < n) out[i] = pre;
        pre += v[j];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) *total = pre;
}

struct ArrayI64 {
    const int64_t *p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};

// out[i] = sum_{j<i} f(j) for i in [0, n); *d_total (device, optional) = sum of all.
template <typename F>
void exclusive_scan(F f, int64_t n, int64_t *out, int64_t *d_total, Scratch &sc) {
    cudaStream_t s = sc.stream();
    if (n <= 0) {
        if (d_total) CK(cudaMemsetAsync(d_total, 0, sizeof(int64_t), s));
        return;
    }
    int64_t tiles = ceil_div<int64_t>(n, kScanTile);
    if (tiles == 1) {
        k_scan_apply<<<1, kScanThreads, 0, s>>>(f, n, nullptr, out, d_total);
        LAUNCHED();
        return;
    }
    int64_t *sums = sc.get<int64_t>(tiles);
    int64_t *offs = sc.get<int64_t>(tiles);
    k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, s>>>(f, n, sums);
    LAUNCHED();
    exclusive_scan(ArrayI64{sums}, tiles, offs, nullptr, sc);
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(f, n, offs, out, d_total);
    LAUNCHED();
}

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;                       // items per lane
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 keys per tile
constexpr int kRadixBits = 9;                          // digit width of one pass
constexpr int kRadix = 1 << kRadixBits;
constexpr int kDigitsPerThread = kRadix / kSortThreads;

// Sorts (keys, vals) stably by key bits [0, nbits).  keys/vals are sorted in
// place (alt buffers are scratch).
void radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int nbits, Scratch &sc);

// Number of significant bits of x (0 for x == 0).
inline int bit_width_u64(uint64_t x) {
    int b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

// ---------------------------------------------------------------- entry -> row

// Largest v in [0, n) with a[v] <= key, for non-decreasing a[0..n) with
// a[0] <= key (0 when n == 0).  Called by all lanes of one warp: every step
// probes 32 evenly spaced points of (lo, hi], and because a is monotone the
// lanes whose probe is <= key form a prefix, so the ballot's population count
// picks the new interval; it shrinks 32-fold per step (five dependent loads
// for 2^22 rows instead of 22).
__device__ __forceinline__ int64_t warp_last_le(const int64_t *a, int64_t n, int64_t key) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;  // a[lo] <= key; hi == n or a[hi] > key
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) >> 5;
        const int64_t p = lo + (int64_t)(lane + 1) * step;
        const unsigned b = __ballot_sync(0xffffffffu, p < hi && a[p] <= key);
        const int c = __popc(b);
        const int64_t first_false = lo + (int64_t)(c + 1) * step;
        lo += (int64_t)c * step;
        if (first_false < hi) hi = first_false;
    }
    return lo;
}

// For the entry range [e0, e0 + len) (len <= NT * PER) of a CSR with row
// offsets xadj[0..n], writes rowof[i] = the row containing entry e0 + i.
// Rows are found once per range (warps 0 and 1 search the first and the last
// row at the same time); each row start inside the range marks its position
// (the largest row id wins, skipping empty rows), and an inclusive max-scan
// spreads the row ids.  All threads call it.
template <int NT, int PER>
__device__ void block_rows(const int64_t *xadj, int64_t n, int64_t e0, int len, int32_t *rowof,
                           int32_t *scan_tmp /* >= NT/32 + 2 */) {
    static_assert(NT >= 64 && NT % 32 == 0, "two whole warps search the rows");
    __shared__ int64_t s_rows[2];
    if (threadIdx.x < 64) {
        // first row: largest v with xadj[v] <= e0; last: largest v with xadj[v] <= e0+len-1
        const int which = threadIdx.x >> 5;
        const int64_t r = warp_last_le(xadj, n, which == 0 ? e0 : e0 + len - 1);
        if ((threadIdx.x & 31) == 0) s_rows[which] = r;
    }
    for (int i = threadIdx.x; i < len; i += NT) rowof[i] = -1;
    __syncthreads();
    const int64_t v0 = s_rows[0], v1 = s_rows[1];
    if (threadIdx.x == 0) atomicMax(&rowof[0], (int32_t)v0);
    for (int64_t v = v0 + 1 + threadIdx.x; v <= v1; v += NT) {
        const int64_t p = xadj[v] - e0;
        if (p >= 0 && p < len) atomicMax(&rowof[p], (int32_t)v);
    }
    __syncthreads();
    // inclusive max-scan over rowof (thread t owns [t*PER, (t+1)*PER))
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t run = -1;
    const int base = threadIdx.x * PER;
#pragma unroll
    for (int j = 0; j < PER; j++)
        if (base + j < len) run = max(run, rowof[base + j]);
    int32_t inc = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc = max(inc, y);
    }
    if (lane == 31) scan_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < NT / 32 ? scan_tmp[lane] : -1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w = max(w, y);
        }
        if (lane < NT / 32) scan_tmp[lane] = w;
    }
    __syncthreads();
    int32_t pre = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) pre = -1;
    if (warp > 0) pre = max(pre, scan_tmp[warp - 1]);
    int32_t cur = pre;
#pragma unroll
    for (int j = 0; j < PER; j++)
        if (base + j < len) {
            cur = max(cur, rowof[base + j]);
            rowof[base + j] = cur;
        }
    __syncthreads();
}

// ---------------------------------------------------------------- reductions

// Device-side sums / maxima used for validation and bounds (results to host).
struct GraphTotals {
    int64_t cV;          // sum of c
    int64_t maxc;        // max c
    int64_t sum_w;       // sum of omega over all directed entries
    int64_t max_wdeg;    // max weighted degree (an upper bound unless computed exactly)
    int64_t max_deg;     // max degree
};
// need_wdeg: make max_wdeg exact when the total edge weight is above INT32_MAX
// (otherwise the total is reported as the bound).
GraphTotals graph_totals(const DGraph &g, Scratch &sc, bool need_wdeg = false);

}  // namespace sclap
