// prims.cu -- scratch pool, launch accounting, radix sort, graph reductions.
#include <atomic>
#include <mutex>

#include "prims.cuh"

namespace sclap {

// ---------------------------------------------------------------- accounting

static std::atomic<int64_t> g_launches{0}, g_graph_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_graph_launch() { g_graph_launches.fetch_add(1, std::memory_order_relaxed); }

static ProfState g_prof;
ProfState &prof() {
    g_prof.kernel_launches = g_launches.load();
    g_prof.graph_launches = g_graph_launches.load();
    return g_prof;
}

void prof_begin(cudaStream_t s, cudaEvent_t *b, cudaEvent_t *e) {
    *b = *e = nullptr;
    if (!g_prof.on) return;
    CK(cudaEventCreate(b));
    CK(cudaEventCreate(e));
    CK(cudaEventRecord(*b, s));
}

void prof_end(cudaStream_t s, cudaEvent_t b, cudaEvent_t e) {
    if (!b) return;
    CK(cudaEventRecord(e, s));
    g_prof.pending.emplace_back(b, e);
    g_prof.propose_launches++;
}

// ---------------------------------------------------------------- device info / pool

static std::mutex g_mu;
static DevInfo g_dev[64];
static bool g_dev_ok[64];
static cudaMemPool_t g_pool[64];

const DevInfo &dev_info() {
    int d = 0;
    CK(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ok[d]) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d));
        g_dev[d] = DevInfo{d, sms};
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = d;
        CK(cudaMemPoolCreate(&g_pool[d], &props));
        uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
        CK(cudaMemPoolSetAttribute(g_pool[d], cudaMemPoolAttrReleaseThreshold, &thr));
        g_dev_ok[d] = true;
    }
    return g_dev[d];
}

// Allocation-failure injection (tests): the scratch allocation that finds
// the counter at 0 fails as if the device were out of memory; -1 disables.
static std::atomic<long long> g_fail_after{-1};
void set_alloc_failure(long long after) { g_fail_after.store(after); }

void *scratch_alloc(size_t bytes, cudaStream_t s) {
    const DevInfo &di = dev_info();
    void *p = nullptr;
    long long f = g_fail_after.load();
    while (f >= 0 && !g_fail_after.compare_exchange_weak(f, f - 1)) {
    }
    if (f == 0) fail(SCLAP_ENOMEM, "scratch allocation (injected)");
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, g_pool[di.device], s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        fail(SCLAP_ENOMEM, "scratch allocation");
    }
    CK(e);
    return p;
}

void scratch_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------- radix sort

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) {
    return (uint32_t)(k >> shift) & (kRadix - 1);
}

// Per-tile digit histogram, written digit-major: hist[d * tiles + tile].
__global__ void __launch_bounds__(kSortThreads)
    k_sort_hist(const uint64_t *keys, int64_t n, int shift, int64_t tiles, int64_t *hist) {
    __shared__ int cnt[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += kSortThreads) cnt[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int j = 0; j < kSortRounds; j++) {
        int64_t i = base + (int64_t)j * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[digit_of(keys[i], shift)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
        hist[(int64_t)d * tiles + blockIdx.x] = cnt[d];
}

// Stable scatter.  Warp w owns tile items [w*32*R, (w+1)*32*R) and walks them
// in order (round-major, lane-minor), so ranks respect the input order.  The
// tile is first rearranged in shared memory in digit order; the global writes
// then go out as one contiguous run per digit.
struct SortSm {
    int wc[kSortWarps][kRadix];
    int64_t goff[kRadix];
    int dstart[kRadix];
    int scan_tmp[kSortWarps + 1];
    uint64_t k[kSortTile];
    int32_t v[kSortTile];
};

__global__ void __launch_bounds__(kSortThreads)
    k_sort_scatter(const uint64_t *keys, const int32_t *vals, uint64_t *okeys, int32_t *ovals,
                   int64_t n, int shift, int64_t tiles, const int64_t *offs) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SortSm &sm = *reinterpret_cast<SortSm *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&sm.wc[0][0])[i] = 0;
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
        sm.goff[d] = offs[(int64_t)d * tiles + blockIdx.x];
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * kSortTile;
    const int64_t wbase = tbase + (int64_t)warp * 32 * kSortRounds;
    const unsigned lt = (1u << lane) - 1;
    uint64_t k[kSortRounds];
    int32_t v[kSortRounds];
    int rk[kSortRounds];
#pragma unroll
    for (int r = 0; r < kSortRounds; r++) {
        int64_t i = wbase + r * 32 + lane;
        bool ok = i < n;
        k[r] = ok ? keys[i] : 0;
        v[r] = ok ? vals[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; r++) {
        const bool ok = wbase + r * 32 + lane < n;
        uint32_t d = ok ? digit_of(k[r], shift) : kRadix;  // kRadix: padding
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int base = (d < kRadix) ? sm.wc[warp][d] : 0;
        __syncwarp();
        if (d < kRadix && (peers & lt) == 0) sm.wc[warp][d] = base + __popc(peers);
        __syncwarp();
        rk[r] = base + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: warp offsets, then the digit's start inside the tile
    // (thread t owns the consecutive digits t * kDigitsPerThread + j)
    int tot[kDigitsPerThread];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; j++) {
        const int d = threadIdx.x * kDigitsPerThread + j;
        int run = 0;
        for (int w = 0; w < kSortWarps; w++) {
            const int t = sm.wc[w][d];
            sm.wc[w][d] = run;
            run += t;
        }
        tot[j] = run;
        sum += run;
    }
    int all;
    int ds = block_exclusive_scan<kSortThreads>(sum, &all, sm.scan_tmp);
#pragma unroll
    for (int j = 0; j < kDigitsPerThread; j++) {
        sm.dstart[threadIdx.x * kDigitsPerThread + j] = ds;
        ds += tot[j];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; r++) {
        if (wbase + r * 32 + lane < n) {
            const uint32_t d = digit_of(k[r], shift);
            const int loc = sm.dstart[d] + sm.wc[warp][d] + rk[r];
            sm.k[loc] = k[r];
            sm.v[loc] = v[r];
        }
    }
    __syncthreads();
    const int len = (int)min64(n - tbase, (int64_t)kSortTile);
    for (int i = threadIdx.x; i < len; i += kSortThreads) {
        const uint64_t key = sm.k[i];
        const uint32_t d = digit_of(key, shift);
        const int64_t dst = sm.goff[d] + (i - sm.dstart[d]);
        okeys[dst] = key;
        ovals[dst] = sm.v[i];
    }
}

void radix_sort_pairs(uint64_t *keys, int32_t *vals, int64_t n, int nbits, Scratch &sc) {
    if (n <= 1 || nbits <= 0) return;
    cudaStream_t s = sc.stream();
    int64_t tiles = ceil_div<int64_t>(n, kSortTile);
    uint64_t *k2 = sc.get<uint64_t>(n);
    int32_t *v2 = sc.get<int32_t>(n);
    int64_t *hist = sc.get<int64_t>(tiles * kRadix);
    int64_t *offs = sc.get<int64_t>(tiles * kRadix);
    static_assert(kRadix % kSortThreads == 0, "whole digits per thread in the scatter");
    CK(cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sizeof(SortSm)));
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < nbits; shift += kRadixBits, passes++) {
        k_sort_hist<<<(unsigned)tiles, kSortThreads, 0, s>>>(ka, n, shift, tiles, hist);
        LAUNCHED();
        exclusive_scan(ArrayI64{hist}, tiles * kRadix, offs, nullptr, sc);
        k_sort_scatter<<<(unsigned)tiles, kSortThreads, sizeof(SortSm), s>>>(ka, va, kb, vb, n,
                                                                             shift, tiles, offs);
        LAUNCHED();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CK(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
}

// ---------------------------------------------------------------- graph totals

__global__ void k_totals(DGraph g, unsigned long long *acc /* [5] */) {
    int64_t cV = 0, maxc = 0, sw = 0, maxd = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = g.vwgt[v];
        cV += c;
        maxc = max64(maxc, c);
        maxd = max64(maxd, g.xadj[v + 1] - g.xadj[v]);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nnz;
         i += (int64_t)gridDim.x * blockDim.x)
        sw += g.adjwgt[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        cV += __shfl_down_sync(0xffffffffu, cV, d);
        sw += __shfl_down_sync(0xffffffffu, sw, d);
        maxc = max64(maxc, __shfl_down_sync(0xffffffffu, maxc, d));
        maxd = max64(maxd, __shfl_down_sync(0xffffffffu, maxd, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], (unsigned long long)cV);
        atomicMax(&acc[1], (unsigned long long)maxc);
        atomicAdd(&acc[2], (unsigned long long)sw);
        atomicMax(&acc[4], (unsigned long long)maxd);
    }
}

// Exact weighted degrees (only needed when the total edge weight exceeds the
// 32-bit range): per-entry sums into wdeg[row], aggregated per warp and row.
constexpr int kWdegTile = 4096;

__global__ void __launch_bounds__(256) k_wdeg(DGraph g, unsigned long long *wdeg) {
    __shared__ int32_t rowof[kWdegTile];
    __shared__ int32_t tmp[16];
    const int64_t tiles = ceil_div<int64_t>(g.nnz, kWdegTile);
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kWdegTile;
        const int len = (int)min64(kWdegTile, g.nnz - e0);
        block_rows<256, 16>(g.xadj, g.n, e0, len, rowof, tmp);
        const int lanes = (len + 31) & ~31;
        for (int i = threadIdx.x; i < lanes; i += 256) {
            const bool in = i < len;
            const int32_t v = in ? rowof[i] : -1 - (int32_t)(threadIdx.x & 31);
            const unsigned peers = __match_any_sync(0xffffffffu, v);
            int64_t w = in ? g.adjwgt[e0 + i] : 0;
            int64_t s = 0;
            for (unsigned m = peers; m; m &= m - 1) s += __shfl_sync(peers, w, __ffs(m) - 1);
            if (in && (peers & ((1u << (threadIdx.x & 31)) - 1)) == 0)
                atomicAdd(&wdeg[v], (unsigned long long)s);
        }
        __syncthreads();
    }
}

__global__ void k_max_u64(const unsigned long long *x, int64_t n, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = x[i] > m ? x[i] : m;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

GraphTotals graph_totals(const DGraph &g, Scratch &sc, bool need_wdeg) {
    cudaStream_t s = sc.stream();
    unsigned long long *acc = sc.zeros<unsigned long long>(5);
    const int sms = dev_info().sms;
    if (g.n > 0) {
        k_totals<<<sms * 4, 256, 0, s>>>(g, acc);
        LAUNCHED();
    }
    unsigned long long h[5];
    CK(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    GraphTotals t{(int64_t)h[0], (int64_t)h[1], (int64_t)h[2], (int64_t)h[2], (int64_t)h[4]};
    // every weighted degree is at most the total; compute it exactly only when
    // the total alone does not settle the 32-bit check
    if (need_wdeg && t.sum_w > INT32_MAX && g.nnz > 0) {
        unsigned long long *wdeg = sc.zeros<unsigned long long>(g.n);
        const int grid = (int)std::min<int64_t>(ceil_div<int64_t>(g.nnz, kWdegTile), sms * 8);
        k_wdeg<<<grid, 256, 0, s>>>(g, wdeg);
        LAUNCHED();
        k_max_u64<<<sms * 4, 256, 0, s>>>(wdeg, g.n, acc + 3);
        LAUNCHED();
        unsigned long long m = 0;
        CK(cudaMemcpyAsync(&m, acc + 3, sizeof(m), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        t.max_wdeg = (int64_t)m;
    }
    return t;
}

}  // namespace sclap
