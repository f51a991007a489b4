// contract.cu -- cluster contraction (Sec. III "contracting a clustering",
// Sec. IV.C): the prefix-sum map q over used cluster ids, C(v) = q(label(v)),
// coarse node weights, and the quotient edges.  Quotient edges are reduced
// in two stages: a shared-memory hash table merges equal (C(u), C(v)) pairs
// inside fixed 2048-entry slices of the fine rows (rows grouped by coarse
// node), then a radix sort by (C(u), C(v)) and a tiled reduce of equal keys
// produce the canonical sorted CSR.  Also projection (uncoarsening) and cut/balance.
#include "contract.cuh"
#include "prims.cuh"

namespace sclap {

constexpr int kCThreads = 256;
constexpr int kCEntries = 2048;
constexpr int kCSlots = 4096;
constexpr int kCBits = 12;
constexpr int kAggItems = kCEntries / kCThreads;  // entries per thread and slice
static_assert(kCEntries % kCThreads == 0, "whole entries per thread");

__global__ void k_mark(int64_t n, const int32_t *lab, int32_t *mark) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        mark[lab[v]] = 1;
}

struct ArrayI32 {
    const int32_t *p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};

// f2c, coarse node weights, member counts and coarse "work" (sum of degrees).
__global__ void k_f2c(DGraph g, const int32_t *lab, const int64_t *q, int32_t *f2c, int32_t *cvwgt,
                      int32_t *ccnt) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = (int32_t)q[lab[v]];
        f2c[v] = c;
        atomicAdd(&cvwgt[c], g.vwgt[v]);
        if (g.xadj[v + 1] > g.xadj[v]) atomicAdd(&ccnt[c], 1);
    }
}

// members of coarse node c (nodes with >= 1 entry) at [mstart[c], mstart[c+1]).
__global__ void k_members(DGraph g, const int32_t *f2c, const int64_t *mstart, int32_t *fill,
                          int32_t *members) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (g.xadj[v + 1] == g.xadj[v]) continue;
        int32_t c = f2c[v];
        members[mstart[c] + atomicAdd(&fill[c], 1)] = (int32_t)v;
    }
}

struct MemberDeg {
    const int64_t *xadj;
    const int32_t *members;
    __device__ int64_t operator()(int64_t i) const {
        int32_t v = members[i];
        return xadj[v + 1] - xadj[v];
    }
};

// Slice state.  K32: keys are ((C(u) - C(first member)) << cbits) | C(v) in
// 32 bits (a slice holds at most kCEntries + 1 members, so the first part
// needs 12 bits; used when cbits <= 20), else (C(u) << cbits) | C(v).
template <bool K32>
struct AggSm {
    typename std::conditional<K32, uint32_t, unsigned long long>::type keys[kCSlots];
    int32_t vals[kCSlots];
    uint16_t dl[kCEntries];
    int32_t rowof[kCEntries];  // member index of each slice entry
    int32_t scan_tmp[kCThreads / 32 + 2];
    unsigned long long out_base;
    int ndl;
    int32_t cu0;
};

// Slice t covers concatenated member entries [t*kCEntries, (t+1)*kCEntries).
template <bool K32>
__global__ void __launch_bounds__(kCThreads, 5)
    k_aggregate(DGraph g, const int32_t *members, int64_t nmem, const int64_t *mpre,
                int64_t total, const int32_t *f2c, int cbits, unsigned long long *out_keys,
                int32_t *out_w, unsigned long long *out_cnt) {
    using Key = typename std::conditional<K32, uint32_t, unsigned long long>::type;
    constexpr Key kEmptyK = (Key)~(Key)0;
    extern __shared__ __align__(16) unsigned char smraw[];
    AggSm<K32> &sm = *reinterpret_cast<AggSm<K32> *>(smraw);
    for (int i = threadIdx.x; i < kCSlots; i += kCThreads) {
        sm.keys[i] = kEmptyK;
        sm.vals[i] = 0;
    }
    const uint64_t cmask = (1ull << cbits) - 1;
    const int64_t slices = ceil_div<int64_t>(total, kCEntries);
    for (int64_t t = blockIdx.x; t < slices; t += gridDim.x) {
        const int64_t e0 = t * kCEntries;
        const int len = (int)min64(total - e0, (int64_t)kCEntries);
        if (threadIdx.x == 0) {
            sm.ndl = 0;
            sm.out_base = 0;
        }
        block_rows<kCThreads, kCEntries / kCThreads>(mpre, nmem, e0, len, sm.rowof, sm.scan_tmp);
        if (threadIdx.x == 0) sm.cu0 = f2c[members[sm.rowof[0]]];
        __syncthreads();
        const int32_t cu0 = sm.cu0;
        // all gathers of the thread's entries first (kAggItems independent
        // load chains in flight), then the inserts
        int32_t ecu[kAggItems], ecv[kAggItems], ew[kAggItems];
#pragma unroll
        for (int j = 0; j < kAggItems; j++) {
            const int le = j * kCThreads + threadIdx.x;
            ecu[j] = 0;
            ecv[j] = 0;
            ew[j] = 0;
            if (le < len) {
                const int32_t mi = sm.rowof[le];
                const int32_t v = __ldg(&members[mi]);
                const int64_t idx = __ldg(&g.xadj[v]) + (e0 + le - __ldg(&mpre[mi]));
                ecu[j] = __ldg(&f2c[v]);
                ecv[j] = __ldg(&f2c[__ldg(&g.adjncy[idx])]);
                ew[j] = __ldg(&g.adjwgt[idx]);
            }
        }
        // the same number of steps in every thread (warp-wide appends of new slots)
#pragma unroll
        for (int j = 0; j < kAggItems; j++) {
            const int le = j * kCThreads + threadIdx.x;
            int created = -1;
            if (le < len) {
                const int32_t cu = ecu[j];
                const int32_t cv = ecv[j];
                if (cu != cv) {  // else an edge inside a cluster
                    const int32_t w = ew[j];
                    Key key;
                    uint32_t slot;
                    if constexpr (K32) {
                        key = ((uint32_t)(cu - cu0) << cbits) | (uint32_t)cv;
                        slot = (key * 0x9E3779B1u) >> (32 - kCBits);
                    } else {
                        key = ((uint64_t)(uint32_t)cu << cbits) | (uint32_t)cv;
                        slot = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - kCBits));
                    }
                    for (int probe = 0; probe < kCSlots; probe++) {  // never full: load <= 1/2
                        const Key prev = atomicCAS(&sm.keys[slot], kEmptyK, key);
                        if (prev == kEmptyK || prev == key) {
                            atomicAdd(&sm.vals[slot], w);
                            if (prev == kEmptyK) created = (int)slot;
                            break;
                        }
                        slot = (slot + 1) & (kCSlots - 1);
                    }
                }
            }
            warp_append(sm.dl, &sm.ndl, created);
        }
        __syncthreads();
        const int ndl = sm.ndl;
        if (threadIdx.x == 0 && ndl) sm.out_base = atomicAdd(out_cnt, (unsigned long long)ndl);
        __syncthreads();
        const int64_t ob = (int64_t)sm.out_base;
        for (int i = threadIdx.x; i < ndl; i += kCThreads) {
            const int slot = sm.dl[i];
            const Key key = sm.keys[slot];
            if constexpr (K32)
                out_keys[ob + i] = ((uint64_t)(uint32_t)(cu0 + (int32_t)(key >> cbits)) << cbits) |
                                   (key & cmask);
            else
                out_keys[ob + i] = key;
            out_w[ob + i] = sm.vals[slot];
            sm.keys[slot] = kEmptyK;
            sm.vals[slot] = 0;
        }
        __syncthreads();
    }
}

// Sorted (key, w) pairs -> unique keys, in tiles of kRTile pairs.  Pass 1
// counts the run starts (first pair of each distinct key) per tile; an
// exclusive scan of the counts gives each tile its first output position.
// Pass 2 stages the tile in shared memory, gives each thread kRItems
// consecutive pairs, ranks its run starts by a block scan, sums each run
// (reading past the tile when a run continues into the next one) and writes
// the coarse entry; row degrees get one atomic per row and thread.
constexpr int kRThreads = 256;
constexpr int kRItems = 16;
constexpr int kRTile = kRThreads * kRItems;

__global__ void __launch_bounds__(kRThreads) k_run_count(const unsigned long long *keys, int64_t P,
                                                         int64_t *tile_cnt) {
    __shared__ int64_t sm[kRThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kRTile;
    int64_t cnt = 0;
#pragma unroll 4
    for (int j = 0; j < kRItems; j++) {
        const int64_t i = base + (int64_t)j * kRThreads + threadIdx.x;
        if (i < P) cnt += (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
    }
    int64_t tot;
    block_exclusive_scan<kRThreads>(cnt, &tot, sm);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// Shared tile, one pad slot after every kRItems pairs so that the threads'
// blocked reads (kRItems apart) fall into different banks.
constexpr int kRPad = kRTile + kRTile / kRItems;
__device__ __forceinline__ int rpad(int l) { return l + l / kRItems; }

struct RunSm {
    unsigned long long k[kRPad];
    int32_t w[kRPad];
    int64_t scan[kRThreads / 32 + 1];
};

__global__ void __launch_bounds__(kRThreads) k_run_emit(const unsigned long long *keys,
                                                        const int32_t *w, int64_t P,
                                                        const int64_t *tile_off, int cbits,
                                                        int32_t *adjncy, int32_t *adjwgt,
                                                        int32_t *cdeg) {
    extern __shared__ __align__(16) unsigned char smraw[];
    RunSm &sm = *reinterpret_cast<RunSm *>(smraw);
    const uint64_t mask = (cbits >= 64) ? ~0ull : ((1ull << cbits) - 1);
    const int64_t base = (int64_t)blockIdx.x * kRTile;
    const int len = (int)min64(P - base, (int64_t)kRTile);
    for (int i = threadIdx.x; i < len; i += kRThreads) {
        sm.k[rpad(i)] = keys[base + i];
        sm.w[rpad(i)] = w[base + i];
    }
    __syncthreads();
    const int l0 = threadIdx.x * kRItems;
    const unsigned long long before = base > 0 ? keys[base - 1] : 0;
    int64_t cnt = 0;
#pragma unroll
    for (int j = 0; j < kRItems; j++) {
        const int l = l0 + j;
        if (l < len)
            cnt += (l == 0 ? (base == 0 || sm.k[0] != before) : sm.k[rpad(l)] != sm.k[rpad(l - 1)])
                       ? 1 : 0;
    }
    int64_t tot;
    int64_t p = tile_off[blockIdx.x] + block_exclusive_scan<kRThreads>(cnt, &tot, sm.scan);
    int64_t row = -1;
    int32_t rcnt = 0;
    for (int j = 0; j < kRItems; j++) {
        const int l = l0 + j;
        if (l >= len) break;
        const unsigned long long k = sm.k[rpad(l)];
        if (!(l == 0 ? (base == 0 || k != before) : k != sm.k[rpad(l - 1)])) continue;
        int64_t sum = sm.w[rpad(l)];
        int m = l + 1;
        for (; m < len && sm.k[rpad(m)] == k; m++) sum += sm.w[rpad(m)];
        if (m == len)
            for (int64_t i = base + len; i < P && keys[i] == k; i++) sum += w[i];
        adjncy[p] = (int32_t)(k & mask);
        adjwgt[p] = (int32_t)sum;
        p++;
        const int64_t r = (int64_t)(k >> cbits);
        if (r != row) {
            if (rcnt) atomicAdd(&cdeg[row], rcnt);
            row = r;
            rcnt = 0;
        }
        rcnt++;
    }
    if (rcnt) atomicAdd(&cdeg[row], rcnt);
}

struct ArrayI32to64 {
    const int32_t *p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};

__global__ void k_finish_xadj(const int64_t *pre, int64_t n, int64_t total, int64_t *xadj) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        xadj[i] = i < n ? pre[i] : total;
}

void contract_impl(const DGraph &g, const int32_t *lab, int32_t *f2c, CoarseGraph *out,
                   Scratch *out_sc, Scratch &sc) {
    cudaStream_t s = sc.stream();
    const int sms = dev_info().sms;
    const int grid = sms * 4;
    auto out_alloc = [&](size_t bytes) -> void * {
        if (bytes == 0) bytes = 16;
        if (out_sc) return out_sc->get<unsigned char>(bytes);
        void *p = nullptr;
        CK(cudaMalloc(&p, bytes));
        return p;
    };
    *out = CoarseGraph{};
    if (g.n == 0) {
        out->xadj = (int64_t *)out_alloc(sizeof(int64_t));
        CK(cudaMemsetAsync(out->xadj, 0, sizeof(int64_t), s));
        out->adjncy = (int32_t *)out_alloc(4);
        out->adjwgt = (int32_t *)out_alloc(4);
        out->vwgt = (int32_t *)out_alloc(4);
        return;
    }
    // q: rank of each used label
    int32_t *mark = sc.zeros<int32_t>(g.n);
    k_mark<<<grid, 256, 0, s>>>(g.n, lab, mark);
    LAUNCHED();
    int64_t *q = sc.get<int64_t>(g.n);
    int64_t *d_n2 = sc.get<int64_t>(1);
    exclusive_scan(ArrayI32{mark}, g.n, q, d_n2, sc);
    int64_t n2 = 0;
    CK(cudaMemcpyAsync(&n2, d_n2, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    int32_t *cvwgt = (int32_t *)out_alloc(n2 * sizeof(int32_t));
    CK(cudaMemsetAsync(cvwgt, 0, n2 * sizeof(int32_t), s));
    int32_t *ccnt = sc.zeros<int32_t>(n2);
    k_f2c<<<grid, 256, 0, s>>>(g, lab, q, f2c, cvwgt, ccnt);
    LAUNCHED();
    int64_t *mstart = sc.get<int64_t>(n2);
    int64_t *d_nmem = sc.get<int64_t>(1);
    exclusive_scan(ArrayI32{ccnt}, n2, mstart, d_nmem, sc);
    int64_t nmem = 0;
    CK(cudaMemcpyAsync(&nmem, d_nmem, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int32_t *members = sc.get<int32_t>(nmem);
    int32_t *fill = sc.zeros<int32_t>(n2);
    k_members<<<grid, 256, 0, s>>>(g, f2c, mstart, fill, members);
    LAUNCHED();
    int64_t *mpre = sc.get<int64_t>(nmem + 1);
    exclusive_scan(MemberDeg{g.xadj, members}, nmem, mpre, mpre + nmem, sc);

    // stage 1: slice-wise hash aggregation of quotient edges
    const int cbits = std::max(1, bit_width_u64((uint64_t)(n2 > 1 ? n2 - 1 : 1)));
    const int64_t total = g.nnz;  // every entry belongs to some member row
    unsigned long long *pk = sc.get<unsigned long long>(total);
    int32_t *pw = sc.get<int32_t>(total);
    unsigned long long *d_P = sc.zeros<unsigned long long>(1);
    if (total > 0) {
        auto launch = [&](auto kern, size_t smem) {
            CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int occ = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kCThreads, smem));
            kern<<<sms * std::max(1, occ), kCThreads, smem, s>>>(g, members, nmem, mpre, total, f2c,
                                                                 cbits, pk, pw, d_P);
            LAUNCHED();
        };
        if (cbits <= 20) launch(k_aggregate<true>, sizeof(AggSm<true>));
        else launch(k_aggregate<false>, sizeof(AggSm<false>));
    }
    unsigned long long P = 0;
    CK(cudaMemcpyAsync(&P, d_P, sizeof(P), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    // stage 2: sort by (C(u), C(v)) and reduce equal keys
    radix_sort_pairs((uint64_t *)pk, pw, (int64_t)P, 2 * cbits, sc);
    const int64_t rtiles = ceil_div<int64_t>((int64_t)P, kRTile);
    int64_t *tcnt = sc.get<int64_t>(rtiles + 1);
    int64_t *toff = sc.get<int64_t>(rtiles + 1);
    int64_t m2 = 0;
    if (P > 0) {
        k_run_count<<<(unsigned)rtiles, kRThreads, 0, s>>>(pk, (int64_t)P, tcnt);
        LAUNCHED();
        exclusive_scan(ArrayI64{tcnt}, rtiles, toff, toff + rtiles, sc);
        CK(cudaMemcpyAsync(&m2, toff + rtiles, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    int32_t *adjncy = (int32_t *)out_alloc(m2 * sizeof(int32_t));
    int32_t *adjwgt = (int32_t *)out_alloc(m2 * sizeof(int32_t));
    int32_t *cdeg = sc.zeros<int32_t>(n2);
    if (P > 0) {
        CK(cudaFuncSetAttribute(k_run_emit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(RunSm)));
        k_run_emit<<<(unsigned)rtiles, kRThreads, sizeof(RunSm), s>>>(
            pk, pw, (int64_t)P, toff, cbits, adjncy, adjwgt, cdeg);
        LAUNCHED();
    }
    int64_t *cpre = sc.get<int64_t>(n2);
    exclusive_scan(ArrayI32to64{cdeg}, n2, cpre, nullptr, sc);
    int64_t *xadj = (int64_t *)out_alloc((n2 + 1) * sizeof(int64_t));
    k_finish_xadj<<<grid, 256, 0, s>>>(cpre, n2, m2, xadj);
    LAUNCHED();
    out->n = n2;
    out->nnz = m2;
    out->xadj = xadj;
    out->adjncy = adjncy;
    out->adjwgt = adjwgt;
    out->vwgt = cvwgt;
}

// ---------------------------------------------------------------- projection

__global__ void k_project(int64_t n, const int32_t *f2c, const int32_t *cp, int32_t *fp) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        fp[v] = cp[f2c[v]];
}

void project_impl(int64_t n, const int32_t *f2c, const int32_t *cp, int32_t *fp, cudaStream_t s) {
    if (n <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div<int64_t>(n, 256), dev_info().sms * 8);
    k_project<<<grid, 256, 0, s>>>(n, f2c, cp, fp);
    LAUNCHED();
}

// ---------------------------------------------------------------- cut / balance

// Entries in tiles of kCutTile; block_rows gives each entry's row.
constexpr int kCutTile = 4096;

__global__ void __launch_bounds__(256) k_cut(DGraph g, const int32_t *part, const int64_t *goff,
                                             int64_t groups, unsigned long long *cut) {
    __shared__ int32_t rowof[kCutTile];
    __shared__ int32_t tmp[16];
    const int64_t tiles = ceil_div<int64_t>(g.nnz, kCutTile);
    // a thread's rows only grow (tiles and entries in increasing order), so
    // it keeps one running sum per group and flushes it when the group changes
    int64_t grp = -1, acc = 0, gend = -1;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kCutTile;
        const int len = (int)min64(kCutTile, g.nnz - e0);
        block_rows<256, 16>(g.xadj, g.n, e0, len, rowof, tmp);
        if (groups == 1) {  // all loads of the thread's 16 entries first
            int32_t u[16], w[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int i = threadIdx.x + j * 256;
                u[j] = i < len ? g.adjncy[e0 + i] : 0;
                w[j] = i < len ? g.adjwgt[e0 + i] : 0;
            }
            int32_t pu[16], pv[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int i = threadIdx.x + j * 256;
                pu[j] = i < len ? __ldg(&part[u[j]]) : 0;
                pv[j] = i < len ? __ldg(&part[rowof[i]]) : 0;
            }
#pragma unroll
            for (int j = 0; j < 16; j++) acc += pu[j] != pv[j] ? w[j] : 0;
            __syncthreads();
            continue;
        }
        for (int i = threadIdx.x; i < len; i += 256) {
            const int32_t v = rowof[i];
            if (v >= gend) {  // rows only grow along a thread's entries
                if (acc) atomicAdd(&cut[grp], (unsigned long long)acc);
                acc = 0;
                if (groups == 1) {
                    grp = 0;
                    gend = g.n;
                } else {
                    int64_t lo = 0, hi = groups;  // largest grp with goff[grp] <= v
                    while (hi - lo > 1) {
                        const int64_t mid = (lo + hi) >> 1;
                        if (goff[mid] <= v) lo = mid;
                        else hi = mid;
                    }
                    grp = lo;
                    gend = goff[lo + 1];
                }
            }
            if (part[g.adjncy[e0 + i]] != part[v]) acc += g.adjwgt[e0 + i];
        }
        __syncthreads();
    }
    if (groups == 1) {  // one group: reduce per warp before the atomic
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&cut[0], (unsigned long long)acc);
    } else if (acc) {
        atomicAdd(&cut[grp], (unsigned long long)acc);
    }
}

__global__ void k_halve(unsigned long long *cut, int64_t groups) {
    for (int64_t t = threadIdx.x; t < groups; t += blockDim.x) cut[t] /= 2;
}

// Block weights.  Ids outside [0, nblocks) are skipped, so every write stays
// inside bw[0, nblocks); they are counted in *bad when bad is given.
__global__ void k_bw(DGraph g, const int32_t *part, int64_t nblocks, unsigned long long *bw,
                     unsigned long long *bad) {
    extern __shared__ unsigned long long lbw[];
    const bool local = nblocks <= 2048;
    if (local)
        for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) lbw[b] = 0;
    __syncthreads();
    unsigned long long nbad = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = part[v];
        if (p < 0 || p >= nblocks) {
            nbad++;
            continue;
        }
        if (local) atomicAdd(&lbw[p], (unsigned long long)g.vwgt[v]);
        else atomicAdd(&bw[p], (unsigned long long)g.vwgt[v]);
    }
    if (bad && nbad) atomicAdd(bad, nbad);
    __syncthreads();
    if (local)
        for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x)
            if (lbw[b]) atomicAdd(&bw[b], lbw[b]);
}

void cut_launch(const DGraph &g, const int32_t *part, int64_t nblocks, unsigned long long *d_cut,
                unsigned long long *d_bw, unsigned long long *d_bad, cudaStream_t s, int sms) {
    const int grid = sms * 8;
    if (g.nnz > 0) {
        const int cgrid = (int)std::min<int64_t>(ceil_div<int64_t>(g.nnz, kCutTile), grid);
        k_cut<<<cgrid, 256, 0, s>>>(g, part, nullptr, 1, d_cut);
        LAUNCHED();
        k_halve<<<1, 256, 0, s>>>(d_cut, 1);
        LAUNCHED();
    }
    if (g.n > 0) {
        size_t shm = nblocks <= 2048 ? nblocks * sizeof(unsigned long long) : 0;
        k_bw<<<grid, 256, shm, s>>>(g, part, nblocks, d_bw, d_bad);
        LAUNCHED();
    }
}

void cut_impl(const DGraph &g, const int32_t *part, int64_t nblocks, int64_t groups,
              const int64_t *goff, int64_t *d_cut, int64_t *d_bw, Scratch &sc) {
    cudaStream_t s = sc.stream();
    const int grid = dev_info().sms * 8;
    CK(cudaMemsetAsync(d_cut, 0, groups * sizeof(int64_t), s));
    if (d_bw) CK(cudaMemsetAsync(d_bw, 0, nblocks * sizeof(int64_t), s));
    if (g.nnz > 0) {
        const int cgrid = (int)std::min<int64_t>(ceil_div<int64_t>(g.nnz, kCutTile), grid);
        k_cut<<<cgrid, 256, 0, s>>>(g, part, goff, groups, (unsigned long long *)d_cut);
        LAUNCHED();
        k_halve<<<1, 256, 0, s>>>((unsigned long long *)d_cut, groups);
        LAUNCHED();
    }
    if (d_bw && g.n > 0) {
        size_t shm = nblocks <= 2048 ? nblocks * sizeof(unsigned long long) : 0;
        k_bw<<<grid, 256, shm, s>>>(g, part, nblocks, (unsigned long long *)d_bw, nullptr);
        LAUNCHED();
    }
}

}  // namespace sclap
