// lp.cu -- the SCLaP sweep: per-round sub-round worklists, degree-binned
// neighbour-label aggregation (propose), exact capacity arbitration and the
// simultaneous apply.  Clustering and refinement share the machinery; the
// refinement form adds the overloaded-block rule (Sec. III.A).
//
// Per round r:
//   k_build_wl    every node with >= 1 neighbour goes to bucket
//                 2*colour + (deg > kHubDeg), colour = (h(v,r) >> 32) mod S.
// Per sub-round j:
//   k_propose     normal nodes: CTA items of kItemNodes worklist nodes, split
//                 into chunks of <= kChunkEntries entries; a shared-memory
//                 open-addressing (linear probing) table keyed by (node slot,
//                 label) accumulates omega(v, L); the best eligible label per
//                 node comes from a 64-bit atomicMax over (omega, ~tie) and an
//                 atomicMin over labels on exact ties.  Hub nodes run in a
//                 second launch on a side stream, one CTA per node, with a
//                 global-memory table when the row exceeds shared memory.
//                 The dense variant (k <= 64 blocks) accumulates into a
//                 per-node k-array instead of a hash table.
//   k_src         refinement only: departures from overloaded blocks.
//   k_classify    uncontested targets (sum of proposed weight <= capacity)
//                 are applied at once; contested targets get a segment.
//   k_scatter     contested proposals are written to their target's segment.
//   k_arbitrate   per contested target: weighted radix select of the first
//                 key (gain desc, id asc) whose inclusive prefix exceeds the
//                 capacity; admitted moves are applied; per-target counters
//                 are reset.
#include <algorithm>

#include "lp.cuh"
#include "prims.cuh"

namespace sclap {

// ---------------------------------------------------------------- tunables

constexpr int kThreads = 256;
constexpr int kItemNodes = 256;       // worklist nodes per CTA work item
constexpr int kHubDeg = 512;          // degree above which a node is a hub
constexpr int kChunkEntries = 2048;   // entries per shared-memory chunk (max)
constexpr int kChunkTarget = kChunkEntries - kHubDeg;  // chunking step
constexpr int kTableSlots = 4096;     // >= 2 * kChunkEntries
constexpr int kTableBits = 12;
constexpr int kDenseMaxK = 64;
constexpr int kDenseItemNodes = 128;
constexpr uint64_t kEmpty = ~0ull;

static_assert((1 << kTableBits) == kTableSlots, "table size");
static_assert(kTableSlots >= 2 * kChunkEntries, "load factor");

struct Prop {
    int32_t v, T, own, gain;
    int32_t c, slot;  // slot: rank among the target's proposals; -2 pending source rule; -1 rejected
    int64_t wT;       // W(T) at sub-round start
};

struct SegEntry {
    uint64_t key;  // (0x7fffffff - gain) << 32 | v : ascending = (gain desc, id asc)
    int32_t c, own;
};

struct Seg {
    int32_t T, cnt;
    int64_t base, thr;  // thr = capacity + 1
};

struct Ctr {
    int32_t nprop, nseg;
    int64_t segtotal;
    int32_t item_next, hub_next;
    int32_t err, pad;
};

struct LPArgs {
    DGraph g;
    int32_t *lab;
    int64_t *W;
    int64_t B, nW;
    const int32_t *cp;
    uint64_t seed;
    int32_t round;
    const int32_t *wl;      // this bucket's worklist
    const int32_t *wl_cnt;  // its length (device)
    Prop *props;
    Ctr *ctr;
    int64_t *tsum;
    int32_t *tcnt;
    int64_t *tbase;
    int64_t *ssum;
    Seg *segs;
    SegEntry *segbuf;
    int64_t *moves;         // moves of this round
    // hub tables (global, one region per hub CTA)
    unsigned long long *gkeys;
    int32_t *gvals;
    int32_t *gdl;
    int64_t gcap;
    int gbits;
    unsigned long long *prof;  // [2] entries, nodes (normal items), or null
};

__device__ __forceinline__ uint64_t seg_key(int32_t gain, int32_t v) {
    return ((uint64_t)(uint32_t)(0x7fffffff - gain) << 32) | (uint32_t)v;
}

__device__ __forceinline__ uint32_t table_hash(uint64_t key, int bits) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

__device__ __forceinline__ uint32_t tie_of(uint64_t h, int32_t L) {
    return (uint32_t)(mix64(h ^ (uint64_t)(uint32_t)L) >> 32);
}

// Applies one admitted move (Sec. III.A: the node joins the target; weights
// move with it).
__device__ __forceinline__ void apply_move(const LPArgs &a, int32_t v, int32_t T, int32_t own,
                                           int32_t c) {
    a.lab[v] = T;
    atomicAdd((unsigned long long *)&a.W[T], (unsigned long long)(int64_t)c);
    atomicAdd((unsigned long long *)&a.W[own], (unsigned long long)(-(int64_t)c));
}

// ---------------------------------------------------------------- worklists

__global__ void __launch_bounds__(kThreads)
    k_build_wl(DGraph g, uint64_t seed, int32_t round, int32_t S, int32_t *wl, int32_t *cnt) {
    __shared__ int lcnt[64], lbase[64];
    const int nb = 2 * S;
    for (int64_t tile = (int64_t)blockIdx.x * kThreads * 4; tile < g.n;
         tile += (int64_t)gridDim.x * kThreads * 4) {
        for (int i = threadIdx.x; i < nb; i += kThreads) lcnt[i] = 0;
        __syncthreads();
        int bk[4], rk[4];
        int32_t vv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int64_t v = tile + (int64_t)j * kThreads + threadIdx.x;
            bk[j] = -1;
            vv[j] = (int32_t)v;
            if (v < g.n) {
                int64_t d = g.xadj[v + 1] - g.xadj[v];
                if (d > 0) {
                    uint32_t col = (uint32_t)(node_hash(seed, round, (uint32_t)v) >> 32) % (uint32_t)S;
                    bk[j] = 2 * (int)col + (d > kHubDeg ? 1 : 0);
                    rk[j] = atomicAdd(&lcnt[bk[j]], 1);
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += kThreads)
            lbase[i] = lcnt[i] ? atomicAdd(&cnt[i], lcnt[i]) : 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (bk[j] >= 0) wl[(int64_t)bk[j] * g.n + lbase[bk[j]] + rk[j]] = vv[j];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- propose (hash tables)

struct NodeSm {
    int32_t v[kItemNodes];
    int32_t own[kItemNodes];
    int32_t c[kItemNodes];
    int32_t cpv[kItemNodes];
    int32_t ownw[kItemNodes];
    int32_t bestL[kItemNodes];
    int32_t epre[kItemNodes + 1];
    int64_t rs[kItemNodes];
    uint64_t h[kItemNodes];
    unsigned long long best[kItemNodes];
    uint8_t ovl[kItemNodes];
};

struct HashSm {
    unsigned long long keys[kTableSlots];
    int32_t vals[kTableSlots];
    int32_t dl[kChunkEntries];
    NodeSm nd;
    int64_t scan_tmp[kThreads / 32 + 1];
    int ndl;
    int item;
    int ns;
    int64_t E;
};

// Index of the node slot owning entry e: largest s in [lo, hi) with epre[s] <= e.
__device__ __forceinline__ int owner_slot(const int32_t *epre, int lo, int hi, int32_t e) {
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (epre[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Inserts (key, w) into a linear-probing table; records first insertions in dl.
__device__ __forceinline__ bool table_add(unsigned long long *keys, int32_t *vals, int32_t *dl,
                                          int *ndl, uint32_t mask, int bits, uint64_t key,
                                          int32_t w) {
    uint32_t slot = table_hash(key, bits);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        unsigned long long prev = atomicCAS(&keys[slot], kEmpty, (unsigned long long)key);
        if (prev == kEmpty || prev == key) {
            atomicAdd(&vals[slot], w);
            if (prev == kEmpty) dl[atomicAdd(ndl, 1)] = (int32_t)slot;
            return true;
        }
        slot = (slot + 1) & mask;
    }
    return false;  // table full: cannot happen at load factor <= 1/2
}

// Emits the proposal of node slot s if `active` and the node proposes.  Every
// lane of the warp must call it (warp-aggregated append).
template <bool REFINE>
__device__ __forceinline__ void emit_hash(const LPArgs &a, NodeSm &nd, int s, bool active) {
    unsigned long long b = active ? nd.best[s] : 0ull;
    bool prop = false;
    int32_t L = 0, gain = 0;
    if (b != 0) {
        L = nd.bestL[s];
        gain = (int32_t)(b >> 32) - nd.ownw[s];
        prop = gain > 0 || (REFINE && nd.ovl[s]);
    }
    unsigned m = __ballot_sync(0xffffffffu, prop);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(&a.ctr->nprop, __popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (!prop) return;
    int pos = base + __popc(m & ((1u << lane) - 1));
    Prop p;
    p.v = nd.v[s];
    p.T = L;
    p.own = nd.own[s];
    p.gain = gain;
    p.c = nd.c[s];
    p.wT = a.W[L];
    if (REFINE && nd.ovl[s]) {
        atomicAdd((unsigned long long *)&a.ssum[p.own], (unsigned long long)(int64_t)p.c);
        p.slot = -2;
    } else {
        atomicAdd((unsigned long long *)&a.tsum[L], (unsigned long long)(int64_t)p.c);
        p.slot = atomicAdd(&a.tcnt[L], 1);
    }
    a.props[pos] = p;
}

// Selection over the distinct (slot, label) entries of the current chunk.
template <bool REFINE>
__device__ __forceinline__ void select_best(const LPArgs &a, const unsigned long long *keys,
                                            const int32_t *vals, const int32_t *dl, int ndl,
                                            NodeSm &nd) {
    for (int i = threadIdx.x; i < ndl; i += kThreads) {
        int32_t slot = dl[i];
        uint64_t key = keys[slot];
        int s = (int)(key >> 32);
        int32_t L = (int32_t)(uint32_t)key;
        int32_t w = vals[slot];
        if (L == nd.own[s]) {
            nd.ownw[s] = w;
        } else if (a.W[L] + nd.c[s] <= a.B) {
            unsigned long long ck =
                ((unsigned long long)(uint32_t)w << 32) | (uint32_t)~tie_of(nd.h[s], L);
            atomicMax(&nd.best[s], ck);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ndl; i += kThreads) {
        int32_t slot = dl[i];
        uint64_t key = keys[slot];
        int s = (int)(key >> 32);
        int32_t L = (int32_t)(uint32_t)key;
        unsigned long long b = nd.best[s];
        if (b == 0 || L == nd.own[s] || (uint32_t)vals[slot] != (uint32_t)(b >> 32)) continue;
        if (a.W[L] + nd.c[s] > a.B) continue;
        unsigned long long ck =
            ((unsigned long long)(uint32_t)vals[slot] << 32) | (uint32_t)~tie_of(nd.h[s], L);
        if (ck == b) atomicMin(&nd.bestL[s], L);
    }
    __syncthreads();
}

template <bool REFINE>
__device__ void load_nodes(const LPArgs &a, NodeSm &nd, int64_t i0, int ns, int64_t *scan_tmp,
                           int64_t *E_out) {
    int32_t deg = 0;
    int t = threadIdx.x;
    if (t < ns) {
        int32_t v = a.wl[i0 + t];
        nd.v[t] = v;
        int64_t b = a.g.xadj[v];
        nd.rs[t] = b;
        deg = (int32_t)(a.g.xadj[v + 1] - b);
        int32_t own = a.lab[v];
        nd.own[t] = own;
        nd.c[t] = a.g.vwgt[v];
        nd.cpv[t] = a.cp ? a.cp[v] : 0;
        nd.h[t] = node_hash(a.seed, a.round, (uint32_t)v);
        nd.ovl[t] = REFINE ? (a.W[own] > a.B) : 0;
    }
    if (t < kItemNodes) {
        nd.ownw[t] = 0;
        nd.best[t] = 0;
        nd.bestL[t] = 0x7fffffff;
    }
    int64_t tot;
    int64_t pre = block_exclusive_scan<kThreads>((int64_t)deg, &tot, scan_tmp);
    if (t < ns) nd.epre[t] = (int32_t)pre;
    if (t == 0) nd.epre[ns] = (int32_t)tot;
    *E_out = tot;
    __syncthreads();
}

template <bool REFINE>
__global__ void __launch_bounds__(kThreads, 3) k_propose_hash(LPArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    HashSm &sm = *reinterpret_cast<HashSm *>(smraw);
    for (int i = threadIdx.x; i < kTableSlots; i += kThreads) {
        sm.keys[i] = kEmpty;
        sm.vals[i] = 0;
    }
    const int64_t nwl = *a.wl_cnt;
    const int items = (int)ceil_div<int64_t>(nwl, kItemNodes);
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) sm.item = atomicAdd(&a.ctr->item_next, 1);
        __syncthreads();
        const int item = sm.item;
        if (item >= items) break;
        const int64_t i0 = (int64_t)item * kItemNodes;
        const int ns = (int)min64(kItemNodes, nwl - i0);
        int64_t E;
        load_nodes<REFINE>(a, sm.nd, i0, ns, sm.scan_tmp, &E);
        if (a.prof && threadIdx.x == 0) {
            atomicAdd(&a.prof[0], (unsigned long long)E);
            atomicAdd(&a.prof[1], (unsigned long long)ns);
        }
        // chunks: node s belongs to chunk epre[s] / kChunkTarget
        const int nchunks = (int)(sm.nd.epre[ns - 1] / kChunkTarget) + 1;
        int s0 = 0;
        for (int ch = 0; ch < nchunks; ch++) {
            // s1 = first slot with epre[s] >= (ch + 1) * kChunkTarget
            int32_t lim = (ch + 1) * kChunkTarget;
            int lo = s0, hi = ns;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sm.nd.epre[mid] >= lim) hi = mid;
                else lo = mid + 1;
            }
            const int s1 = lo;
            if (s1 == s0) continue;
            if (threadIdx.x == 0) sm.ndl = 0;
            __syncthreads();
            const int32_t e0 = sm.nd.epre[s0], e1 = sm.nd.epre[s1];
            for (int32_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
                int s = owner_slot(sm.nd.epre, s0, s1, e);
                int64_t idx = sm.nd.rs[s] + (e - sm.nd.epre[s]);
                int32_t u = __ldg(&a.g.adjncy[idx]);
                int32_t w = __ldg(&a.g.adjwgt[idx]);
                if (a.cp && __ldg(&a.cp[u]) != sm.nd.cpv[s]) continue;
                int32_t L = __ldg(&a.lab[u]);
                uint64_t key = ((uint64_t)(uint32_t)s << 32) | (uint32_t)L;
                if (!table_add(sm.keys, sm.vals, sm.dl, &sm.ndl, kTableSlots - 1, kTableBits, key, w))
                    a.ctr->err = 1;
            }
            __syncthreads();
            const int ndl = sm.ndl;
            select_best<REFINE>(a, sm.keys, sm.vals, sm.dl, ndl, sm.nd);
            // emit: every thread takes part (warp-aggregated appends)
            for (int base = s0; base < s1; base += kThreads)
                emit_hash<REFINE>(a, sm.nd, base + threadIdx.x, base + (int)threadIdx.x < s1);
            for (int i = threadIdx.x; i < ndl; i += kThreads) {
                int32_t slot = sm.dl[i];
                sm.keys[slot] = kEmpty;
                sm.vals[slot] = 0;
            }
            s0 = s1;
            __syncthreads();
        }
    }
}

// Hub nodes: one CTA per node; the row's (label, omega) table lives in shared
// memory when deg <= kChunkEntries, otherwise in this CTA's global region.
template <bool REFINE>
__global__ void __launch_bounds__(kThreads) k_propose_hub(LPArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    HashSm &sm = *reinterpret_cast<HashSm *>(smraw);
    for (int i = threadIdx.x; i < kTableSlots; i += kThreads) {
        sm.keys[i] = kEmpty;
        sm.vals[i] = 0;
    }
    const int64_t nwl = *a.wl_cnt;
    unsigned long long *gk = a.gkeys ? a.gkeys + (int64_t)blockIdx.x * a.gcap : nullptr;
    int32_t *gv = a.gvals ? a.gvals + (int64_t)blockIdx.x * a.gcap : nullptr;
    int32_t *gdl = a.gdl ? a.gdl + (int64_t)blockIdx.x * (a.gcap / 2) : nullptr;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) sm.item = atomicAdd(&a.ctr->hub_next, 1);
        __syncthreads();
        const int item = sm.item;
        if (item >= nwl) break;
        int64_t E;
        load_nodes<REFINE>(a, sm.nd, item, 1, sm.scan_tmp, &E);
        const bool global = E > kChunkEntries;
        unsigned long long *keys = global ? gk : sm.keys;
        int32_t *vals = global ? gv : sm.vals;
        int32_t *dl = global ? gdl : sm.dl;
        const uint32_t mask = global ? (uint32_t)(a.gcap - 1) : (kTableSlots - 1);
        const int bits = global ? a.gbits : kTableBits;
        if (threadIdx.x == 0) sm.ndl = 0;
        __syncthreads();
        const int64_t rs = sm.nd.rs[0];
        const int32_t cpv = sm.nd.cpv[0];
        for (int64_t e = threadIdx.x; e < E; e += kThreads) {
            int32_t u = __ldg(&a.g.adjncy[rs + e]);
            int32_t w = __ldg(&a.g.adjwgt[rs + e]);
            if (a.cp && __ldg(&a.cp[u]) != cpv) continue;
            int32_t L = __ldg(&a.lab[u]);
            if (!table_add(keys, vals, dl, &sm.ndl, mask, bits, (uint64_t)(uint32_t)L, w))
                a.ctr->err = 1;
        }
        __syncthreads();
        const int ndl = sm.ndl;
        select_best<REFINE>(a, keys, vals, dl, ndl, sm.nd);
        if (threadIdx.x < 32) emit_hash<REFINE>(a, sm.nd, 0, threadIdx.x == 0);
        for (int i = threadIdx.x; i < ndl; i += kThreads) {
            int32_t slot = dl[i];
            keys[slot] = kEmpty;
            vals[slot] = 0;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- propose (dense k <= 64)

struct DenseSm {
    int32_t acc[kDenseItemNodes * kDenseMaxK];
    int64_t W[kDenseMaxK];
    int32_t v[kDenseItemNodes], own[kDenseItemNodes], c[kDenseItemNodes];
    int32_t epre[kDenseItemNodes + 1];
    int64_t rs[kDenseItemNodes];
    uint64_t h[kDenseItemNodes];
    // staged proposals of the item
    int32_t pT[kDenseItemNodes], pgain[kDenseItemNodes], pslot[kDenseItemNodes];
    uint8_t povl[kDenseItemNodes], pflag[kDenseItemNodes];
    int32_t lcnt[kDenseMaxK];
    int64_t lsum[kDenseMaxK];
    int64_t lssum[kDenseMaxK];
    int32_t gbase[kDenseMaxK];
    int64_t scan_tmp[kThreads / 32 + 1];
    int item, nprop, pbase;
};

template <bool HUB>
__global__ void __launch_bounds__(kThreads) k_propose_dense(LPArgs a, int k) {
    extern __shared__ __align__(16) unsigned char smraw[];
    DenseSm &sm = *reinterpret_cast<DenseSm *>(smraw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kDenseItemNodes * k; i += kThreads) sm.acc[i] = 0;
    for (int b = threadIdx.x; b < k; b += kThreads) {
        sm.W[b] = a.W[b];
        sm.lcnt[b] = 0;
        sm.lsum[b] = 0;
        sm.lssum[b] = 0;
    }
    const int64_t nwl = *a.wl_cnt;
    const int items = HUB ? (int)nwl : (int)ceil_div<int64_t>(nwl, kDenseItemNodes);
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            sm.item = atomicAdd(HUB ? &a.ctr->hub_next : &a.ctr->item_next, 1);
            sm.nprop = 0;
        }
        __syncthreads();
        const int item = sm.item;
        if (item >= items) break;
        const int64_t i0 = HUB ? item : (int64_t)item * kDenseItemNodes;
        const int ns = HUB ? 1 : (int)min64(kDenseItemNodes, nwl - i0);
        int32_t deg = 0;
        const int t = threadIdx.x;
        if (t < ns) {
            int32_t v = a.wl[i0 + t];
            sm.v[t] = v;
            int64_t b = a.g.xadj[v];
            sm.rs[t] = b;
            deg = (int32_t)(a.g.xadj[v + 1] - b);
            sm.own[t] = a.lab[v];
            sm.c[t] = a.g.vwgt[v];
            sm.h[t] = node_hash(a.seed, a.round, (uint32_t)v);
        }
        int64_t E;
        int64_t pre = block_exclusive_scan<kThreads>((int64_t)deg, &E, sm.scan_tmp);
        if (t < ns) sm.epre[t] = (int32_t)pre;
        if (t == 0) sm.epre[ns] = (int32_t)E;
        if (!HUB && a.prof && t == 0) {
            atomicAdd(&a.prof[0], (unsigned long long)E);
            atomicAdd(&a.prof[1], (unsigned long long)ns);
        }
        __syncthreads();
        // accumulate omega(v, b) for every entry of the item
        for (int64_t e = t; e < E; e += kThreads) {
            int s = HUB ? 0 : owner_slot(sm.epre, 0, ns, (int32_t)e);
            int64_t idx = sm.rs[s] + (e - sm.epre[s]);
            int32_t u = __ldg(&a.g.adjncy[idx]);
            int32_t w = __ldg(&a.g.adjwgt[idx]);
            int32_t L = __ldg(&a.lab[u]);
            atomicAdd(&sm.acc[s * k + L], w);
        }
        __syncthreads();
        // selection: one warp per node, lanes over blocks b = lane, lane + 32
        for (int s = warp; s < ns; s += kThreads / 32) {
            const int32_t own = sm.own[s], c = sm.c[s];
            const uint64_t h = sm.h[s];
            int32_t w0 = lane < k ? sm.acc[s * k + lane] : 0;
            int32_t w1 = lane + 32 < k ? sm.acc[s * k + lane + 32] : 0;
            __syncwarp();
            if (lane < k) sm.acc[s * k + lane] = 0;
            if (lane + 32 < k) sm.acc[s * k + lane + 32] = 0;
            int32_t ownw = __shfl_sync(0xffffffffu, (own < 32) ? w0 : w1, own & 31);
            unsigned long long ck0 = 0, ck1 = 0;
            if (w0 > 0 && lane != own && sm.W[lane] + c <= a.B)
                ck0 = ((unsigned long long)(uint32_t)w0 << 32) | (uint32_t)~tie_of(h, lane);
            if (w1 > 0 && lane + 32 != own && sm.W[lane + 32] + c <= a.B)
                ck1 = ((unsigned long long)(uint32_t)w1 << 32) | (uint32_t)~tie_of(h, lane + 32);
            unsigned long long m = ck0 > ck1 ? ck0 : ck1;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                unsigned long long o = __shfl_xor_sync(0xffffffffu, m, d);
                m = o > m ? o : m;
            }
            int32_t L = 0x7fffffff;
            if (m != 0) {
                if (ck0 == m) L = lane;
                else if (ck1 == m) L = lane + 32;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) L = min(L, __shfl_xor_sync(0xffffffffu, L, d));
            }
            if (lane == 0) {
                bool ovl = sm.W[own] > a.B;
                int32_t gain = (int32_t)(m >> 32) - ownw;
                bool prop = m != 0 && (gain > 0 || ovl);
                sm.pflag[s] = prop;
                if (prop) {
                    sm.pT[s] = L;
                    sm.pgain[s] = gain;
                    sm.povl[s] = ovl;
                    atomicAdd(&sm.nprop, 1);
                    if (ovl) {
                        atomicAdd((unsigned long long *)&sm.lssum[own], (unsigned long long)c);
                        sm.pslot[s] = -2;
                    } else {
                        atomicAdd((unsigned long long *)&sm.lsum[L], (unsigned long long)c);
                        sm.pslot[s] = atomicAdd(&sm.lcnt[L], 1);
                    }
                }
            }
        }
        __syncthreads();
        if (sm.nprop == 0) continue;
        for (int b = threadIdx.x; b < k; b += kThreads) {
            if (sm.lcnt[b]) {
                sm.gbase[b] = atomicAdd(&a.tcnt[b], sm.lcnt[b]);
                atomicAdd((unsigned long long *)&a.tsum[b], (unsigned long long)sm.lsum[b]);
            }
            if (sm.lssum[b]) atomicAdd((unsigned long long *)&a.ssum[b], (unsigned long long)sm.lssum[b]);
            sm.lcnt[b] = 0;
            sm.lsum[b] = 0;
            sm.lssum[b] = 0;
        }
        if (threadIdx.x == 0) sm.pbase = atomicAdd(&a.ctr->nprop, sm.nprop);
        if (threadIdx.x == 0) sm.nprop = 0;
        __syncthreads();
        // write the staged proposals (positions by a block scan over flags)
        int flag = (t < ns) ? sm.pflag[t] : 0;
        int64_t tot;
        int64_t pos = block_exclusive_scan<kThreads>((int64_t)flag, &tot, sm.scan_tmp);
        if (flag) {
            Prop p;
            p.v = sm.v[t];
            p.T = sm.pT[t];
            p.own = sm.own[t];
            p.gain = sm.pgain[t];
            p.c = sm.c[t];
            p.slot = sm.pslot[t] >= 0 ? sm.gbase[p.T] + sm.pslot[t] : -2;
            p.wT = sm.W[p.T];
            a.props[sm.pbase + pos] = p;
        }
    }
}

// ---------------------------------------------------------------- arbitration

// Weighted radix select: the smallest key K such that the total weight of
// entries with key <= K is >= thr (entries (key, c) in [0, cnt)); ~0 if the
// total is < thr.  All threads of the CTA call it.
template <typename Get>
__device__ uint64_t select_first_reaching(Get get, int64_t cnt, int64_t thr,
                                          unsigned long long *hist /* [256] */,
                                          int64_t *shared_acc, uint64_t *shared_prefix,
                                          int *shared_done) {
    if (threadIdx.x == 0) {
        *shared_acc = 0;
        *shared_prefix = 0;
        *shared_done = 0;
    }
    __syncthreads();
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t hm = (shift == 56) ? 0ull : (~0ull << (shift + 8));
        const uint64_t pf = *shared_prefix;
        for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            uint64_t k;
            int32_t c;
            get(i, &k, &c);
            if ((k & hm) == (pf & hm) && c > 0)
                atomicAdd(&hist[(k >> shift) & 255], (unsigned long long)c);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            unsigned long long local = 0;
            for (int j = 0; j < 8; j++) local += hist[lane * 8 + j];
            unsigned long long inc = local;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
            const int64_t acc = *shared_acc;
            bool reach = acc + (int64_t)inc >= thr;
            unsigned m = __ballot_sync(0xffffffffu, reach);
            if (m == 0) {
                if (lane == 0) *shared_done = 1;  // total below threshold
            } else {
                int first = __ffs(m) - 1;
                if (lane == first) {
                    int64_t run = acc + (int64_t)(inc - local);
                    int d = lane * 8;
                    for (int j = 0; j < 8; j++) {
                        if (run + (int64_t)hist[lane * 8 + j] >= thr) { d = lane * 8 + j; break; }
                        run += (int64_t)hist[lane * 8 + j];
                    }
                    *shared_acc = run;
                    *shared_prefix = pf | ((uint64_t)d << shift);
                }
            }
        }
        __syncthreads();
        if (*shared_done) return ~0ull;
    }
    return *shared_prefix;
}

// Refinement: departures from overloaded blocks (slot == -2).  CTAs with
// blockIdx < nW handle block b = blockIdx when its departures are contested;
// the others pass the uncontested sources' proposals through.
__global__ void __launch_bounds__(kThreads) k_src(LPArgs a) {
    __shared__ unsigned long long hist[256];
    __shared__ int64_t s_acc;
    __shared__ uint64_t s_pf;
    __shared__ int s_done;
    const int nprop = a.ctr->nprop;
    if (blockIdx.x < a.nW) {
        const int32_t b = blockIdx.x;
        const int64_t Wb = a.W[b];
        if (Wb <= a.B) return;
        const int64_t X = Wb - a.B;
        if (a.ssum[b] < X) return;  // uncontested: handled by the pass-through CTAs
        auto get = [&](int64_t i, uint64_t *k, int32_t *c) {
            const Prop &p = a.props[i];
            bool mine = p.slot == -2 && p.own == b;
            *k = mine ? seg_key(p.gain, p.v) : 0;
            *c = mine ? p.c : 0;
        };
        uint64_t K = select_first_reaching(get, nprop, X, hist, &s_acc, &s_pf, &s_done);
        for (int64_t i = threadIdx.x; i < nprop; i += blockDim.x) {
            Prop &p = a.props[i];
            if (p.slot != -2 || p.own != b) continue;
            if (seg_key(p.gain, p.v) <= K) {
                atomicAdd((unsigned long long *)&a.tsum[p.T], (unsigned long long)(int64_t)p.c);
                p.slot = atomicAdd(&a.tcnt[p.T], 1);
            } else {
                p.slot = -1;
            }
        }
        return;
    }
    for (int64_t i = (int64_t)(blockIdx.x - a.nW) * blockDim.x + threadIdx.x; i < nprop;
         i += (int64_t)(gridDim.x - a.nW) * blockDim.x) {
        Prop &p = a.props[i];
        if (p.slot != -2) continue;
        if (a.ssum[p.own] < a.W[p.own] - a.B) {
            atomicAdd((unsigned long long *)&a.tsum[p.T], (unsigned long long)(int64_t)p.c);
            p.slot = atomicAdd(&a.tcnt[p.T], 1);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_classify(LPArgs a) {
    const int nprop = a.ctr->nprop;
    int64_t moved = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nprop;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Prop p = a.props[i];
        if (p.slot < 0) continue;
        const int64_t cap = a.B - p.wT;
        if (a.tsum[p.T] <= cap) {
            apply_move(a, p.v, p.T, p.own, p.c);
            moved++;
        } else if (p.slot == 0) {
            const int32_t cnt = a.tcnt[p.T];
            const int si = atomicAdd(&a.ctr->nseg, 1);
            const int64_t base = (int64_t)atomicAdd((unsigned long long *)&a.ctr->segtotal,
                                                    (unsigned long long)cnt);
            a.tbase[p.T] = base;
            a.segs[si] = Seg{p.T, cnt, base, cap + 1};
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) moved += __shfl_down_sync(0xffffffffu, moved, d);
    if ((threadIdx.x & 31) == 0 && moved) atomicAdd((unsigned long long *)a.moves, (unsigned long long)moved);
}

__global__ void __launch_bounds__(kThreads) k_scatter(LPArgs a) {
    const int nprop = a.ctr->nprop;
    if (a.ctr->nseg == 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nprop;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Prop p = a.props[i];
        if (p.slot < 0) continue;
        if (a.tsum[p.T] <= a.B - p.wT) continue;
        a.segbuf[a.tbase[p.T] + p.slot] = SegEntry{seg_key(p.gain, p.v), p.c, p.own};
    }
}

__global__ void __launch_bounds__(kThreads) k_arbitrate(LPArgs a) {
    __shared__ unsigned long long hist[256];
    __shared__ int64_t s_acc;
    __shared__ uint64_t s_pf;
    __shared__ int s_done;
    const int nseg = a.ctr->nseg;
    const int lane = threadIdx.x & 31;
    int64_t moved = 0;
    // small segments: one warp each, exact prefix by brute force over <= 32 lanes
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int si = gwarp; si < nseg; si += nwarps) {
        const Seg sg = a.segs[si];
        if (sg.cnt > 32) continue;
        uint64_t key = ~0ull;
        int32_t c = 0, own = 0;
        if (lane < sg.cnt) {
            SegEntry e = a.segbuf[sg.base + lane];
            key = e.key;
            c = e.c;
            own = e.own;
        }
        int64_t pre = 0;
        for (int j = 0; j < sg.cnt; j++) {
            uint64_t kj = __shfl_sync(0xffffffffu, key, j);
            int32_t cj = __shfl_sync(0xffffffffu, c, j);
            if (kj <= key) pre += cj;
        }
        if (lane < sg.cnt && (c == 0 || pre < sg.thr)) {
            apply_move(a, (int32_t)(uint32_t)key, sg.T, own, c);
            moved++;
        }
    }
    // larger segments: one CTA each
    for (int si = blockIdx.x; si < nseg; si += gridDim.x) {
        const Seg sg = a.segs[si];
        if (sg.cnt <= 32) continue;
        const SegEntry *ent = a.segbuf + sg.base;
        auto get = [&](int64_t i, uint64_t *k, int32_t *c) {
            SegEntry e = ent[i];
            *k = e.key;
            *c = e.c;
        };
        uint64_t K = select_first_reaching(get, sg.cnt, sg.thr, hist, &s_acc, &s_pf, &s_done);
        for (int64_t i = threadIdx.x; i < sg.cnt; i += blockDim.x) {
            SegEntry e = ent[i];
            if (e.key < K || e.c == 0) {
                apply_move(a, (int32_t)(uint32_t)e.key, sg.T, e.own, e.c);
                moved++;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) moved += __shfl_down_sync(0xffffffffu, moved, d);
    if (lane == 0 && moved) atomicAdd((unsigned long long *)a.moves, (unsigned long long)moved);
}

// Clears the per-target (and per-source) accumulators touched this sub-round.
__global__ void __launch_bounds__(kThreads) k_reset_targets(LPArgs a) {
    const int nprop = a.ctr->nprop;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nprop;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Prop p = a.props[i];
        a.tsum[p.T] = 0;
        a.tcnt[p.T] = 0;
        if (a.ssum) a.ssum[p.own] = 0;
    }
}

// ---------------------------------------------------------------- weights

__global__ void k_init_cluster(DGraph g, int32_t *lab, int64_t *W) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        lab[v] = (int32_t)v;
        W[v] = g.vwgt[v];
    }
}

__global__ void k_block_weights(DGraph g, const int32_t *lab, int64_t *W, int64_t nW) {
    extern __shared__ unsigned long long lw[];
    const bool local = nW <= 1024;
    if (local)
        for (int i = threadIdx.x; i < nW; i += blockDim.x) lw[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (local) atomicAdd(&lw[lab[v]], (unsigned long long)g.vwgt[v]);
        else atomicAdd((unsigned long long *)&W[lab[v]], (unsigned long long)g.vwgt[v]);
    }
    __syncthreads();
    if (local)
        for (int i = threadIdx.x; i < nW; i += blockDim.x)
            if (lw[i]) atomicAdd((unsigned long long *)&W[i], lw[i]);
}

// ---------------------------------------------------------------- isolated nodes

// The paper is silent on nodes without neighbours: label propagation never
// moves them, so they would stay singleton clusters and stall coarsening.
// After the rounds they are packed in id order (per block of cp when given):
// with U' = U - cmax + 1 (cmax: largest weight among them) and P(v) the weight
// of the earlier ones in the same block, v joins group floor(P(v) / U'), whose
// label is its smallest id; a group weighs at most U.

struct IsoFlag {
    const int64_t *xadj;
    __device__ int64_t operator()(int64_t v) const { return xadj[v + 1] == xadj[v] ? 1 : 0; }
};

__global__ void k_iso_compact(DGraph g, const int64_t *pos, const int32_t *cp, int32_t *iso,
                              uint64_t *key, unsigned long long *cmax) {
    unsigned long long m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (g.xadj[v + 1] != g.xadj[v]) continue;
        int64_t i = pos[v];
        iso[i] = (int32_t)v;
        key[i] = cp ? (uint64_t)((uint32_t)cp[v] ^ 0x80000000u) : 0;
        m = max(m, (unsigned long long)g.vwgt[v]);
    }
    if (m) atomicMax(cmax, m);
}

struct IsoWeight {
    const int32_t *iso, *vwgt;
    __device__ int64_t operator()(int64_t i) const { return vwgt[iso[i]]; }
};

struct SegStart {
    const uint64_t *key;
    __device__ int64_t operator()(int64_t i) const { return (i == 0 || key[i] != key[i - 1]) ? 1 : 0; }
};

__global__ void k_iso_segbase(int64_t ni, const uint64_t *key, const int64_t *P, const int64_t *sidx,
                              int64_t *segP) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni;
         i += (int64_t)gridDim.x * blockDim.x)
        if (i == 0 || key[i] != key[i - 1]) segP[sidx[i]] = P[i];
}

struct GroupStart {
    const uint64_t *key;
    const int64_t *P, *sidx, *segP;
    int64_t Up;
    __device__ int64_t group(int64_t i) const {
        int64_t s = sidx[i] + ((i == 0 || key[i] != key[i - 1]) ? 1 : 0) - 1;
        return (P[i] - segP[s]) / Up;
    }
    __device__ int64_t operator()(int64_t i) const {
        if (i == 0 || key[i] != key[i - 1]) return 1;
        return group(i) != group(i - 1) ? 1 : 0;
    }
};

__global__ void k_iso_label(int64_t ni, const int32_t *iso, GroupStart gs, const int64_t *gidx,
                            int32_t *rep, int32_t *lab, int pass) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t st = gs(i);
        int64_t gi = gidx[i] + st - 1;
        if (pass == 0) {
            if (st) rep[gi] = iso[i];
        } else {
            lab[iso[i]] = rep[gi];
        }
    }
}

void pack_isolated(const DGraph &g, const int32_t *cp, int64_t U, int32_t *lab, Scratch &sc) {
    cudaStream_t s = sc.stream();
    if (g.n == 0) return;
    const int grid = dev_info().sms * 4;
    int64_t *pos = sc.get<int64_t>(g.n);
    int64_t *d_ni = sc.get<int64_t>(1);
    exclusive_scan(IsoFlag{g.xadj}, g.n, pos, d_ni, sc);
    int64_t ni = 0;
    CK(cudaMemcpyAsync(&ni, d_ni, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ni == 0) return;
    int32_t *iso = sc.get<int32_t>(ni);
    uint64_t *key = sc.get<uint64_t>(ni);
    unsigned long long *d_cmax = sc.zeros<unsigned long long>(1);
    k_iso_compact<<<grid, 256, 0, s>>>(g, pos, cp, iso, key, d_cmax);
    LAUNCHED();
    if (cp) radix_sort_pairs(key, iso, ni, 32, sc);  // stable: id order within a block
    unsigned long long cmax = 0;
    CK(cudaMemcpyAsync(&cmax, d_cmax, sizeof(cmax), cudaMemcpyDeviceToHost, s));
    int64_t *P = sc.get<int64_t>(ni);
    exclusive_scan(IsoWeight{iso, g.vwgt}, ni, P, nullptr, sc);
    int64_t *sidx = sc.get<int64_t>(ni);
    int64_t *d_ns = sc.get<int64_t>(1);
    exclusive_scan(SegStart{key}, ni, sidx, d_ns, sc);
    CK(cudaStreamSynchronize(s));
    int64_t ns = 0;
    CK(cudaMemcpyAsync(&ns, d_ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int64_t *segP = sc.get<int64_t>(ns);
    k_iso_segbase<<<grid, 256, 0, s>>>(ni, key, P, sidx, segP);
    LAUNCHED();
    GroupStart gs{key, P, sidx, segP, U - (int64_t)cmax + 1};
    int64_t *gidx = sc.get<int64_t>(ni);
    int64_t *d_ng = sc.get<int64_t>(1);
    exclusive_scan(gs, ni, gidx, d_ng, sc);
    int64_t ng = 0;
    CK(cudaMemcpyAsync(&ng, d_ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int32_t *rep = sc.get<int32_t>(ng);
    k_iso_label<<<grid, 256, 0, s>>>(ni, iso, gs, gidx, rep, lab, 0);
    LAUNCHED();
    k_iso_label<<<grid, 256, 0, s>>>(ni, iso, gs, gidx, rep, lab, 1);
    LAUNCHED();
}

// ---------------------------------------------------------------- host driver

static size_t hash_smem() { return sizeof(HashSm); }
static size_t dense_smem() { return sizeof(DenseSm); }

int lp_run(const LPConfig &cfg, Scratch &sc, std::vector<int64_t> *moves_out, int64_t *W_out) {
    cudaStream_t s = sc.stream();
    const DGraph &g = cfg.g;
    const int S = cfg.S;
    const int sms = dev_info().sms;
    if (moves_out) moves_out->clear();
    if (g.n == 0 || cfg.rounds == 0) {
        if (W_out && g.n == 0) CK(cudaMemsetAsync(W_out, 0, cfg.nW * sizeof(int64_t), s));
        return 0;
    }
    const bool dense = cfg.refine && cfg.nW <= kDenseMaxK;

    int64_t *W = W_out ? W_out : sc.get<int64_t>(cfg.nW);
    if (cfg.refine) {
        CK(cudaMemsetAsync(W, 0, cfg.nW * sizeof(int64_t), s));
        size_t shm = cfg.nW <= 1024 ? cfg.nW * sizeof(unsigned long long) : 0;
        k_block_weights<<<sms * 4, 256, shm, s>>>(g, cfg.lab, W, cfg.nW);
        LAUNCHED();
    } else {
        k_init_cluster<<<sms * 4, 256, 0, s>>>(g, cfg.lab, W);
        LAUNCHED();
    }

    LPArgs a{};
    a.g = g;
    a.lab = cfg.lab;
    a.W = W;
    a.B = cfg.B;
    a.nW = cfg.nW;
    a.cp = cfg.refine ? nullptr : cfg.cp;
    a.seed = cfg.seed;
    a.tsum = sc.zeros<int64_t>(cfg.nW);
    a.tcnt = sc.zeros<int32_t>(cfg.nW);
    a.tbase = sc.get<int64_t>(cfg.nW);
    a.ssum = cfg.refine ? sc.zeros<int64_t>(cfg.nW) : nullptr;
    a.props = sc.get<Prop>(g.n);
    a.segs = sc.get<Seg>(g.n);
    a.segbuf = sc.get<SegEntry>(g.n);
    int32_t *wl = sc.get<int32_t>((size_t)2 * S * g.n);
    int32_t *wl_cnt = sc.get<int32_t>(2 * S);
    Ctr *ctr = sc.get<Ctr>(S);
    int64_t *d_moves = sc.zeros<int64_t>(cfg.rounds);
    a.prof = prof().on ? prof().d_counts : nullptr;

    // hub tables (hash variant only)
    const int hub_ctas = std::max(1, std::min(sms, 152));
    if (!dense && cfg.max_deg > kChunkEntries) {
        int bits = bit_width_u64((uint64_t)(2 * cfg.max_deg - 1));
        a.gbits = bits;
        a.gcap = (int64_t)1 << bits;
        a.gkeys = sc.get<unsigned long long>((size_t)hub_ctas * a.gcap);
        a.gvals = sc.zeros<int32_t>((size_t)hub_ctas * a.gcap);
        a.gdl = sc.get<int32_t>((size_t)hub_ctas * (a.gcap / 2));
        CK(cudaMemsetAsync(a.gkeys, 0xff, (size_t)hub_ctas * a.gcap * sizeof(uint64_t), s));
    }

    {
        CK(cudaFuncSetAttribute(k_propose_hash<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_smem()));
        CK(cudaFuncSetAttribute(k_propose_hash<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_smem()));
        CK(cudaFuncSetAttribute(k_propose_hub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_smem()));
        CK(cudaFuncSetAttribute(k_propose_hub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hash_smem()));
        CK(cudaFuncSetAttribute(k_propose_dense<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem()));
        CK(cudaFuncSetAttribute(k_propose_dense<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem()));
    }
    int occ_hash = 0, occ_dense = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_hash, k_propose_hash<false>, kThreads, hash_smem()));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_dense, k_propose_dense<false>, kThreads, dense_smem()));
    const int grid_main = sms * std::max(1, dense ? occ_dense : occ_hash);
    const int grid_small = sms * 4;

    cudaStream_t side;
    CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    cudaEvent_t ev_fork, ev_join;
    CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));

    int done = 0;
    int64_t hmoves = 0;
    try {
        for (int r = 0; r < cfg.rounds; r++) {
            a.round = r;
            a.moves = d_moves + r;
            CK(cudaMemsetAsync(wl_cnt, 0, 2 * S * sizeof(int32_t), s));
            CK(cudaMemsetAsync(ctr, 0, S * sizeof(Ctr), s));
            k_build_wl<<<sms * 4, kThreads, 0, s>>>(g, cfg.seed, r, S, wl, wl_cnt);
            LAUNCHED();
            for (int j = 0; j < S; j++) {
                a.ctr = ctr + j;
                // hub nodes on the side stream, concurrently with the normal nodes
                CK(cudaEventRecord(ev_fork, s));
                CK(cudaStreamWaitEvent(side, ev_fork, 0));
                LPArgs ah = a;
                ah.wl = wl + (int64_t)(2 * j + 1) * g.n;
                ah.wl_cnt = wl_cnt + 2 * j + 1;
                ah.prof = nullptr;
                if (dense) k_propose_dense<true><<<hub_ctas, kThreads, dense_smem(), side>>>(ah, (int)cfg.nW);
                else if (cfg.refine) k_propose_hub<true><<<hub_ctas, kThreads, hash_smem(), side>>>(ah);
                else k_propose_hub<false><<<hub_ctas, kThreads, hash_smem(), side>>>(ah);
                LAUNCHED();
                CK(cudaEventRecord(ev_join, side));

                a.wl = wl + (int64_t)(2 * j) * g.n;
                a.wl_cnt = wl_cnt + 2 * j;
                cudaEvent_t pb, pe;
                prof_begin(s, &pb, &pe);
                if (dense) k_propose_dense<false><<<grid_main, kThreads, dense_smem(), s>>>(a, (int)cfg.nW);
                else if (cfg.refine) k_propose_hash<true><<<grid_main, kThreads, hash_smem(), s>>>(a);
                else k_propose_hash<false><<<grid_main, kThreads, hash_smem(), s>>>(a);
                LAUNCHED();
                prof_end(s, pb, pe);
                CK(cudaStreamWaitEvent(s, ev_join, 0));

                if (cfg.refine) {
                    k_src<<<(unsigned)(cfg.nW + grid_small), kThreads, 0, s>>>(a);
                    LAUNCHED();
                }
                k_classify<<<grid_small, kThreads, 0, s>>>(a);
                LAUNCHED();
                k_scatter<<<grid_small, kThreads, 0, s>>>(a);
                LAUNCHED();
                k_arbitrate<<<grid_small, kThreads, 0, s>>>(a);
                LAUNCHED();
                k_reset_targets<<<grid_small, kThreads, 0, s>>>(a);
                LAUNCHED();
            }
            CK(cudaMemcpyAsync(&hmoves, d_moves + r, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            done = r + 1;
            if (moves_out) moves_out->push_back(hmoves);
            if (hmoves == 0) break;
        }
        Ctr hc[64];
        CK(cudaMemcpyAsync(hc, ctr, S * sizeof(Ctr), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int j = 0; j < S; j++)
            if (hc[j].err) fail(SCLAP_ECUDA, "hash table overflow");
    } catch (...) {
        cudaStreamSynchronize(side);
        cudaEventDestroy(ev_fork);
        cudaEventDestroy(ev_join);
        cudaStreamDestroy(side);
        throw;
    }
    CK(cudaStreamSynchronize(side));
    CK(cudaEventDestroy(ev_fork));
    CK(cudaEventDestroy(ev_join));
    CK(cudaStreamDestroy(side));
    return done;
}

}  // namespace sclap
