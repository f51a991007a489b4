// lp.cu -- the SCLaP sweep: per-round sub-round worklists, degree-binned
// neighbour-label aggregation (propose), exact capacity arbitration and the
// simultaneous apply.  Clustering and refinement share the machinery; the
// refinement form adds the overloaded-block rule (Sec. III.A).
//
// Per round r:
//   k_build_wl    colour = (h(v,r) >> 32) mod S (or the degree-ordered
//                 colours).  Nodes with 1..med_max neighbours go to bucket
//                 5*colour + class (degree <= 4, 8, 16, small_max, med_max);
//                 rows up to the pipelined bound (mid_max) to per-colour
//                 lists of four length classes; longer rows as kChunk-entry
//                 pieces (a single piece up to kChunk), kChunk+1..kHugeDeg in
//                 the hash modes to the cluster list.  The learned gate
//                 (learned.cu) can leave nodes out of a round.
// Per sub-round j, the propose step runs on three streams:
//   k_propose_small  small rows: one thread per node for rows of <= 4, 8
//                 and 16 entries (labels merged in registers); rows up to
//                 small_max on lane groups (__match_any_sync on the label,
//                 __reduce_add_sync gives omega(v, L)); rows up to med_max
//                 one warp each with a warp-private linear-probing table (the
//                 paper's Sec. IV.A choice of linear probing) or a k-array.
//   k_propose_pipe<MODE, PipeShape>  rows of med_max+1..2048 entries in
//                 three length classes: one CTA per row, software-pipelined
//                 over the CTA's rows, with a shared table of packed
//                 (label, omega) words sized to the row.
//   k_propose_stage  rows of 2049..4096 entries when the pipelined bound is
//                 4096: rows staged in shared memory three deep by cp.async.
//   k_propose<MODE, BigRows>  rows above the pipelined bound up to kChunk
//                 entries, one CTA per row with a table of 32-bit labels;
//                 pieces of longer rows merge into a global table (hash) or
//                 k-array (dense) and are finished by k_hub_cand / k_hub_tie
//                 / k_hub_emit or the last piece.
//   k_propose_huge  hash modes, rows up to kHugeDeg: an 8-CTA cluster per
//                 row, its table spread over the CTAs' shared memory.
//   The best eligible label maximises (omega << 32 | ~tie); exact ties on
//   that key go to the smallest label.  Every path finds the largest
//   eligible omega first and hashes ties only for a row that proposes.
// Then arbitration:
//   k_src         refinement only: departures from overloaded blocks.
//   k_arbitrate   one cooperative launch (every CTA resident) with grid
//                 barriers between its phases: classify (uncontested targets,
//                 whose proposed weight fits the capacity, are applied at
//                 once; contested targets get a segment), scatter contested
//                 proposals into their segments and clear the per-target
//                 accumulators, then per contested target a weighted radix
//                 select of the first key in (gain desc, id asc) order whose
//                 inclusive prefix exceeds the capacity (a warp, a CTA, or
//                 the whole grid by segment size); admitted moves are applied.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>

#include "lp.cuh"
#include "prims.cuh"

namespace cg = cooperative_groups;

namespace sclap {

// ---------------------------------------------------------------- tunables

constexpr int kThreads = 256;
constexpr int kSmallDeg = 32;            // small nodes: <= 32 entries (one warp pass)
constexpr int kMedDeg = 256;             // medium nodes: 33..256 entries (one warp each)
constexpr int kChunk = 4096;             // entries per large-row piece (one CTA)
constexpr int kMidDeg = 4096;            // rows up to this size: the pipelined CTA kernels
constexpr int kPipeClasses = 4;          // ... in four length classes (bounds below)
constexpr int kWSlots = 512;             // per-warp table slots for medium rows (>= 2 * kMedDeg)
constexpr int kSlots = 8192;             // hash table slots (>= 2 * kChunk)
constexpr int kSlotBits = 13;
constexpr int kMedItem = 1;              // node slots of the CTA path (one large row at a time)
constexpr int kDenseMaxK = 64;
constexpr int kClasses = 5;              // buckets per colour
constexpr int kHugeCS = 8;               // CTAs per cluster for rows above kChunk (hash modes)
constexpr int kHugeSlots = 4096;         // table slots per CTA of such a cluster (2^12)
constexpr int kHugeDeg = kHugeCS * kHugeSlots / 2;  // longest row one cluster takes (16384)
constexpr int kSegSmem = 6144;           // contested segments staged in shared memory
constexpr int kBigTile = 4096;           // longer segments: tiles spread over the grid
constexpr int kDigit = 11;               // radix-select digit width
constexpr int kBins = 1 << kDigit;
constexpr int kBigUnroll = 4;            // entries in flight per thread: CTA-table rows,
constexpr int kMedUnroll = 4;            //   warp rows,
constexpr int kHugeUnroll = 4;           //   cluster rows
constexpr int kAggW = 1024;              // label weights aggregated in shared memory up to this
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kEmpty32 = 0xffffffffu;

static_assert((1 << kSlotBits) == kSlots, "table size");
static_assert(kSlots >= 2 * kChunk, "load factor <= 1/2");
static_assert(kWSlots >= 2 * kMedDeg, "per-warp table load <= 1/2");

// MODE: 0 clustering (hash), 1 refinement (hash, k > 64), 2 refinement (dense)
constexpr int kCluster = 0, kRefineHash = 1, kRefineDense = 2;

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

// L2-coherent loads of segment state written by other CTAs of the same launch.
__device__ __forceinline__ SegEntry ldcg_entry(const SegEntry *p) {
    const int4 v = __ldcg(reinterpret_cast<const int4 *>(p));
    SegEntry e;
    e.key = ((uint64_t)(uint32_t)v.y << 32) | (uint32_t)v.x;
    e.c = v.z;
    e.own = v.w;
    return e;
}
__device__ __forceinline__ Seg ldcg_seg(const Seg *p) {
    Seg sg;
    sg.T = __ldcg(&p->T);
    sg.cnt = __ldcg(&p->cnt);
    sg.base = __ldcg(&p->base);
    sg.thr = __ldcg(&p->thr);
    return sg;
}
static_assert(sizeof(SegEntry) == 16 && alignof(SegEntry) == 8, "SegEntry as one 16-byte load");

struct Ctr {
    int32_t nprop, nseg;
    int64_t segtotal;
    int32_t large_next, med_next, small_next;
    int32_t err;              // kErrTable or kErrBarrier
    int32_t nbig, bigtiles;   // segments above kSegSmem and their tiles
    int32_t huge_next;        // next row of the cluster path
};

static_assert(sizeof(Ctr) % sizeof(int32_t) == 0, "Ctr cleared as int32 words");

constexpr int32_t kErrTable = 1;
constexpr int32_t kErrBarrier = 2;
constexpr int32_t kErrBig = 4;

// A contested segment too long for one CTA: its select is spread over tiles
// of kBigTile entries handled by all CTAs of the arbitration grid.
struct BigSeg {
    int32_t si;                     // index into segs
    int32_t tiles, t0;              // its tiles: [t0, t0 + tiles)
    int32_t arrived;                // tiles histogrammed in the current pass
    unsigned long long kmin, kmax;  // over entries with c > 0
    unsigned long long pf;          // key bits fixed by the passes so far
    long long acc;                  // weight of the entries below the prefix
    int32_t done;                   // 1: total weight below the threshold
    unsigned idmax;                 // largest node id among entries with c > 0
};

struct GridBar {
    unsigned count, gen;
};

struct LPArgs {
    DGraph g;
    int32_t *lab;
    int64_t *W;
    int64_t B, nW;
    const int64_t *Bv;      // per-label bounds (batched runs) or null: B for every label
    const int32_t *cp;
    uint64_t seed;
    int32_t round, colour, S;
    const int32_t *wl;      // worklists of this round: bucket b at wl + b * n
    const int32_t *wl_cnt;  // bucket lengths (device)
    Prop *props;
    Ctr *ctr;
    int64_t *tsum;
    int32_t *tcnt;
    int64_t *tbase;
    int64_t *ssum;
    Seg *segs;
    SegEntry *segbuf;
    int64_t *moves;         // moves of this round
    // large nodes (degree > kMedDeg), enumerated once per call
    int64_t nL;
    const int32_t *Lnodes;
    const int64_t *Lpre;    // piece prefix [nL + 1]
    const int64_t *Loff;    // global table offset of multi-piece rows (hash) [nL + 1]
    const int64_t *Ldlo;    // global distinct-list offset [nL + 1]
    int32_t *Ldone, *Lndl;
    unsigned long long *gkeys;
    int32_t *gvals;
    int32_t *gdl;
    int32_t *gacc;          // dense: [nL * k]
    int64_t *plist;         // per-colour piece lists: colour c at plist + c * Ptot
    int32_t *pcnt;          // their lengths
    int64_t Ptot;
    const int64_t *Hfin;    // hash: selection items of multi-piece rows [nL + 1]
    unsigned long long *hbest, *htl;  // per multi-piece row: omega M << 32; (tie << 32) | label
    int32_t *hown;
    unsigned long long *prof;  // [2] entries, nodes, or null
    // rows of kChunk < degree <= kHugeDeg in the hash modes: one CTA cluster
    // each; hlist + c * nL lists colour c's rows (indices into Lnodes)
    int32_t huge_on;
    int32_t *hlist;
    int32_t *hcnt;
    // rows of kMedDeg < degree <= kMidDeg for the pipelined kernels: colour
    // c's rows of length class q at pl[q] + c * nL (node ids), their number
    // in pc[q][c]
    int32_t *pl[kPipeClasses];
    int32_t *pc[kPipeClasses];
    int64_t nP;                // capacity of each colour's pipelined list
    // segments above kSegSmem entries (arbitrated by the whole grid)
    BigSeg *big;
    int32_t *tileseg;          // tile -> index into big
    unsigned long long *bhist; // [maxbig * kBins], zero between uses
    GridBar *bar;
    long long bar_cycles;      // bound of every grid-barrier wait (SM clock cycles)
    int32_t maxbig, maxtiles;
    const uint8_t *active;     // learned refinement: rows visited this round (null: all)
    const int32_t *stop;       // device flag: the run has ended (every round kernel returns)
    // batched runs over a disjoint union (null run_of: one graph, one seed):
    // node v belongs to run run_of[v], whose nodes start at run_off[r] and
    // whose blocks are r * run_k .. r * run_k + run_k - 1; its hashes use
    // run_seed[r] with local node and block ids
    const int32_t *run_of;
    const uint64_t *run_seed;
    const int64_t *run_off;
    int32_t run_k;
    const int32_t *col;        // degree-ordered sub-rounds: sub-round per node (null: hash)
    Tuning t;                  // degree-bin and segment thresholds of this call
    // learned refinement (null otherwise): per visited node, the weight to the
    // best eligible other label and to its own label that the visit saw
    int32_t *vb, *vo;
};

// Records what the visit of v saw (learned refinement): best = the best
// eligible candidate key (0: none), ownw = omega(v, own).
__device__ __forceinline__ void record_visit(const LPArgs &a, int32_t v, unsigned long long best,
                                             int32_t ownw) {
    if (!a.vb) return;
    a.vb[v] = best ? (int32_t)(best >> 32) : 0;
    a.vo[v] = ownw;
}

// Every kernel of a round returns at once after the run has ended (the rounds
// of a call are enqueued, or captured in a CUDA graph, ahead of time).
__device__ __forceinline__ bool stopped(const LPArgs &a) { return a.stop && *(volatile const int32_t *)a.stop; }

// Bound of label L (U, L_max, or the run's L_max in batched runs).
__device__ __forceinline__ int64_t bnd(const LPArgs &a, int64_t L) {
    return a.Bv ? __ldg(&a.Bv[L]) : a.B;
}

// h(v, round) of node v: its run's seed and its local id in batched runs.
__device__ __forceinline__ uint64_t nhash(const LPArgs &a, int32_t v) {
    if (!a.run_of) return node_hash(a.seed, a.round, (uint32_t)v);
    const int32_t r = __ldg(&a.run_of[v]);
    return node_hash(__ldg(&a.run_seed[r]), a.round, (uint32_t)(v - __ldg(&a.run_off[r])));
}

// First label of v's run (0 unless batched): ties hash local block ids.
__device__ __forceinline__ int32_t lbase(const LPArgs &a, int32_t v) {
    return a.run_of ? __ldg(&a.run_of[v]) * a.run_k : 0;
}

__device__ __forceinline__ uint64_t seg_key(int32_t gain, int32_t v) {
    return ((uint64_t)(uint32_t)(0x7fffffff - gain) << 32) | (uint32_t)v;
}

__device__ __forceinline__ uint32_t table_hash(uint64_t key, int bits) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

__device__ __forceinline__ uint32_t tie_of(uint64_t h, int32_t L) {
    return (uint32_t)(mix64(h ^ (uint64_t)(uint32_t)L) >> 32);
}

__device__ __forceinline__ uint32_t colour_of(const LPArgs &a, int32_t v) {
    if (a.col) return (uint32_t)__ldg(&a.col[v]);
    return (uint32_t)(nhash(a, v) >> 32) % (uint32_t)a.S;
}

__device__ __forceinline__ unsigned long long cand_key(int32_t w, uint64_t h, int32_t L) {
    return ((unsigned long long)(uint32_t)w << 32) | (uint32_t)~tie_of(h, L);
}

// Weight deltas of applied moves: with few labels (refinement) they collect in
// shared memory and are flushed once per CTA; otherwise moves into and out of
// the same label are merged per warp (labelled partitions) before the global
// atomics.
struct WDelta {
    long long d[kAggW];
};

__device__ __forceinline__ void wd_init(WDelta &wd, int64_t nW) {
    if (nW <= kAggW)
        for (int i = threadIdx.x; i < nW; i += blockDim.x) wd.d[i] = 0;
    __syncthreads();
}

// Applies a move (label write, weight delta).  Called by moving threads only.
// The deltas are summed over the calling threads of the warp that share a
// label first, so one atomic per distinct label and warp reaches the
// CTA-local (nW <= kAggW) or global weight array.
__device__ __forceinline__ void apply_agg(const LPArgs &a, WDelta &wd, int32_t v, int32_t T,
                                          int32_t own, int32_t c) {
    a.lab[v] = T;
    unsigned long long *dst = a.nW <= kAggW ? (unsigned long long *)wd.d
                                             : (unsigned long long *)a.W;
    cg::coalesced_group g = cg::coalesced_threads();
    {
        cg::coalesced_group t = cg::labeled_partition(g, (unsigned)T);
        const long long sum = cg::reduce(t, (long long)c, cg::plus<long long>());
        if (t.thread_rank() == 0) atomicAdd(&dst[T], (unsigned long long)sum);
    }
    {
        cg::coalesced_group o = cg::labeled_partition(g, (unsigned)own);
        const long long sum = cg::reduce(o, (long long)c, cg::plus<long long>());
        if (o.thread_rank() == 0) atomicAdd(&dst[own], (unsigned long long)(-sum));
    }
}

__device__ __forceinline__ void wd_flush(const LPArgs &a, WDelta &wd) {
    __syncthreads();
    if (a.nW <= kAggW)
        for (int i = threadIdx.x; i < a.nW; i += blockDim.x)
            if (wd.d[i]) atomicAdd((unsigned long long *)&a.W[i], (unsigned long long)wd.d[i]);
}

// ---------------------------------------------------------------- worklists

__device__ __forceinline__ int degree_class(int64_t d, int small_max) {
    if (d > small_max) return 4;
    return d <= 4 ? 0 : d <= 8 ? 1 : d <= 16 ? 2 : 3;
}

// Length class of a row of kMedDeg < d <= kMidDeg entries (pipelined kernels).
__device__ __forceinline__ int pipe_class(int64_t d) {
    return d <= 512 ? 0 : d <= 1024 ? 1 : d <= 2048 ? 2 : 3;
}

__global__ void __launch_bounds__(kThreads) k_build_wl(LPArgs a, int32_t *wl, int32_t *cnt) {
    if (stopped(a)) return;
    __shared__ int lcnt[32 * kClasses], lbase[32 * kClasses];
    const DGraph &g = a.g;
    const int S = a.S;
    const int nb = kClasses * S;
    unsigned long long p_entries = 0, p_nodes = 0;  // profiling: rows the round visits
    for (int64_t tile = (int64_t)blockIdx.x * kThreads * 4; tile < g.n;
         tile += (int64_t)gridDim.x * kThreads * 4) {
        for (int i = threadIdx.x; i < nb; i += kThreads) lcnt[i] = 0;
        __syncthreads();
        int bk[4], rk[4];
        int32_t vv[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t v = tile + (int64_t)j * kThreads + threadIdx.x;
            bk[j] = -1;
            vv[j] = (int32_t)v;
            if (v < g.n) {
                const int64_t d = g.xadj[v + 1] - g.xadj[v];
                if (d > 0 && (!a.active || a.active[v])) {
                    p_entries += (unsigned long long)d;
                    p_nodes++;
                    const uint32_t col = colour_of(a, (int32_t)v);
                    if (d <= a.t.med_max) {
                        bk[j] = kClasses * (int)col + degree_class(d, a.t.small_max);
                        rk[j] = atomicAdd(&lcnt[bk[j]], 1);
                    } else if (d <= a.t.mid_max) {
                        // a mid row: the pipelined kernel of its length class
                        const int q = pipe_class(d);
                        const int pos = atomicAdd(&a.pc[q][col], 1);
                        a.pl[q][(int64_t)col * a.nP + pos] = (int32_t)v;
                    } else {
                        // a large row: list its pieces for sub-round `col`
                        int64_t lo = 0, hi = a.nL;  // li: Lnodes[li] == v
                        while (hi - lo > 1) {
                            const int64_t mid = (lo + hi) >> 1;
                            if (a.Lnodes[mid] <= v) lo = mid;
                            else hi = mid;
                        }
                        if (a.huge_on && d > kChunk && d <= kHugeDeg) {
                            const int pos = atomicAdd(&a.hcnt[col], 1);
                            a.hlist[(int64_t)col * a.nL + pos] = (int32_t)lo;
                        } else {
                            const int64_t np = a.Lpre[lo + 1] - a.Lpre[lo];
                            const int base = atomicAdd(&a.pcnt[col], (int)np);
                            int64_t *pl = a.plist + (int64_t)col * a.Ptot + base;
                            for (int64_t p = 0; p < np; p++) pl[p] = (lo << 20) | p;
                        }
                    }
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
    if (a.prof) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            p_entries += __shfl_down_sync(0xffffffffu, p_entries, d);
            p_nodes += __shfl_down_sync(0xffffffffu, p_nodes, d);
        }
        if ((threadIdx.x & 31) == 0 && p_nodes) {
            atomicAdd(&a.prof[0], p_entries);
            atomicAdd(&a.prof[1], p_nodes);
        }
    }
}

// ---------------------------------------------------------------- emission

// Appends the proposal of the calling thread (called by proposing threads
// only; appends are aggregated over the coalesced threads).  AGG groups the
// threads by target for the per-target counters (few targets: refinement).
template <bool AGG>
__device__ __forceinline__ void emit(const LPArgs &a, int32_t v, int32_t T, int32_t own,
                                     int32_t gain, int32_t c, bool ovl, int64_t wT) {
    cg::coalesced_group g = cg::coalesced_threads();
    int pos = 0;
    if (g.thread_rank() == 0) pos = atomicAdd(&a.ctr->nprop, (int)g.size());
    pos = g.shfl(pos, 0) + (int)g.thread_rank();
    int slot;
    if (ovl) {
        atomicAdd((unsigned long long *)&a.ssum[own], (unsigned long long)(int64_t)c);
        slot = -2;
    } else if (AGG) {
        cg::coalesced_group h = cg::coalesced_threads();
        cg::coalesced_group t = cg::labeled_partition(h, (unsigned)T);
        long long sum = cg::reduce(t, (long long)c, cg::plus<long long>());
        int base = 0;
        if (t.thread_rank() == 0) {
            base = atomicAdd(&a.tcnt[T], (int)t.size());
            atomicAdd((unsigned long long *)&a.tsum[T], (unsigned long long)sum);
        }
        slot = t.shfl(base, 0) + (int)t.thread_rank();
    } else {
        atomicAdd((unsigned long long *)&a.tsum[T], (unsigned long long)(int64_t)c);
        slot = atomicAdd(&a.tcnt[T], 1);
    }
    Prop p;
    p.v = v;
    p.T = T;
    p.own = own;
    p.gain = gain;
    p.c = c;
    p.slot = slot;
    p.wT = wT;
    a.props[pos] = p;
}

// ---------------------------------------------------------------- shared memory

struct NodeSm {
    int32_t v[kMedItem], own[kMedItem], c[kMedItem], cpv[kMedItem], ownw[kMedItem],
        bestL[kMedItem];
    int32_t epre[kMedItem + 1];
    int64_t rs[kMedItem];
    uint64_t h[kMedItem];
    int32_t lb[kMedItem];
    unsigned long long best[kMedItem];
    uint8_t ovl[kMedItem];
};

// Shape of a CTA-row kernel: threads, table slots (2^SBITS) and the longest
// piece it takes.  BigRows: rows above the pipelined bound (the tuning's
// mid_max) up to kChunk entries and kChunk-entry pieces of longer rows.
template <int NT, int SBITS, int CHUNK>
struct RowShape {
    static constexpr int kNT = NT, kSBits = SBITS, kSl = 1 << SBITS, kCh = CHUNK;
    static_assert((1 << SBITS) >= 2 * CHUNK, "load factor <= 1/2");
};
using BigRows = RowShape<kThreads, kSlotBits, kChunk>;

template <typename RS>
struct HashTab {
    uint32_t keys[RS::kSl];  // labels; kEmpty32 = empty
    int32_t vals[RS::kSl];
    uint16_t dl[RS::kCh];
};

struct DenseTab {
    int32_t acc[kDenseMaxK];
};

template <int MODE, typename RS>
struct PropSm {
    typename std::conditional<MODE == kRefineDense, DenseTab, HashTab<RS>>::type t;
    NodeSm nd;
    int64_t W[kDenseMaxK];
    unsigned long long red[RS::kNT / 32];
    int64_t li;
    int ndl, item, flag;
};

// Inserts (label L, w) into a linear-probing table of 32-bit labels.  Returns
// the slot when this call created it (the caller appends it to the distinct
// list, one reservation per warp), -1 when the label was there, -2 only if
// the table is full (never at load <= 1/2).
__device__ __forceinline__ int table_insert(uint32_t *keys, int32_t *vals, uint32_t mask, int bits,
                                            uint32_t L, int32_t w) {
    uint32_t slot = (L * 0x9E3779B1u) >> (32 - bits);
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const uint32_t prev = atomicCAS(&keys[slot], kEmpty32, L);
        if (prev == kEmpty32 || prev == L) {
            atomicAdd(&vals[slot], w);
            return prev == kEmpty32 ? (int)slot : -1;
        }
        slot = (slot + 1) & mask;
    }
    return -2;
}

// Loads that bypass L1 (tables merged by other CTAs through L2 atomics).
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld(const T *p) {
    if constexpr (COHERENT) return __ldcg(p);
    else return *p;
}

// Best eligible label of the CTA's row (node slot 0) over the distinct labels,
// in two steps: the largest eligible omega and the own label's omega first
// (per-thread maxima, warp reductions, red holds one value per warp), then,
// only when the row proposes (that omega beats the own one, or the block is
// overloaded), the smallest (tie, label) over the labels reaching it.  The
// result is the label of the largest (omega, ~tie) key, ties on the key to
// the smallest label; nd.best gets omega << 32 alone when the row does not
// propose.
template <int NT>
__device__ __forceinline__ void select_best(const LPArgs &a, const uint32_t *keys,
                                            const int32_t *vals, const uint16_t *dl, int ndl,
                                            NodeSm &nd, unsigned long long *red) {
    uint32_t mw = 0;
    for (int i = threadIdx.x; i < ndl; i += NT) {
        const int slot = dl[i];
        const int32_t L = (int32_t)keys[slot];
        const uint32_t w = (uint32_t)vals[slot];
        if (L == nd.own[0]) nd.ownw[0] = (int32_t)w;
        else if (w > mw && a.W[L] + nd.c[0] <= bnd(a, L)) mw = w;
    }
    mw = __reduce_max_sync(0xffffffffu, mw);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mw;
    __syncthreads();
    uint32_t M = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) M = max(M, (uint32_t)red[w]);
    const bool prop = M > 0 && ((int32_t)M > nd.ownw[0] || nd.ovl[0]);
    __syncthreads();  // red is reused below
    if (!prop) {
        if (threadIdx.x == 0) nd.best[0] = (unsigned long long)M << 32;
        __syncthreads();
        return;
    }
    unsigned long long tl = ~0ull;  // (tie << 32) | label, smallest wins
    for (int i = threadIdx.x; i < ndl; i += NT) {
        const int slot = dl[i];
        const int32_t L = (int32_t)keys[slot];
        if ((uint32_t)vals[slot] != M || L == nd.own[0]) continue;
        if (a.W[L] + nd.c[0] > bnd(a, L)) continue;
        const unsigned long long x =
            ((unsigned long long)tie_of(nd.h[0], L - nd.lb[0]) << 32) | (uint32_t)L;
        tl = x < tl ? x : tl;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, tl, d);
        tl = o < tl ? o : tl;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tl;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NT / 32; w++) tl = red[w] < tl ? red[w] : tl;
        nd.best[0] = ((unsigned long long)M << 32) | (uint32_t)~(uint32_t)(tl >> 32);
        nd.bestL[0] = (int32_t)(uint32_t)tl;
    }
    __syncthreads();
}

// Dense selection on one warp over k <= 64 block sums (lane b holds w0 for
// block b and w1 for block b + 32): the largest eligible omega M first;
// only for a row that proposes (M beats the own omega, or the block is
// overloaded) the tie hashes of the blocks at M, the smallest (tie, block)
// winning.  *best = M << 32 | ~tie, or M << 32 alone for a row that does not
// propose; *bl the block (0x7fffffff if none).
__device__ __forceinline__ void dense_pick(const LPArgs &a, const int64_t *Wsm, int32_t w0,
                                           int32_t w1, int32_t own, int32_t c, uint64_t h,
                                           int32_t lb, int32_t ownw, bool ovl,
                                           unsigned long long *best, int32_t *bl) {
    const int lane = threadIdx.x & 31;
    const bool e0 = w0 > 0 && lane != own && Wsm[lane] + c <= bnd(a, lane);
    const bool e1 = w1 > 0 && lane + 32 != own && Wsm[lane + 32] + c <= bnd(a, lane + 32);
    const uint32_t M =
        __reduce_max_sync(0xffffffffu, max(e0 ? (uint32_t)w0 : 0u, e1 ? (uint32_t)w1 : 0u));
    *best = (unsigned long long)M << 32;
    *bl = 0x7fffffff;
    if (M > 0 && ((int32_t)M > ownw || ovl)) {  // the same in every lane
        const unsigned long long x0 =
            e0 && (uint32_t)w0 == M ? ((unsigned long long)tie_of(h, lane - lb) << 32) | lane : ~0ull;
        const unsigned long long x1 =
            e1 && (uint32_t)w1 == M
                ? ((unsigned long long)tie_of(h, lane + 32 - lb) << 32) | (lane + 32)
                : ~0ull;
        const unsigned long long x = x0 < x1 ? x0 : x1;
        const uint32_t tmin = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32));
        const uint32_t b = __reduce_min_sync(0xffffffffu, (uint32_t)(x >> 32) == tmin ? (uint32_t)x
                                                                                     : 0xffffffffu);
        *best |= (uint32_t)~tmin;
        *bl = (int32_t)b;
    }
}

// Dense variant for node slot s with blocks 0..k-1 in acc[0..k): one warp;
// clears the k-array; result in nd.best / nd.bestL / nd.ownw.
__device__ __forceinline__ void select_dense_warp(const LPArgs &a, const int64_t *Wsm,
                                                  int32_t *acc, int k, NodeSm &nd, int s) {
    const int lane = threadIdx.x & 31;
    const int32_t own = nd.own[s];
    int32_t w0 = lane < k ? acc[lane] : 0;
    int32_t w1 = lane + 32 < k ? acc[lane + 32] : 0;
    __syncwarp();
    if (lane < k) acc[lane] = 0;
    if (lane + 32 < k) acc[lane + 32] = 0;
    const int32_t ownw = __shfl_sync(0xffffffffu, (own < 32) ? w0 : w1, own & 31);
    unsigned long long m;
    int32_t L;
    dense_pick(a, Wsm, w0, w1, own, nd.c[s], nd.h[s], nd.lb[s], ownw, nd.ovl[s] != 0, &m, &L);
    if (lane == 0) {
        nd.best[s] = m;
        nd.bestL[s] = L;
        nd.ownw[s] = ownw;
    }
}

// Proposal decision of node slot s after selection (one thread per node).
template <int MODE>
__device__ __forceinline__ void decide_and_emit(const LPArgs &a, const int64_t *Wsm, NodeSm &nd,
                                                int s) {
    const unsigned long long b = nd.best[s];
    record_visit(a, nd.v[s], b, nd.ownw[s]);
    if (b == 0) return;
    const int32_t gain = (int32_t)(b >> 32) - nd.ownw[s];
    const bool ovl = MODE != kCluster && nd.ovl[s];
    if (!(gain > 0 || ovl)) return;
    const int32_t L = nd.bestL[s];
    const int64_t wT = MODE == kRefineDense ? Wsm[L] : a.W[L];
    emit<MODE == kRefineDense>(a, nd.v[s], L, nd.own[s], gain, nd.c[s], ovl, wT);
}

// Loads node v into slot t and resets its selection state; returns its degree.
template <int MODE>
__device__ __forceinline__ int32_t load_node(const LPArgs &a, const int64_t *Wsm, NodeSm &nd,
                                             int t, int32_t v) {
    nd.v[t] = v;
    const int64_t b = a.g.xadj[v];
    nd.rs[t] = b;
    const int32_t deg = (int32_t)(a.g.xadj[v + 1] - b);
    const int32_t own = a.lab[v];
    nd.own[t] = own;
    nd.c[t] = a.g.vwgt[v];
    nd.cpv[t] = a.cp ? a.cp[v] : 0;
    nd.h[t] = nhash(a, v);
    nd.lb[t] = lbase(a, v);
    nd.ovl[t] = MODE == kCluster ? 0 : ((MODE == kRefineDense ? Wsm[own] : a.W[own]) > bnd(a, own));
    nd.ownw[t] = 0;
    nd.best[t] = 0;
    nd.bestL[t] = 0x7fffffff;
    return deg;
}

// ---------------------------------------------------------------- fused propose kernel

template <int MODE, typename RS>
__device__ void process_large(const LPArgs &a, PropSm<MODE, RS> &sm, int k, const int64_t *plist,
                              int npieces, int32_t *next) {
    constexpr bool DENSE = MODE == kRefineDense;
    constexpr int NT = RS::kNT;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int p = atomicAdd(next, 1);
            sm.item = p;
            if (p < npieces) sm.li = plist[p];
        }
        __syncthreads();
        const int p = sm.item;
        if (p >= npieces) break;
        const int64_t li = sm.li >> 20;
        const int64_t pi = sm.li & ((1 << 20) - 1);
        const int32_t v = a.Lnodes[li];
        const int64_t pieces = a.Lpre[li + 1] - a.Lpre[li];
        if (threadIdx.x == 0) {
            load_node<MODE>(a, sm.W, sm.nd, 0, v);
            sm.ndl = 0;
        }
        __syncthreads();
        const int64_t deg = a.g.xadj[v + 1] - a.g.xadj[v];
        const int64_t e0 = pi * kChunk;  // pieces are kChunk entries (RS::kCh >= any row given here)
        const int64_t e1 = min64(deg, e0 + kChunk);
        const int64_t rs = sm.nd.rs[0];
        const int32_t cpv = sm.nd.cpv[0];
        // every thread runs the same number of steps (warp-wide appends)
        for (int64_t ebase = e0; ebase < e1; ebase += kBigUnroll * NT) {
            const int64_t eb = ebase + threadIdx.x;
            int32_t u[kBigUnroll], w[kBigUnroll], L[kBigUnroll];
#pragma unroll
            for (int j = 0; j < kBigUnroll; j++) {
                const int64_t e = eb + j * NT;
                u[j] = e < e1 ? __ldg(&a.g.adjncy[rs + e]) : -1;
                w[j] = e < e1 ? __ldg(&a.g.adjwgt[rs + e]) : 0;
            }
#pragma unroll
            for (int j = 0; j < kBigUnroll; j++) {
                if (u[j] >= 0 && MODE == kCluster && a.cp && __ldg(&a.cp[u[j]]) != cpv) u[j] = -1;
                L[j] = u[j] >= 0 ? __ldg(&a.lab[u[j]]) : 0;
            }
#pragma unroll
            for (int j = 0; j < kBigUnroll; j++) {
                if constexpr (DENSE) {
                    if (u[j] >= 0) atomicAdd(&sm.t.acc[L[j]], w[j]);
                } else {
                    const int cs = u[j] >= 0 ? table_insert(sm.t.keys, sm.t.vals, RS::kSl - 1,
                                                            RS::kSBits, (uint32_t)L[j], w[j])
                                             : -1;
                    if (cs == -2) a.ctr->err = kErrTable;
                    warp_append(sm.t.dl, &sm.ndl, cs);
                }
            }
        }
        __syncthreads();
        if (pieces == 1) {
            // the whole row is in shared memory: select and emit here
            if constexpr (DENSE) {
                if (threadIdx.x < 32) select_dense_warp(a, sm.W, sm.t.acc, k, sm.nd, 0);
            } else {
                const int ndl = sm.ndl;
                select_best<NT>(a, sm.t.keys, sm.t.vals, sm.t.dl, ndl, sm.nd, sm.red);
                for (int i = threadIdx.x; i < ndl; i += NT) {
                    const int slot = sm.t.dl[i];
                    sm.t.keys[slot] = kEmpty32;
                    sm.t.vals[slot] = 0;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) decide_and_emit<MODE>(a, sm.W, sm.nd, 0);
            continue;
        }
        // merge the piece into the row's global state
        if constexpr (DENSE) {
            int32_t *gacc = a.gacc + li * k;
            for (int b = threadIdx.x; b < k; b += NT) {
                const int32_t w = sm.t.acc[b];
                if (w) {
                    atomicAdd(&gacc[b], w);
                    sm.t.acc[b] = 0;
                }
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) sm.flag = atomicAdd(&a.Ldone[li], 1) == (int)pieces - 1;
            __syncthreads();
            if (!sm.flag) continue;
            // the last piece of this row: select over the k merged sums
            __threadfence();
            if (threadIdx.x < 32) {
                for (int b = threadIdx.x; b < k; b += 32) sm.t.acc[b] = atomicExch(&gacc[b], 0);
                __syncwarp();
                select_dense_warp(a, sm.W, sm.t.acc, k, sm.nd, 0);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                decide_and_emit<MODE>(a, sm.W, sm.nd, 0);
                a.Ldone[li] = 0;
            }
        } else {
            // hash: insert into the row's global table; the best label is
            // selected afterwards by k_hub_cand / k_hub_tie / k_hub_emit
            const int ndl = sm.ndl;
            const int64_t off = a.Loff[li];
            const uint32_t cap = (uint32_t)(a.Loff[li + 1] - off);
            const int bits = 31 - __clz((int)cap);
            int32_t *gdl = a.gdl + a.Ldlo[li];
            unsigned long long *gk = a.gkeys + off;
            int32_t *gv = a.gvals + off;
            const int lane = threadIdx.x & 31;
            const int ndl_r = (ndl + 31) & ~31;
            for (int i = threadIdx.x; i < ndl_r; i += NT) {
                int32_t gslot = -1;
                if (i < ndl) {
                    const int slot = sm.t.dl[i];
                    const uint64_t key = sm.t.keys[slot];  // the global table keeps 64-bit keys
                    const int32_t w = sm.t.vals[slot];
                    sm.t.keys[slot] = kEmpty32;
                    sm.t.vals[slot] = 0;
                    uint32_t q = table_hash(key, bits);
                    bool placed = false;
                    for (uint32_t probe = 0; probe < cap; probe++) {
                        const unsigned long long prev = atomicCAS(&gk[q], kEmpty, key);
                        if (prev == kEmpty || prev == key) {
                            atomicAdd(&gv[q], w);
                            if (prev == kEmpty) gslot = (int32_t)q;
                            placed = true;
                            break;
                        }
                        q = (q + 1) & (cap - 1);
                    }
                    if (!placed) a.ctr->err = kErrTable;
                }
                // one append per warp for the slots it inserted first
                const unsigned m = __ballot_sync(0xffffffffu, gslot >= 0);
                if (m) {
                    int base = 0;
                    if (lane == __ffs(m) - 1) base = atomicAdd(&a.Lndl[li], __popc(m));
                    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
                    if (gslot >= 0) gdl[base + __popc(m & ((1u << lane) - 1))] = gslot;
                }
            }
        }
    }
}

// Small nodes: G lanes per node, one pass (deg <= G).  Loading and computing
// are split so a warp keeps kSmallIlp items' load chains in flight.
constexpr int kSmallIlp = 4;

// One item's loads: node, own label, weight, one entry's label and omega, and
// (hash modes) the gathered weight of that label, kept in 32 bits (every
// label weight is <= c(V) <= INT32_MAX); dense refinement reads the k block
// weights from shared memory when it rates.
struct SmallLoad {
    int32_t v, own, c, L, w, WL, Wown;
    bool has, valid;
};

template <int MODE, int G>
__device__ __forceinline__ SmallLoad small_load(const LPArgs &a, const int32_t *wl, int64_t cnt,
                                                int64_t item) {
    constexpr int NPW = 32 / G;  // nodes per warp item
    const int lane = threadIdx.x & 31;
    const int q = lane / G, r = lane % G;
    const int64_t idx = item * NPW + q;
    SmallLoad x;
    x.has = item >= 0 && idx < cnt;
    x.valid = false;
    x.v = x.own = x.c = x.L = x.w = x.WL = x.Wown = 0;
    if (x.has) {
        x.v = wl[idx];
        const int64_t b = a.g.xadj[x.v];
        const int32_t deg = (int32_t)(a.g.xadj[x.v + 1] - b);
        x.own = a.lab[x.v];
        x.c = a.g.vwgt[x.v];
        if (r < deg) {
            const int32_t u = __ldg(&a.g.adjncy[b + r]);
            x.w = __ldg(&a.g.adjwgt[b + r]);
            if (!(MODE == kCluster && a.cp && __ldg(&a.cp[u]) != a.cp[x.v])) {
                x.L = __ldg(&a.lab[u]);
                x.valid = true;
                if (MODE != kRefineDense) x.WL = (int32_t)a.W[x.L];
            }
        }
        if (MODE == kRefineHash) x.Wown = (int32_t)a.W[x.own];
    }
    return x;
}

template <int MODE, int G>
__device__ __forceinline__ void small_compute(const LPArgs &a, const int64_t *Wsm, const SmallLoad &x) {
    const int lane = threadIdx.x & 31;
    const int q = lane / G, r = lane % G;
    const uint64_t h = x.has ? nhash(a, x.v) : 0;
    const int32_t lb = x.has ? lbase(a, x.v) : 0;
    const unsigned long long mkey =
        x.valid ? (((unsigned long long)q << 32) | (uint32_t)x.L) : (0xffffffff00000000ull | lane);
    const unsigned peers = __match_any_sync(0xffffffffu, mkey);
    const unsigned wsum = __reduce_add_sync(peers, x.valid ? (unsigned)x.w : 0u);
    const bool leader = x.valid && (peers & ((1u << lane) - 1)) == 0;
    unsigned long long ck = 0;
    int32_t ownw = 0;
    if (leader) {
        const int64_t WL = MODE == kRefineDense ? Wsm[x.L] : (int64_t)x.WL;
        if (x.L == x.own) ownw = (int32_t)wsum;
        else if (WL + x.c <= bnd(a, x.L)) ck = cand_key((int32_t)wsum, h, x.L - lb);
    }
    unsigned long long best = ck;  // reduce within the node's G lanes
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, d);
        best = o > best ? o : best;
        ownw += __shfl_xor_sync(0xffffffffu, ownw, d);
    }
    int32_t bl = (best != 0 && ck == best) ? x.L : 0x7fffffff;
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) bl = min(bl, __shfl_xor_sync(0xffffffffu, bl, d));
    if (x.has && r == 0) record_visit(a, x.v, best, ownw);
    if (x.has && r == 0 && best != 0) {
        const int32_t gain = (int32_t)(best >> 32) - ownw;
        const int64_t Wown = MODE == kRefineDense ? Wsm[x.own] : (int64_t)x.Wown;
        const bool ovl = MODE != kCluster && Wown > bnd(a, x.own);
        if (gain > 0 || ovl) {
            const int64_t wT = MODE == kRefineDense ? Wsm[bl] : a.W[bl];
            emit<MODE == kRefineDense>(a, x.v, bl, x.own, gain, x.c, ovl, wT);
        }
    }
}

template <int MODE, int G>
__device__ __forceinline__ void small_bin(const LPArgs &a, const int64_t *Wsm, const int32_t *wl,
                                          int64_t cnt, int64_t gwarp, int64_t nwarps) {
    constexpr int NPW = 32 / G;
    const int64_t items = ceil_div<int64_t>(cnt, NPW);
    for (int64_t it = gwarp; it < items; it += kSmallIlp * nwarps) {
        SmallLoad x[kSmallIlp];
#pragma unroll
        for (int j = 0; j < kSmallIlp; j++) {
            const int64_t t = it + j * nwarps;
            x[j] = small_load<MODE, G>(a, wl, cnt, t < items ? t : -1);
        }
#pragma unroll
        for (int j = 0; j < kSmallIlp; j++)
            if (it + j * nwarps < items) small_compute<MODE, G>(a, Wsm, x[j]);  // warp-uniform
    }
}

// Rows of <= D entries (D = 4, 8, 16): one thread per node.  The node's
// (label, omega) pairs are merged in registers (the first occurrence of a
// label keeps the sum), then rated like every other path: the largest omega
// over the eligible labels first, tie hashes only when the node proposes and
// only at that omega.  A warp thus rates 32 nodes with one instruction stream
// instead of 32 / G nodes in groups of G lanes.
template <int MODE, int D>
__device__ __forceinline__ void tiny_node(const LPArgs &a, const int64_t *Wsm, int32_t v) {
    constexpr bool DENSE = MODE == kRefineDense;
    const int64_t b = a.g.xadj[v];
    const int32_t deg = (int32_t)(a.g.xadj[v + 1] - b);
    const int32_t own = a.lab[v];
    const int32_t c = a.g.vwgt[v];
    const int32_t cpv = (MODE == kCluster && a.cp) ? a.cp[v] : 0;
    int32_t L[D], w[D];
#pragma unroll
    for (int j = 0; j < D; j++) {
        L[j] = -1;
        w[j] = 0;
        if (j < deg) {
            const int32_t u = __ldg(&a.g.adjncy[b + j]);
            w[j] = __ldg(&a.g.adjwgt[b + j]);
            if (!(MODE == kCluster && a.cp && __ldg(&a.cp[u]) != cpv)) L[j] = __ldg(&a.lab[u]);
        }
    }
#pragma unroll
    for (int j = 1; j < D; j++)
#pragma unroll
        for (int i = 0; i < j; i++)
            if (L[j] >= 0 && L[i] == L[j]) {
                w[i] += w[j];
                L[j] = -1;
            }
    int32_t ownw = 0;
    uint32_t M = 0, ew[D];  // ew: omega of an eligible label, else 0
#pragma unroll
    for (int j = 0; j < D; j++) {
        ew[j] = 0;
        if (L[j] < 0) continue;
        if (L[j] == own) {
            ownw = w[j];
        } else {
            const int64_t WL = DENSE ? Wsm[L[j]] : a.W[L[j]];
            if (WL + c <= bnd(a, L[j])) {
                ew[j] = (uint32_t)w[j];
                M = max(M, ew[j]);
            }
        }
    }
    record_visit(a, v, (unsigned long long)M << 32, ownw);
    const bool ovl = MODE != kCluster && (DENSE ? Wsm[own] : a.W[own]) > bnd(a, own);
    if (M > 0 && ((int32_t)M > ownw || ovl)) {
        const uint64_t h = nhash(a, v);
        const int32_t lb = lbase(a, v);
        uint32_t bt = 0xffffffffu;
        int32_t bl = 0x7fffffff;
#pragma unroll
        for (int j = 0; j < D; j++) {
            if (ew[j] != M) continue;
            const uint32_t t = tie_of(h, L[j] - lb);
            if (t < bt || (t == bt && L[j] < bl)) {
                bt = t;
                bl = L[j];
            }
        }
        const int64_t wT = DENSE ? Wsm[bl] : a.W[bl];
        emit<DENSE>(a, v, bl, own, (int32_t)M - ownw, c, ovl, wT);
    }
}

template <int MODE, int D>
__device__ __forceinline__ void tiny_bin(const LPArgs &a, const int64_t *Wsm, const int32_t *wl,
                                         int64_t cnt) {
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += nth)
        tiny_node<MODE, D>(a, Wsm, wl[i]);
}

template <int MODE>
__device__ void process_small(const LPArgs &a, const int64_t *Wsm) {
    const int b0 = kClasses * a.colour;
    const int64_t n = a.g.n;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    tiny_bin<MODE, 4>(a, Wsm, a.wl + b0 * n, a.wl_cnt[b0]);
    tiny_bin<MODE, 8>(a, Wsm, a.wl + (b0 + 1) * n, a.wl_cnt[b0 + 1]);
    tiny_bin<MODE, 16>(a, Wsm, a.wl + (b0 + 2) * n, a.wl_cnt[b0 + 2]);
    small_bin<MODE, 32>(a, Wsm, a.wl + (b0 + 3) * n, a.wl_cnt[b0 + 3], gwarp, nwarps);
}

// CTA rows: the pieces listed in plist (rows above the pipelined bound).
template <int MODE, typename RS>
__global__ void __launch_bounds__(RS::kNT) k_propose(LPArgs a, int k) {
    if (stopped(a)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    PropSm<MODE, RS> &sm = *reinterpret_cast<PropSm<MODE, RS> *>(smraw);
    if (a.nL == 0) return;
    if constexpr (MODE == kRefineDense) {
        for (int i = threadIdx.x; i < kDenseMaxK; i += RS::kNT) sm.t.acc[i] = 0;
        for (int b = threadIdx.x; b < k; b += RS::kNT) sm.W[b] = a.W[b];
    } else {
        for (int i = threadIdx.x; i < RS::kSl; i += RS::kNT) {
            sm.t.keys[i] = kEmpty32;
            sm.t.vals[i] = 0;
        }
    }
    process_large<MODE, RS>(a, sm, k, a.plist + (int64_t)a.colour * a.Ptot, a.pcnt[a.colour],
                            &a.ctr->large_next);
}

// ---------------------------------------------------------------- pipelined CTA rows

// Rows of kMedDeg < degree <= kMidDeg.  One CTA per row; CTA b takes rows b,
// b + grid, b + 2 grid, ... of its colour's list of one length class,
// software-pipelined: while the current row is aggregated, the neighbour
// labels of the next row are being gathered, the entries (adjncy, adjwgt; E
// per thread, in registers) of the row after it and the scalars of the third
// are in flight, and the node id of the fourth.  The table packs the label in
// the high and omega in the low 32 bits of one word (weighted degrees fit 31
// bits, so adding omega never carries into the label) and has
// 2^ceil(log2(2 deg)) slots for a row of deg entries.  The thread whose CAS
// creates a slot owns it: it gathers W(L) at once, and after the barrier
// reads the slot's total, rates the label, and empties the slot, so a row
// costs work in proportion to its length.  Proposals are buffered in shared
// memory and emitted 32 at a time by warp 0 (one reservation of proposal
// slots per batch instead of one contended atomic per row).  Two barriers
// per row, three when the row proposes (tie hashes only then, see below).
template <int NT, int E, int TBITS, int MINB>
struct PipeShape {
    static constexpr int kNT = NT, kE = E, kMaxD = NT * E, kTBits = TBITS, kTS = 1 << TBITS;
    static constexpr int kMinBlocks = MINB;  // CTAs per SM the register budget must allow
    static_assert(kTS >= 2 * kMaxD, "load factor <= 1/2");
    static_assert(NT >= kDenseMaxK, "dense selection: one thread per block");
};
using PipeA = PipeShape<128, 4, 10, 8>;   // rows of kMedDeg + 1 .. 512 entries
using PipeB = PipeShape<128, 8, 11, 5>;   // rows of 513 .. 1024 entries
using PipeC = PipeShape<512, 4, 12, 2>;   // rows of 1025 .. 2048 entries
// rows of 2049 .. kMidDeg entries: the staged kernel below
static_assert(PipeA::kMaxD == 512 && PipeB::kMaxD == 1024 && PipeC::kMaxD == 2048 &&
                  kMidDeg <= kChunk,
              "pipelined row classes (pipe_class)");

template <int MODE, typename PS>
struct PipeSm {
    unsigned long long tab[MODE == kRefineDense ? 1 : PS::kTS];
    int32_t dacc[MODE == kRefineDense ? PS::kNT / 32 : 1][kDenseMaxK];
    int64_t W[kDenseMaxK];
    unsigned long long wk[PS::kNT / 32];  // per warp: best candidate key (dense)
    uint32_t wm[PS::kNT / 32];            //           largest eligible omega
    uint32_t wt[PS::kNT / 32];            //           smallest tie at that omega
    int32_t wl[PS::kNT / 32];             //           its label
    int32_t wo[PS::kNT / 32];             //           omega(v, own) seen
    int32_t bv[32], bT[32], bown[32], bgain[32], bc[32];  // decided proposals,
    uint8_t bovl[32];                                    // emitted 32 at a time
    int nbuf;
};

struct PipeRow {  // scalars of one row (the same in every thread)
    int64_t rs, re;
    int32_t v, own, c, cpv;
};

template <int MODE>
__device__ __forceinline__ PipeRow pipe_row(const LPArgs &a, int32_t v) {
    PipeRow r;
    r.v = v;
    r.rs = r.re = 0;
    r.own = r.c = r.cpv = 0;
    if (v >= 0) {
        r.rs = a.g.xadj[v];
        r.re = a.g.xadj[v + 1];
        r.own = a.lab[v];
        r.c = a.g.vwgt[v];
        if (MODE == kCluster && a.cp) r.cpv = a.cp[v];
    }
    return r;
}

// Entries j*NT + t of row r (t = thread), E per thread.  Whole unrolled steps
// past the row's end are skipped (the test is the same in every thread).
template <int NT, int E>
__device__ __forceinline__ void pipe_entries(const LPArgs &a, const PipeRow &r, int32_t *u,
                                             int32_t *w) {
    const int64_t deg = r.re - r.rs;
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int e = (int)threadIdx.x + j * NT;
        u[j] = 0;
        w[j] = 0;
        if (j * NT < deg && e < deg) {
            u[j] = __ldcs(&a.g.adjncy[r.rs + e]);
            w[j] = __ldcs(&a.g.adjwgt[r.rs + e]);
        }
    }
}

// Warp 0 emits the buffered proposals (one reservation per batch, weights
// per target summed over the batch in dense mode) once 32 have collected, or
// all of them when `all`.
template <int MODE, typename SM>
__device__ __forceinline__ void pipe_flush(const LPArgs &a, SM &sm, bool all) {
    if (threadIdx.x >= 32) return;
    __syncwarp();
    const int nb = sm.nbuf;
    if (nb == 0 || (!all && nb < 32)) return;
    const int lane = threadIdx.x;
    if (lane < nb) {
        const int32_t T = sm.bT[lane];
        const int64_t wT = MODE == kRefineDense ? sm.W[T] : a.W[T];
        emit<MODE == kRefineDense>(a, sm.bv[lane], T, sm.bown[lane], sm.bgain[lane], sm.bc[lane],
                                   sm.bovl[lane] != 0, wT);
    }
    __syncwarp();
    if (lane == 0) sm.nbuf = 0;
    __syncwarp();
}

// (key, label) order of candidates: larger key first, then smaller label.
__device__ __forceinline__ bool cand_better(unsigned long long k1, int32_t l1,
                                            unsigned long long k2, int32_t l2) {
    return k1 > k2 || (k1 == k2 && l1 < l2);
}

// Thread 0 buffers the current row's proposal (target T).
template <typename SM>
__device__ __forceinline__ void pipe_buffer(SM &sm, const PipeRow &r, int32_t T, int32_t gain,
                                            bool ovl) {
    const int i = sm.nbuf++;
    sm.bv[i] = r.v;
    sm.bT[i] = T;
    sm.bown[i] = r.own;
    sm.bgain[i] = gain;
    sm.bc[i] = r.c;
    sm.bovl[i] = ovl ? 1 : 0;
}

template <int MODE, typename PS>
__global__ void __launch_bounds__(PS::kNT, PS::kMinBlocks) k_propose_pipe(LPArgs a, int k, int cls) {
    if (stopped(a)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    PipeSm<MODE, PS> &sm = *reinterpret_cast<PipeSm<MODE, PS> *>(smraw);
    constexpr int NT = PS::kNT, E = PS::kE, NW = NT / 32;
    constexpr bool DENSE = MODE == kRefineDense;
    const int32_t *list = a.pl[cls] + (int64_t)a.colour * a.nP;
    const int cnt = a.pc[cls][a.colour];
    const int G = gridDim.x;
    int idx = blockIdx.x;
    if (idx >= cnt) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (DENSE) {
        for (int i = threadIdx.x; i < NW * kDenseMaxK; i += NT) (&sm.dacc[0][0])[i] = 0;
        for (int b = threadIdx.x; b < k; b += NT) sm.W[b] = a.W[b];
    } else {
        for (int i = threadIdx.x; i < PS::kTS; i += NT) sm.tab[i] = kEmpty;
    }
    if (threadIdx.x == 0) sm.nbuf = 0;
    // prologue: labels of row 0, entries of row 1, scalars of row 2, id of row 3
    PipeRow cur = pipe_row<MODE>(a, list[idx]);
    int32_t u[E], w[E], L[E], cpu[E];
    pipe_entries<NT, E>(a, cur, u, w);
    PipeRow nxt = pipe_row<MODE>(a, idx + G < cnt ? list[idx + G] : -1);
    int32_t v3 = idx + 2 * G < cnt ? list[idx + 2 * G] : -1;
    {
        const int64_t deg = cur.re - cur.rs;
#pragma unroll
        for (int j = 0; j < E; j++) {
            const bool in = (int)threadIdx.x + j * NT < deg;
            L[j] = in ? __ldg(&a.lab[u[j]]) : 0;
            cpu[j] = (MODE == kCluster && a.cp && in) ? __ldg(&a.cp[u[j]]) : cur.cpv;
        }
    }
    int32_t w0[E];
#pragma unroll
    for (int j = 0; j < E; j++) w0[j] = w[j];
    pipe_entries<NT, E>(a, nxt, u, w);
    PipeRow nn = pipe_row<MODE>(a, v3);
    v3 = idx + 3 * G < cnt ? list[idx + 3 * G] : -1;
    __syncthreads();
    for (; idx < cnt; idx += G) {
        // labels of the next row (its entries arrived during the last row)
        const int64_t deg1 = nxt.re - nxt.rs;
        int32_t L1[E], cpu1[E], w1[E];
#pragma unroll
        for (int j = 0; j < E; j++) {
            const bool in = (int)threadIdx.x + j * NT < deg1;
            L1[j] = in ? __ldg(&a.lab[u[j]]) : 0;
            cpu1[j] = (MODE == kCluster && a.cp && in) ? __ldg(&a.cp[u[j]]) : nxt.cpv;
            w1[j] = w[j];
        }
        // entries of the row after it, scalars of the third, id of the fourth
        pipe_entries<NT, E>(a, nn, u, w);
        const PipeRow n3 = pipe_row<MODE>(a, v3);
        v3 = idx + 4 * G < cnt ? list[idx + 4 * G] : -1;
        const int64_t deg = cur.re - cur.rs;
        const uint64_t h = nhash(a, cur.v);
        const int32_t lb = lbase(a, cur.v);
        const int64_t wown = MODE == kRefineHash ? a.W[cur.own] : 0;
        pipe_flush<MODE>(a, sm, false);
        // aggregation of the current row; a slot's creator gathers W(L)
        const uint32_t tbits = deg <= 32 ? 6u : 33u - (uint32_t)__clz((int)(deg - 1));
        const uint32_t tmask = (1u << tbits) - 1;
        int32_t myslot[E];
        int64_t WL[E];
#pragma unroll
        for (int j = 0; j < E; j++) {
            myslot[j] = -1;
            WL[j] = 0;
            const bool in = (int)threadIdx.x + j * NT < deg && cpu[j] == cur.cpv;
            if (!in) continue;
            if constexpr (DENSE) {
                atomicAdd(&sm.dacc[warp][L[j]], w0[j]);
            } else {
                const unsigned long long key = (unsigned long long)(uint32_t)L[j] << 32;
                uint32_t slot = ((uint32_t)L[j] * 0x9E3779B1u) >> (32 - tbits);
                for (uint32_t probe = 0; probe <= tmask; probe++) {
                    const unsigned long long prev =
                        atomicCAS(&sm.tab[slot], kEmpty, key | (uint32_t)w0[j]);
                    if (prev == kEmpty) {
                        myslot[j] = (int32_t)slot;
                        WL[j] = __ldg(&a.W[L[j]]);
                        break;
                    }
                    if ((prev & 0xffffffff00000000ull) == key) {
                        atomicAdd(&sm.tab[slot], (unsigned long long)(uint32_t)w0[j]);
                        break;
                    }
                    slot = (slot + 1) & tmask;
                }
            }
        }
        __syncthreads();
        if constexpr (DENSE) {
            // selection: the first k threads rate the k block sums
            unsigned long long bk = 0;
            int32_t bl = 0x7fffffff, ow = 0;
            if ((int)threadIdx.x < k) {
                const int b = threadIdx.x;
                int32_t tot = 0;
#pragma unroll
                for (int q = 0; q < NW; q++) {
                    tot += sm.dacc[q][b];
                    sm.dacc[q][b] = 0;
                }
                if (b == cur.own) ow = tot;
                else if (tot > 0 && sm.W[b] + cur.c <= bnd(a, b)) {
                    bk = cand_key(tot, h, b - lb);
                    bl = b;
                }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(0xffffffffu, bk, d);
                const int32_t ol = __shfl_xor_sync(0xffffffffu, bl, d);
                if (cand_better(ok, ol, bk, bl)) {
                    bk = ok;
                    bl = ol;
                }
                ow += __shfl_xor_sync(0xffffffffu, ow, d);
            }
            if (lane == 0) {
                sm.wk[warp] = bk;
                sm.wl[warp] = bl;
                sm.wo[warp] = ow;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 1; q < NW; q++) {
                    if (cand_better(sm.wk[q], sm.wl[q], bk, bl)) {
                        bk = sm.wk[q];
                        bl = sm.wl[q];
                    }
                    ow += sm.wo[q];
                }
                record_visit(a, cur.v, bk, ow);
                if (bk != 0) {
                    const int32_t gain = (int32_t)(bk >> 32) - ow;
                    const bool ovl = sm.W[cur.own] > bnd(a, cur.own);
                    if (gain > 0 || ovl) pipe_buffer(sm, cur, bl, gain, ovl);
                }
            }
        } else {
            // selection in two steps.  The slot owners empty their slots and
            // find the largest omega over the eligible labels and the own
            // label's omega, with no tie hashes.  Only when the row proposes
            // (that omega beats the own one, or the block is overloaded) do
            // the labels reaching it hash their ties, and the smallest (tie,
            // label) wins.  This is the label of the largest (omega, ~tie)
            // key, ties on the key to the smallest label.
            uint32_t mw = 0, xw[E];
            int32_t ow = 0;
#pragma unroll
            for (int j = 0; j < E; j++) {
                xw[j] = 0;
                if (myslot[j] < 0) continue;
                const uint32_t wx = (uint32_t)sm.tab[myslot[j]];
                sm.tab[myslot[j]] = kEmpty;
                if (L[j] == cur.own) {
                    ow = (int32_t)wx;
                } else if (WL[j] + cur.c <= bnd(a, L[j])) {
                    xw[j] = wx;
                    mw = max(mw, wx);
                }
            }
            mw = __reduce_max_sync(0xffffffffu, mw);
            ow = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)ow);
            if (lane == 0) {
                sm.wm[warp] = mw;
                sm.wo[warp] = ow;
            }
            __syncthreads();
            uint32_t M = 0;
            int32_t OW = 0;
#pragma unroll
            for (int q = 0; q < NW; q++) {
                M = max(M, sm.wm[q]);
                OW += sm.wo[q];
            }
            const bool ovl = MODE == kRefineHash && wown > bnd(a, cur.own);
            if (threadIdx.x == 0) record_visit(a, cur.v, (unsigned long long)M << 32, OW);
            if (M > 0 && ((int32_t)M > OW || ovl)) {  // the same in every thread
                uint32_t bt = 0xffffffffu, bl = 0x7fffffffu;
#pragma unroll
                for (int j = 0; j < E; j++) {
                    if (xw[j] != M) continue;
                    const uint32_t t = tie_of(h, L[j] - lb);
                    if (t < bt || (t == bt && (uint32_t)L[j] < bl)) {
                        bt = t;
                        bl = (uint32_t)L[j];
                    }
                }
                const uint32_t wt = __reduce_min_sync(0xffffffffu, bt);
                bl = __reduce_min_sync(0xffffffffu, bt == wt ? bl : 0x7fffffffu);
                if (lane == 0) {
                    sm.wt[warp] = wt;
                    sm.wl[warp] = (int32_t)bl;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t tb = sm.wt[0];
                    int32_t lbest = sm.wl[0];
                    for (int q = 1; q < NW; q++) {
                        if (sm.wt[q] < tb || (sm.wt[q] == tb && sm.wl[q] < lbest)) {
                            tb = sm.wt[q];
                            lbest = sm.wl[q];
                        }
                    }
                    pipe_buffer(sm, cur, lbest, (int32_t)M - OW, ovl);
                }
            }
        }
        cur = nxt;
        nxt = nn;
        nn = n3;
#pragma unroll
        for (int j = 0; j < E; j++) {
            L[j] = L1[j];
            cpu[j] = cpu1[j];
            w0[j] = w1[j];
        }
    }
    pipe_flush<MODE>(a, sm, true);
}

// ---------------------------------------------------------------- staged CTA rows

// Rows of 2049..kMidDeg entries (length class 3): one 256-thread CTA per row,
// rows b, b + grid, ... of the colour's class-3 list, staged in shared memory
// three rows deep by asynchronous copies (cp.async): while row i is
// aggregated from shared memory, the neighbour labels of row i + 1 are being
// gathered (a cp.async of lab[u] for each u already staged) and the entries of
// row i + 2 are being copied.  No registers hold the data in flight.  The
// table packs (label, omega) like the pipelined kernels; new slots go to a
// distinct list (one reservation per warp); selection rates the largest
// eligible omega first and hashes ties only for a row that proposes.
constexpr int kStNT = 256;
constexpr int kStMax = kMidDeg;
constexpr int kStSlots = 2 * kStMax;  // load <= 1/2

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct StageRow {
    int32_t u[kStMax], w[kStMax], L[kStMax];
};

template <int MODE>
struct StageSm {
    StageRow r[3];
    unsigned long long tab[MODE == kRefineDense ? 1 : kStSlots];
    uint16_t dl[MODE == kRefineDense ? 1 : kStMax];
    int32_t dacc[MODE == kRefineDense ? kStNT / 32 : 1][kDenseMaxK];
    int64_t W[kDenseMaxK];
    uint32_t wm[kStNT / 32], wt[kStNT / 32];
    int32_t wl[kStNT / 32], wo[kStNT / 32];
    int32_t bv[32], bT[32], bown[32], bgain[32], bc[32];
    uint8_t bovl[32];
    int nbuf, ndl;
};

// Entries of row r into R (thread t copies entries t, t + kStNT, ...).
__device__ __forceinline__ void stage_entries(const LPArgs &a, const PipeRow &r, StageRow &R) {
    const int deg = (int)(r.re - r.rs);
    for (int e = threadIdx.x; e < deg; e += kStNT) {
        cp_async4(&R.u[e], &a.g.adjncy[r.rs + e]);
        cp_async4(&R.w[e], &a.g.adjwgt[r.rs + e]);
    }
}

// Labels of row r's staged neighbours (the same thread staged u[e]).
__device__ __forceinline__ void stage_labels(const LPArgs &a, const PipeRow &r, StageRow &R) {
    const int deg = (int)(r.re - r.rs);
    for (int e = threadIdx.x; e < deg; e += kStNT) cp_async4(&R.L[e], &a.lab[R.u[e]]);
}

template <int MODE>
__global__ void __launch_bounds__(kStNT, 1) k_propose_stage(LPArgs a, int k) {
    if (stopped(a)) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    StageSm<MODE> &sm = *reinterpret_cast<StageSm<MODE> *>(smraw);
    constexpr int NT = kStNT, NW = NT / 32;
    constexpr bool DENSE = MODE == kRefineDense;
    const int32_t *list = a.pl[3] + (int64_t)a.colour * a.nP;
    const int cnt = a.pc[3][a.colour];
    const int G = gridDim.x;
    int idx = blockIdx.x;
    if (idx >= cnt) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (DENSE) {
        for (int i = threadIdx.x; i < NW * kDenseMaxK; i += NT) (&sm.dacc[0][0])[i] = 0;
        for (int b = threadIdx.x; b < k; b += NT) sm.W[b] = a.W[b];
    } else {
        for (int i = threadIdx.x; i < kStSlots; i += NT) sm.tab[i] = kEmpty;
    }
    if (threadIdx.x == 0) {
        sm.nbuf = 0;
        sm.ndl = 0;
    }
    // prologue: entries of rows 0 and 1, then the labels of row 0
    PipeRow cur = pipe_row<MODE>(a, list[idx]);
    PipeRow nxt = pipe_row<MODE>(a, idx + G < cnt ? list[idx + G] : -1);
    stage_entries(a, cur, sm.r[0]);
    cp_async_commit();
    stage_entries(a, nxt, sm.r[1]);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    stage_labels(a, cur, sm.r[0]);
    cp_async_commit();
    int sl = 0;  // slot of the current row
    for (; idx < cnt; idx += G) {
        const int i2 = idx + 2 * G;
        const PipeRow nn = pipe_row<MODE>(a, i2 < cnt ? list[i2] : -1);
        stage_entries(a, nn, sm.r[sl == 0 ? 2 : sl - 1]);  // slot (sl + 2) % 3
        cp_async_commit();
        cp_async_wait<1>();  // the entries of row i + 1 and the labels of row i are in
        __syncthreads();
        stage_labels(a, nxt, sm.r[sl == 2 ? 0 : sl + 1]);
        cp_async_commit();
        pipe_flush<MODE>(a, sm, false);
        const StageRow &R = sm.r[sl];
        const int deg = (int)(cur.re - cur.rs);
        const uint64_t h = nhash(a, cur.v);
        const int32_t lb = lbase(a, cur.v);
        if constexpr (DENSE) {
            for (int e = threadIdx.x; e < deg; e += NT) atomicAdd(&sm.dacc[warp][R.L[e]], R.w[e]);
            __syncthreads();
            // thread b rates block b: largest eligible omega first
            int32_t tot = 0;
            bool el = false;
            if ((int)threadIdx.x < k) {
                const int b = threadIdx.x;
#pragma unroll
                for (int q = 0; q < NW; q++) {
                    tot += sm.dacc[q][b];
                    sm.dacc[q][b] = 0;
                }
                el = b != cur.own && tot > 0 && sm.W[b] + cur.c <= bnd(a, b);
            }
            const uint32_t mw = __reduce_max_sync(0xffffffffu, el ? (uint32_t)tot : 0u);
            const int32_t ow = (int32_t)__reduce_add_sync(
                0xffffffffu, (int)threadIdx.x == cur.own ? (uint32_t)tot : 0u);
            if (lane == 0) {
                sm.wm[warp] = mw;
                sm.wo[warp] = ow;
            }
            __syncthreads();
            uint32_t M = 0;
            int32_t OW = 0;
#pragma unroll
            for (int q = 0; q < NW; q++) {
                M = max(M, sm.wm[q]);
                OW += sm.wo[q];
            }
            const bool ovl = sm.W[cur.own] > bnd(a, cur.own);
            if (threadIdx.x == 0) record_visit(a, cur.v, (unsigned long long)M << 32, OW);
            if (M > 0 && ((int32_t)M > OW || ovl)) {  // the same in every thread
                const uint32_t t = el && (uint32_t)tot == M ? tie_of(h, (int)threadIdx.x - lb)
                                                           : 0xffffffffu;
                const uint32_t wt = __reduce_min_sync(0xffffffffu, t);
                const uint32_t b = __reduce_min_sync(
                    0xffffffffu, t == wt && el && (uint32_t)tot == M ? threadIdx.x : 0x7fffffffu);
                if (lane == 0) {
                    sm.wt[warp] = wt;
                    sm.wl[warp] = (int32_t)b;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t tb = sm.wt[0];
                    int32_t best = sm.wl[0];
                    for (int q = 1; q < NW; q++)
                        if (sm.wt[q] < tb || (sm.wt[q] == tb && sm.wl[q] < best)) {
                            tb = sm.wt[q];
                            best = sm.wl[q];
                        }
                    pipe_buffer(sm, cur, best, (int32_t)M - OW, ovl);
                }
            }
        } else {
            const uint32_t tbits = 33u - (uint32_t)__clz(deg - 1);  // deg > 2048
            const uint32_t tmask = (1u << tbits) - 1;
            for (int e0 = 0; e0 < deg; e0 += NT) {  // the same steps in every thread
                const int e = e0 + threadIdx.x;
                int cs = -1;
                if (e < deg && !(MODE == kCluster && a.cp && __ldg(&a.cp[R.u[e]]) != cur.cpv)) {
                    const uint32_t L = (uint32_t)R.L[e];
                    const unsigned long long key = (unsigned long long)L << 32;
                    uint32_t slot = (L * 0x9E3779B1u) >> (32 - tbits);
                    for (uint32_t probe = 0; probe <= tmask; probe++) {
                        const unsigned long long prev =
                            atomicCAS(&sm.tab[slot], kEmpty, key | (uint32_t)R.w[e]);
                        if (prev == kEmpty) {
                            cs = (int)slot;
                            break;
                        }
                        if ((prev & 0xffffffff00000000ull) == key) {
                            atomicAdd(&sm.tab[slot], (unsigned long long)(uint32_t)R.w[e]);
                            break;
                        }
                        slot = (slot + 1) & tmask;
                    }
                }
                warp_append(sm.dl, &sm.ndl, cs);
            }
            __syncthreads();
            const int ndl = sm.ndl;
            uint32_t mw = 0;
            int32_t ow = 0;
            for (int i = threadIdx.x; i < ndl; i += NT) {
                const unsigned long long x = sm.tab[sm.dl[i]];
                const int32_t L = (int32_t)(x >> 32);
                const uint32_t wx = (uint32_t)x;
                if (L == cur.own) ow = (int32_t)wx;
                else if (wx > mw && a.W[L] + cur.c <= bnd(a, L)) mw = wx;
            }
            mw = __reduce_max_sync(0xffffffffu, mw);
            ow = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)ow);
            if (lane == 0) {
                sm.wm[warp] = mw;
                sm.wo[warp] = ow;
            }
            __syncthreads();
            uint32_t M = 0;
            int32_t OW = 0;
#pragma unroll
            for (int q = 0; q < NW; q++) {
                M = max(M, sm.wm[q]);
                OW += sm.wo[q];
            }
            const bool ovl = MODE == kRefineHash && a.W[cur.own] > bnd(a, cur.own);
            if (threadIdx.x == 0) record_visit(a, cur.v, (unsigned long long)M << 32, OW);
            if (M > 0 && ((int32_t)M > OW || ovl)) {  // the same in every thread
                uint32_t bt = 0xffffffffu, bl = 0x7fffffffu;
                for (int i = threadIdx.x; i < ndl; i += NT) {
                    const unsigned long long x = sm.tab[sm.dl[i]];
                    const int32_t L = (int32_t)(x >> 32);
                    if ((uint32_t)x != M || L == cur.own || a.W[L] + cur.c > bnd(a, L)) continue;
                    const uint32_t t = tie_of(h, L - lb);
                    if (t < bt || (t == bt && (uint32_t)L < bl)) {
                        bt = t;
                        bl = (uint32_t)L;
                    }
                }
                const uint32_t wt = __reduce_min_sync(0xffffffffu, bt);
                bl = __reduce_min_sync(0xffffffffu, bt == wt ? bl : 0x7fffffffu);
                if (lane == 0) {
                    sm.wt[warp] = wt;
                    sm.wl[warp] = (int32_t)bl;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t tb = sm.wt[0];
                    int32_t best = sm.wl[0];
                    for (int q = 1; q < NW; q++)
                        if (sm.wt[q] < tb || (sm.wt[q] == tb && sm.wl[q] < best)) {
                            tb = sm.wt[q];
                            best = sm.wl[q];
                        }
                    pipe_buffer(sm, cur, best, (int32_t)M - OW, ovl);
                }
            }
            for (int i = threadIdx.x; i < ndl; i += NT) sm.tab[sm.dl[i]] = kEmpty;
        }
        __syncthreads();  // slot sl and the table are free again
        if (!DENSE && threadIdx.x == 0) sm.ndl = 0;
        cur = nxt;
        nxt = nn;
        sl = sl == 2 ? 0 : sl + 1;
    }
    cp_async_wait<0>();
    pipe_flush<MODE>(a, sm, true);
}

// Medium rows (up to kMedDeg entries): one warp per row with a warp-private
// shared-memory table, no block-wide barriers.  A slot packs the label in the
// high and omega in the low 32 bits (a row's weighted degree fits 31 bits, so
// adding omega never carries into the label): a new label is one CAS, a
// repeated one one add.
struct WarpTab {
    unsigned long long s[kWSlots];  // kEmpty = empty
    uint16_t dl[kMedDeg];           // slots in insertion order
    int ndl;
};

// Adds (L, w); returns the slot when this call created it, else -1.
__device__ __forceinline__ int wtab_insert(WarpTab &t, uint32_t L, int32_t w) {
    const unsigned long long key = (unsigned long long)L << 32;
    uint32_t slot = (uint32_t)(((uint64_t)L * 0x9E3779B97F4A7C15ull) >> 55) & (kWSlots - 1);
    for (int probe = 0; probe < kWSlots; probe++) {
        const unsigned long long prev = atomicCAS(&t.s[slot], kEmpty, key | (uint32_t)w);
        if (prev == kEmpty) return (int)slot;
        if ((prev & 0xffffffff00000000ull) == key) {
            atomicAdd(&t.s[slot], (unsigned long long)(uint32_t)w);
            return -1;
        }
        slot = (slot + 1) & (kWSlots - 1);
    }
    return -1;
}

template <int MODE>
__device__ __forceinline__ void medium_row(const LPArgs &a, const int64_t *Wsm, WarpTab &t,
                                           int32_t *dacc, int k, int32_t v) {
    constexpr bool DENSE = MODE == kRefineDense;
    const int lane = threadIdx.x & 31;
    const int64_t b = a.g.xadj[v];
    const int32_t deg = (int32_t)(a.g.xadj[v + 1] - b);
    const int32_t own = a.lab[v];
    const int32_t c = a.g.vwgt[v];
    const int32_t cpv = (MODE == kCluster && a.cp) ? a.cp[v] : 0;
    const int64_t Wown = MODE == kCluster ? 0 : (DENSE ? Wsm[own] : a.W[own]);
    const uint64_t h = nhash(a, v);
    const int32_t lb = lbase(a, v);
    for (int32_t e0 = 0; e0 < deg; e0 += 32 * kMedUnroll) {
        int32_t u[kMedUnroll], w[kMedUnroll], L[kMedUnroll];
#pragma unroll
        for (int j = 0; j < kMedUnroll; j++) {
            const int32_t e = e0 + j * 32 + lane;
            u[j] = e < deg ? __ldg(&a.g.adjncy[b + e]) : -1;
            w[j] = e < deg ? __ldg(&a.g.adjwgt[b + e]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kMedUnroll; j++) {
            if (u[j] >= 0 && MODE == kCluster && a.cp && __ldg(&a.cp[u[j]]) != cpv) u[j] = -1;
            L[j] = u[j] >= 0 ? __ldg(&a.lab[u[j]]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kMedUnroll; j++) {
            if constexpr (DENSE) {
                if (u[j] >= 0) atomicAdd(&dacc[L[j]], w[j]);
            } else {
                const int cs = u[j] >= 0 ? wtab_insert(t, (uint32_t)L[j], w[j]) : -1;
                // the warp appends its new slots to the insertion-order list
                const unsigned m = __ballot_sync(0xffffffffu, cs >= 0);
                if (m) {
                    const int base = t.ndl;
                    if (cs >= 0) t.dl[base + __popc(m & ((1u << lane) - 1))] = (uint16_t)cs;
                    __syncwarp();
                    if (lane == 0) t.ndl = base + __popc(m);
                    __syncwarp();
                }
            }
        }
    }
    __syncwarp();
    unsigned long long best = 0;
    int32_t ownw = 0, bl = 0x7fffffff;
    if constexpr (DENSE) {
        const int32_t w0 = lane < k ? dacc[lane] : 0;
        const int32_t w1 = lane + 32 < k ? dacc[lane + 32] : 0;
        __syncwarp();
        if (lane < k) dacc[lane] = 0;
        if (lane + 32 < k) dacc[lane + 32] = 0;
        ownw = __shfl_sync(0xffffffffu, (own < 32) ? w0 : w1, own & 31);
        dense_pick(a, Wsm, w0, w1, own, c, h, lb, ownw, Wown > bnd(a, own), &best, &bl);
    } else {
        // the largest eligible omega and the own omega first; tie hashes
        // only when the row proposes, and only for the labels reaching that
        // omega (the label of the largest (omega, ~tie) key, then the
        // smallest label)
        const int nd = t.ndl;
        constexpr int PER = kMedDeg / 32;  // distinct labels per lane (<= deg)
        uint32_t xw[PER], mw = 0;
        int32_t lab[PER];
#pragma unroll
        for (int j = 0; j < PER; j++) {
            xw[j] = 0;
            lab[j] = 0;
            const int i = lane + 32 * j;
            if (i < nd) {
                const int slot = t.dl[i];
                const unsigned long long x = t.s[slot];
                const int32_t L = (int32_t)(x >> 32);
                const int32_t w = (int32_t)(uint32_t)x;
                t.s[slot] = kEmpty;
                lab[j] = L;
                if (L == own) {
                    ownw = w;
                } else if (a.W[L] + c <= bnd(a, L)) {
                    xw[j] = (uint32_t)w;
                    mw = max(mw, (uint32_t)w);
                }
            }
        }
        mw = __reduce_max_sync(0xffffffffu, mw);
        ownw = (int32_t)__reduce_add_sync(0xffffffffu, (uint32_t)ownw);
        best = (unsigned long long)mw << 32;
        const bool ovl = MODE != kCluster && Wown > bnd(a, own);
        if (mw > 0 && ((int32_t)mw > ownw || ovl)) {
            uint32_t bt = 0xffffffffu, lb2 = 0x7fffffffu;
#pragma unroll
            for (int j = 0; j < PER; j++) {
                if (xw[j] != mw) continue;
                const uint32_t tj = tie_of(h, lab[j] - lb);
                if (tj < bt || (tj == bt && (uint32_t)lab[j] < lb2)) {
                    bt = tj;
                    lb2 = (uint32_t)lab[j];
                }
            }
            const uint32_t wt = __reduce_min_sync(0xffffffffu, bt);
            bl = (int32_t)__reduce_min_sync(0xffffffffu, bt == wt ? lb2 : 0x7fffffffu);
            best |= (uint32_t)~wt;
        }
        __syncwarp();
        if (lane == 0) t.ndl = 0;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) bl = min(bl, __shfl_xor_sync(0xffffffffu, bl, d));
    __syncwarp();
    if (lane == 0) record_visit(a, v, best, ownw);
    if (lane == 0 && best != 0) {
        const int32_t gain = (int32_t)(best >> 32) - ownw;
        const bool ovl = MODE != kCluster && Wown > bnd(a, own);
        if (gain > 0 || ovl) {
            const int64_t wT = DENSE ? Wsm[bl] : a.W[bl];
            emit<DENSE>(a, v, bl, own, gain, c, ovl, wT);
        }
    }
}

// Rows of <= kMedDeg entries: warps take small-row items (G lanes per row)
// and then medium rows (a warp per row).  Runs next to k_propose (side stream).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 5) k_propose_small(LPArgs a, int k) {
    if (stopped(a)) return;
    __shared__ int64_t W[kDenseMaxK];
    __shared__ WarpTab tabs[MODE == kRefineDense ? 1 : kThreads / 32];
    __shared__ int32_t dacc[MODE == kRefineDense ? kThreads / 32 : 1][kDenseMaxK];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (MODE == kRefineDense) {
        for (int b = threadIdx.x; b < k; b += kThreads) W[b] = a.W[b];
        for (int b = lane; b < kDenseMaxK; b += 32) dacc[warp][b] = 0;
    } else {
        for (int i = lane; i < kWSlots; i += 32) {
            tabs[warp].s[i] = kEmpty;
        }
        if (lane == 0) tabs[warp].ndl = 0;
    }
    __syncthreads();
    process_small<MODE>(a, W);
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int bm = kClasses * a.colour + 4;
    const int32_t *wl = a.wl + (int64_t)bm * a.g.n;
    const int64_t nmed = a.wl_cnt[bm];
    WarpTab &t = tabs[MODE == kRefineDense ? 0 : warp];
    int32_t *dacc_w = dacc[MODE == kRefineDense ? warp : 0];
    for (int64_t i = gwarp; i < nmed; i += nwarps) medium_row<MODE>(a, W, t, dacc_w, k, wl[i]);
}

// ---------------------------------------------------------------- arbitration

// Digit windows of the weighted radix select.  Keys are (order-flipped gain
// << 32) | node id.  The first window starts at `top`, the highest bit where
// the smallest and largest weighted keys differ; windows are at most kDigit
// bits wide and do not cross bit 32; below bit 32 they start at `idtop`, the
// highest bit set in any weighted key's node id (the bits in between are zero
// in every key).  Returns false when no window is left.
__device__ __forceinline__ bool sel_window(int top, int idtop, int p, int *hb, int *width) {
    int cur = top;
    for (int q = 0;; q++) {
        if (cur >= 32) {
            const int lo = max(32, cur - kDigit + 1);
            if (q == p) { *hb = cur; *width = cur - lo + 1; return true; }
            cur = lo - 1;
            if (cur == 31) cur = min(31, idtop);
        } else {
            if (cur < 0) return false;
            const int lo = max(0, cur - kDigit + 1);
            if (q == p) { *hb = cur; *width = cur - lo + 1; return true; }
            cur = lo - 1;
        }
    }
}

// Highest differing key bit, or -1 if kmin > kmax (no weighted entry).
__device__ __forceinline__ int key_top(unsigned long long kmin, unsigned long long kmax) {
    if (kmin > kmax) return -1;
    const unsigned long long diff = kmin ^ kmax;
    return diff ? 63 - __clzll((long long)diff) : 0;
}

__device__ __forceinline__ int id_top(unsigned idmax) {
    return idmax ? 31 - __clz((int)idmax) : 0;
}

// Adds weight c (>= 0) to bin d: lo sums the low 16 bits, hi the rest (native
// 32-bit shared atomics; exact while a histogram takes <= 65536 entries).
__device__ __forceinline__ void split_add(uint32_t *lo, uint32_t *hi, unsigned d, int32_t c) {
    atomicAdd(&lo[d], (uint32_t)c & 0xffffu);
    if ((uint32_t)c >> 16) atomicAdd(&hi[d], (uint32_t)c >> 16);
}

// Digit choice of one pass over the bins h[0, nb): the first bin d where
// acc + (weight of bins <= d) >= thr, by a block-wide scan (thread t owns 8
// consecutive bins).  Writes *s_pf |= d << shift and *s_acc, or *s_done = 1
// when the total stays below thr.  All threads of the CTA call it.
__device__ __forceinline__ void sel_decide(const unsigned long long *h, unsigned nb, int shift,
                                           int64_t thr, int64_t *s_acc, uint64_t *s_pf,
                                           int *s_done, int64_t *scan_tmp /* kThreads/32+1 */) {
    static_assert(kBins == 8 * kThreads, "8 bins per thread");
    const unsigned b0 = threadIdx.x * 8;
    int64_t v[8], local = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        v[j] = b0 + j < nb ? (int64_t)h[b0 + j] : 0;
        local += v[j];
    }
    const int64_t acc = *s_acc;
    int64_t total;
    const int64_t ex = block_exclusive_scan<kThreads>(local, &total, scan_tmp);
    if (acc + total < thr) {
        if (threadIdx.x == 0) *s_done = 1;
    } else if (acc + ex + local >= thr && (threadIdx.x == 0 || acc + ex < thr)) {
        int64_t run = acc + ex;
        unsigned d = b0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (run + v[j] >= thr) { d = b0 + j; break; }
            run += v[j];
        }
        *s_acc = run;
        *s_pf |= (uint64_t)d << shift;
    }
    __syncthreads();
}

// Min and max key and max node id over the entries with c > 0 (all threads).
template <typename Get>
__device__ void block_minmax(Get get, int64_t cnt, uint64_t *out_min, uint64_t *out_max,
                             unsigned *out_idmax, unsigned long long *red /* [96] */) {
    unsigned long long mn = ~0ull, mx = 0;
    unsigned im = 0;
    for (int64_t base = threadIdx.x; base < cnt; base += 4 * (int64_t)blockDim.x) {
        uint64_t kk[4];
        int32_t cc[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t i = base + j * (int64_t)blockDim.x;
            kk[j] = 0;
            cc[j] = 0;
            if (i < cnt) get(i, &kk[j], &cc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (cc[j] <= 0) continue;
            mn = kk[j] < mn ? kk[j] : mn;
            mx = kk[j] > mx ? kk[j] : mx;
            im = max(im, (unsigned)kk[j]);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, mn, d);
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, d);
        mn = x < mn ? x : mn;
        mx = y > mx ? y : mx;
        im = max(im, __shfl_xor_sync(0xffffffffu, im, d));
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[w] = mn;
        red[32 + w] = mx;
        red[64 + w] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
            mn = red[i] < mn ? red[i] : mn;
            mx = red[32 + i] > mx ? red[32 + i] : mx;
            im = max(im, (unsigned)red[64 + i]);
        }
        red[0] = mn;
        red[32] = mx;
        red[64] = im;
    }
    __syncthreads();
    *out_min = red[0];
    *out_max = red[32];
    *out_idmax = (unsigned)red[64];
    __syncthreads();
}

// Weighted radix select: the smallest key K such that the total weight of the
// entries with key <= K is >= thr; ~0 if the total is < thr.  get(i, &key, &c)
// returns entry i (c = 0 entries carry no weight); kmin / kmax / idmax come
// from block_minmax.  Windows from sel_window; each pass histograms the
// entries that match the digits fixed so far.  All threads of the CTA call it.
template <typename Get>
__device__ uint64_t select_first_reaching(Get get, int64_t cnt, int64_t thr, uint64_t kmin,
                                          uint64_t kmax, unsigned idmax,
                                          unsigned long long *hist /* [kBins] */,
                                          int64_t *s_acc, uint64_t *s_pf, int *s_done,
                                          int64_t *scan_tmp /* kThreads/32+1 */) {
    const int top = key_top(kmin, kmax);
    if (top < 0) return ~0ull;  // no weighted entry: everything is admitted
    const int itop = id_top(idmax);
    if (threadIdx.x == 0) {
        *s_acc = 0;
        *s_pf = top >= 63 ? 0ull : (kmin & (~0ull << (top + 1)));
        *s_done = 0;
    }
    __syncthreads();
    const bool split = cnt <= 65536;  // else 64-bit bins
    uint32_t *hlo = reinterpret_cast<uint32_t *>(hist), *hhi = hlo + kBins;
    const int64_t step = 4 * (int64_t)blockDim.x;
    int hb, width;
    for (int p = 0; sel_window(top, itop, p, &hb, &width); p++) {
        const int shift = hb - width + 1;
        const unsigned nb = 1u << width;
        for (unsigned i = threadIdx.x; i < kBins; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t hm = (hb >= 63) ? 0ull : (~0ull << (hb + 1));
        const uint64_t pf = *s_pf;
        for (int64_t base = threadIdx.x; base < cnt; base += step) {
            uint64_t kk[4];
            int32_t cc[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t i = base + j * (int64_t)blockDim.x;
                kk[j] = 0;
                cc[j] = 0;
                if (i < cnt) get(i, &kk[j], &cc[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (cc[j] <= 0 || (kk[j] & hm) != (pf & hm)) continue;
                const unsigned d = (unsigned)((kk[j] >> shift) & (nb - 1));
                if (split) split_add(hlo, hhi, d, cc[j]);
                else atomicAdd(&hist[d], (unsigned long long)cc[j]);
            }
        }
        __syncthreads();
        if (split) {  // to 64-bit bins: bin i reads its halves before anyone writes it
            unsigned long long t[kBins / kThreads];
#pragma unroll
            for (int j = 0; j < kBins / kThreads; j++) {
                const unsigned i = threadIdx.x + j * kThreads;
                t[j] = (unsigned long long)hlo[i] + ((unsigned long long)hhi[i] << 16);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < kBins / kThreads; j++) hist[threadIdx.x + j * kThreads] = t[j];
            __syncthreads();
        }
        sel_decide(hist, nb, shift, thr, s_acc, s_pf, s_done, scan_tmp);
        if (*s_done) return ~0ull;
    }
    return *s_pf;
}

struct ArbSm {
    WDelta wd;
    unsigned long long hist[kBins];
    unsigned long long red[96];
    int64_t scan_tmp[kThreads / 32 + 1];
    uint64_t keys[kSegSmem];
    int32_t c[kSegSmem];
    int64_t acc;
    uint64_t pf;
    int done;
};

// Copies entries [0, cnt) of a contested segment into shared memory (key,
// weight); each thread issues 8 loads before its stores.
__device__ __forceinline__ void stage_segment(const SegEntry *ent, int cnt, uint64_t *keys,
                                              int32_t *c) {
    for (int base = threadIdx.x; base < cnt; base += 8 * blockDim.x) {
        SegEntry e[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = base + j * blockDim.x;
            if (i < cnt) e[j] = ldcg_entry(&ent[i]);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = base + j * blockDim.x;
            if (i < cnt) {
                keys[i] = e[j].key;
                c[i] = e[j].c;
            }
        }
    }
}

// Admits the staged entries of a segment with key < K (and weight 0).  The
// owners are loaded 8 per thread ahead of the moves; the weight leaving each
// owner is summed over the warp's lanes with that owner, the weight entering
// T per thread and then per warp.  Whole warps iterate.
__device__ __forceinline__ int64_t admit_segment(const LPArgs &a, WDelta &wd, const SegEntry *ent,
                                                 int cnt, const uint64_t *keys, const int32_t *c,
                                                 uint64_t K, int32_t T) {
    const int lane = threadIdx.x & 31;
    unsigned long long *dst = a.nW <= kAggW ? (unsigned long long *)wd.d
                                             : (unsigned long long *)a.W;
    int64_t moved = 0;
    long long tin = 0;
    const int cnt_r = (cnt + 31) & ~31;
    for (int base = threadIdx.x; base < cnt_r; base += 8 * blockDim.x) {
        int32_t own[8];
        bool adm[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = base + j * blockDim.x;
            adm[j] = i < cnt && (keys[i] < K || c[i] == 0);
            own[j] = adm[j] ? __ldcg(&ent[i].own) : -1;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int i = base + j * blockDim.x;
            if (i - lane >= cnt_r) break;  // warp-uniform
            const int32_t cj = adm[j] ? c[i] : 0;
            if (adm[j]) {
                a.lab[(int32_t)(uint32_t)keys[i]] = T;
                tin += cj;
                moved++;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, (unsigned)own[j]);
            const unsigned lo = __reduce_add_sync(peers, (unsigned)cj & 0xffffu);
            const unsigned hi = __reduce_add_sync(peers, (unsigned)cj >> 16);
            if (adm[j] && (peers & ((1u << lane) - 1)) == 0)
                atomicAdd(&dst[own[j]], (unsigned long long)(-(((long long)hi << 16) + lo)));
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tin += __shfl_down_sync(0xffffffffu, tin, d);
    if (lane == 0 && tin) atomicAdd(&dst[T], (unsigned long long)tin);
    return moved;
}

// Refinement: departures from overloaded blocks (slot == -2).  CTAs with
// blockIdx < nW handle block b = blockIdx when its departures are contested;
// the others pass the uncontested sources' proposals through.
__global__ void __launch_bounds__(kThreads) k_src(LPArgs a) {
    if (stopped(a)) return;
    __shared__ unsigned long long hist[kBins];
    __shared__ unsigned long long red[96];
    __shared__ int64_t scan_tmp[kThreads / 32 + 1];
    __shared__ int64_t s_acc;
    __shared__ uint64_t s_pf;
    __shared__ int s_done;
    const int nprop = a.ctr->nprop;
    if (blockIdx.x < a.nW) {
        const int32_t b = blockIdx.x;
        const int64_t Wb = a.W[b];
        if (Wb <= bnd(a, b)) return;
        const int64_t X = Wb - bnd(a, b);
        if (a.ssum[b] < X) return;  // uncontested: handled by the pass-through CTAs
        auto get = [&](int64_t i, uint64_t *key, int32_t *c) {
            const Prop &p = a.props[i];
            const bool mine = p.slot == -2 && p.own == b;
            *key = mine ? seg_key(p.gain, p.v) : 0;
            *c = mine ? p.c : 0;
        };
        uint64_t kmin, kmax;
        unsigned idmax;
        block_minmax(get, nprop, &kmin, &kmax, &idmax, red);
        const uint64_t K = select_first_reaching(get, nprop, X, kmin, kmax, idmax, hist, &s_acc,
                                                 &s_pf, &s_done, scan_tmp);
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
        if (a.ssum[p.own] < a.W[p.own] - bnd(a, p.own)) {
            atomicAdd((unsigned long long *)&a.tsum[p.T], (unsigned long long)(int64_t)p.c);
            p.slot = atomicAdd(&a.tcnt[p.T], 1);
        }
    }
}

// Grid-wide barrier of a cooperative launch.  The wait is bounded: a CTA
// that waits longer than `limit` SM clock cycles (or sees the error flag
// raised) sets kErrBarrier and goes on; the host then reports the failure.
constexpr long long kBarCycles = 4000000000ll;  // about two seconds at 2 GHz

__device__ void grid_barrier(GridBar *bar, int32_t *err, long long limit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &bar->gen;
        volatile int32_t *verr = err;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned old = atomicAdd(&bar->count, 1u);
        if (old == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (*verr & kErrBarrier) break;
                if (clock64() - t0 > limit) {
                    atomicOr(err, kErrBarrier);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Self-test of the bounded wait: CTA 0 never arrives, so CTA 1 must give up
// after `limit` cycles, raise kErrBarrier and return.
__global__ void k_barrier_selftest(GridBar *bar, int32_t *err, long long limit) {
    if (blockIdx.x == 0) return;
    grid_barrier(bar, err, limit);
}

// Number of select passes of a big segment.
__device__ __forceinline__ int big_passes(int top, int itop) {
    if (top < 0) return 0;
    int hb, width, p = 0;
    while (sel_window(top, itop, p, &hb, &width)) p++;
    return p;
}

// Control values of big-segment tile t, read by thread 0 and handed to the
// CTA through shared memory so that every thread takes the same branches.
struct BigTile {
    int32_t ok, bi, len, top, itop, done;
    int64_t i0;
    Seg sg;
    unsigned long long kmin, pf;
};

__device__ __forceinline__ BigTile big_tile(const LPArgs &a, int t, int nbig, BigTile *s_bt) {
    if (threadIdx.x == 0) {
        BigTile bt{};
        const int32_t bi = __ldcg(&a.tileseg[t]);
        if (bi >= 0 && bi < nbig) {
            const BigSeg *b = &a.big[bi];
            bt.bi = bi;
            bt.sg = ldcg_seg(&a.segs[__ldcg(&b->si)]);
            bt.i0 = (int64_t)(t - __ldcg(&b->t0)) * kBigTile;
            const int64_t rest = bt.sg.cnt - bt.i0;
            bt.len = (int)(rest < kBigTile ? rest : kBigTile);
            bt.kmin = __ldcg(&b->kmin);
            bt.top = key_top(bt.kmin, __ldcg(&b->kmax));
            bt.itop = id_top(__ldcg(&b->idmax));
            bt.done = __ldcg(&b->done);
            bt.pf = __ldcg(&b->pf);
            bt.ok = bt.len > 0 && bt.i0 >= 0;
        }
        *s_bt = bt;
    }
    __syncthreads();
    const BigTile bt = *s_bt;
    __syncthreads();
    return bt;
}

// Segments of more than kSegSmem entries: the weighted select of
// select_first_reaching, with each pass's histogram summed over the tiles of
// all CTAs.  The CTA that flushes a segment's last tile of a pass picks the
// digit; a grid barrier separates the passes.  Tile blockIdx.x stays staged in
// shared memory from the first read to the last.
__device__ void arbitrate_big(const LPArgs &a, ArbSm &sm, int nbig, int ntiles, int64_t &moved) {
    __shared__ int s_flag, s_passes, s_done;
    __shared__ int64_t s_acc;
    __shared__ uint64_t s_pf;
    __shared__ BigTile s_bt;
    const int lane = threadIdx.x & 31;
    // pass 0: key range of each segment
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BigTile bt = big_tile(a, t, nbig, &s_bt);
        if (!bt.ok) continue;
        const SegEntry *ent = a.segbuf + bt.sg.base + bt.i0;
        const bool stage = t == (int)blockIdx.x;
        unsigned long long mn = ~0ull, mx = 0;
        unsigned im = 0;
        for (int base = threadIdx.x; base < bt.len; base += 8 * blockDim.x) {
            SegEntry e[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = base + j * blockDim.x;
                e[j].c = 0;
                if (i < bt.len) e[j] = ldcg_entry(&ent[i]);
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int i = base + j * blockDim.x;
                if (i >= bt.len) continue;
                if (stage) {
                    sm.keys[i] = e[j].key;
                    sm.c[i] = e[j].c;
                }
                if (e[j].c > 0) {
                    mn = e[j].key < mn ? e[j].key : mn;
                    mx = e[j].key > mx ? e[j].key : mx;
                    im = max(im, (unsigned)e[j].key);
                }
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long x = __shfl_xor_sync(0xffffffffu, mn, d);
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, d);
            mn = x < mn ? x : mn;
            mx = y > mx ? y : mx;
            im = max(im, __shfl_xor_sync(0xffffffffu, im, d));
        }
        if (lane == 0 && mn <= mx) {
            atomicMin(&a.big[bt.bi].kmin, mn);
            atomicMax(&a.big[bt.bi].kmax, mx);
            atomicMax(&a.big[bt.bi].idmax, im);
        }
        __syncthreads();
    }
    grid_barrier(a.bar, &a.ctr->err, a.bar_cycles);
    if (threadIdx.x == 0) s_passes = 0;
    __syncthreads();
    {
        int mp = 0;
        for (int bi = threadIdx.x; bi < nbig; bi += blockDim.x)
            mp = max(mp, big_passes(key_top(__ldcg(&a.big[bi].kmin), __ldcg(&a.big[bi].kmax)),
                                    id_top(__ldcg(&a.big[bi].idmax))));
        atomicMax(&s_passes, mp);
    }
    __syncthreads();
    const int passes = s_passes;
    for (int p = 0; p < passes; p++) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const BigTile bt = big_tile(a, t, nbig, &s_bt);
            int hb, width;
            if (!bt.ok || bt.top < 0 || bt.done || !sel_window(bt.top, bt.itop, p, &hb, &width))
                continue;
            BigSeg *b = &a.big[bt.bi];
            const int shift = hb - width + 1;
            const unsigned nb = 1u << width;
            const unsigned long long hm = hb >= 63 ? 0ull : (~0ull << (hb + 1));
            const unsigned long long pf =
                p == 0 ? (bt.top >= 63 ? 0ull : (bt.kmin & (~0ull << (bt.top + 1)))) : bt.pf;
            uint32_t *hlo = reinterpret_cast<uint32_t *>(sm.hist), *hhi = hlo + kBins;
            for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) hlo[i] = hhi[i] = 0;
            __syncthreads();
            const bool staged = t == (int)blockIdx.x;
            const SegEntry *ent = a.segbuf + bt.sg.base + bt.i0;
            const int len_r = (bt.len + blockDim.x - 1) / blockDim.x * blockDim.x;
            for (int i = threadIdx.x; i < len_r; i += blockDim.x) {
                uint64_t key = 0;
                int32_t c = 0;
                if (i < bt.len) {
                    if (staged) {
                        key = sm.keys[i];
                        c = sm.c[i];
                    } else {
                        const SegEntry e = ent[i];
                        key = e.key;
                        c = e.c;
                    }
                }
                if (c > 0 && (key & hm) == (pf & hm))  // a tile has <= 4096 entries
                    split_add(hlo, hhi, (unsigned)((key >> shift) & (nb - 1)), c);
            }
            __syncthreads();
            unsigned long long *gh = a.bhist + (size_t)bt.bi * kBins;
            for (unsigned i = threadIdx.x; i < nb; i += blockDim.x) {
                const unsigned long long tot =
                    (unsigned long long)hlo[i] + ((unsigned long long)hhi[i] << 16);
                if (tot) atomicAdd(&gh[i], tot);
            }
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_flag = atomicAdd(&b->arrived, 1) == __ldcg(&b->tiles) - 1;
            __syncthreads();
            const int last = s_flag;
            __syncthreads();
            if (!last) continue;
            // last tile of this segment in this pass: pick the digit from the
            // summed histogram, staged in shared memory (and cleared behind)
            __threadfence();
            {
                unsigned long long hv[kBins / kThreads];
#pragma unroll
                for (int j = 0; j < kBins / kThreads; j++) {
                    const unsigned i = threadIdx.x + j * kThreads;
                    hv[j] = i < nb ? __ldcg(&gh[i]) : 0ull;
                }
#pragma unroll
                for (int j = 0; j < kBins / kThreads; j++) {
                    const unsigned i = threadIdx.x + j * kThreads;
                    if (i < nb) {
                        sm.hist[i] = hv[j];
                        gh[i] = 0;
                    }
                }
            }
            if (threadIdx.x == 0) {
                s_acc = p == 0 ? 0ll : __ldcg(&b->acc);
                s_pf = pf;
                s_done = 0;
            }
            __syncthreads();
            sel_decide(sm.hist, nb, shift, bt.sg.thr, &s_acc, &s_pf, &s_done, sm.scan_tmp);
            if (threadIdx.x == 0) {
                if (s_done) b->done = 1;
                else {
                    b->acc = s_acc;
                    b->pf = s_pf;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) b->arrived = 0;
            __threadfence();
            __syncthreads();
        }
        grid_barrier(a.bar, &a.ctr->err, a.bar_cycles);
    }
    // admissions: keys below K (and entries of weight 0)
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BigTile bt = big_tile(a, t, nbig, &s_bt);
        if (!bt.ok) continue;
        const unsigned long long K = (bt.top < 0 || bt.done) ? ~0ull : bt.pf;
        const SegEntry *ent = a.segbuf + bt.sg.base + bt.i0;
        if (t != (int)blockIdx.x) {  // tiles after the first: stage them now
            stage_segment(ent, bt.len, sm.keys, sm.c);
            __syncthreads();
        }
        moved += admit_segment(a, sm.wd, ent, bt.len, sm.keys, sm.c, K, bt.sg.T);
        __syncthreads();
    }
}

// Launched cooperatively (all CTAs resident): segments of <= 32 entries take
// one warp, up to kSegSmem one CTA, longer ones the whole grid.
// The whole settle step of a sub-round in one cooperative launch (every CTA
// resident): classify the proposals (uncontested targets applied, contested
// ones get a segment), grid barrier, scatter contested proposals into their
// segments and clear the per-target accumulators, grid barrier, then admit
// per segment.  State that other CTAs wrote in this launch is read with
// L2-coherent loads.
__global__ void __launch_bounds__(kThreads) k_arbitrate(LPArgs a) {
    if (stopped(a)) return;  // the same in every CTA, before any grid barrier
    extern __shared__ __align__(16) unsigned char smraw[];
    ArbSm &sm = *reinterpret_cast<ArbSm *>(smraw);
    wd_init(sm.wd, a.nW);
    const int lane = threadIdx.x & 31;
    int64_t moved = 0;
    const int nprop = __ldcg(&a.ctr->nprop);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    // classify
    for (int64_t i = gtid; i < nprop; i += gthreads) {
        const Prop p = a.props[i];
        if (p.slot < 0) continue;
        const int64_t cap = bnd(a, p.T) - p.wT;
        if (a.tsum[p.T] <= cap) {
            apply_agg(a, sm.wd, p.v, p.T, p.own, p.c);
            moved++;
        } else if (p.slot == 0) {
            const int32_t cnt = a.tcnt[p.T];
            const int si = atomicAdd(&a.ctr->nseg, 1);
            const int64_t base = (int64_t)atomicAdd((unsigned long long *)&a.ctr->segtotal,
                                                    (unsigned long long)cnt);
            a.tbase[p.T] = base;
            a.segs[si] = Seg{p.T, cnt, base, cap + 1};
            if (cnt > a.t.seg_smem) {
                const int nt = (cnt + kBigTile - 1) / kBigTile;
                const int bi = atomicAdd(&a.ctr->nbig, 1);
                const int t0 = atomicAdd(&a.ctr->bigtiles, nt);
                if (bi >= a.maxbig || t0 + nt > a.maxtiles) {
                    atomicOr(&a.ctr->err, kErrBig);  // cannot happen: capacities bound the totals
                } else {
                    a.big[bi] = BigSeg{si, nt, t0, 0, ~0ull, 0ull, 0ull, 0ll, 0, 0u};
                    for (int t = 0; t < nt; t++) a.tileseg[t0 + t] = bi;
                }
            }
        }
    }
    grid_barrier(a.bar, &a.ctr->err, a.bar_cycles);
    const int nseg = __ldcg(&a.ctr->nseg);
    // scatter contested proposals; then nothing reads the per-target sums
    if (nseg > 0) {
        for (int64_t i = gtid; i < nprop; i += gthreads) {
            const Prop p = a.props[i];
            if (p.slot < 0) continue;
            if (a.tsum[p.T] <= bnd(a, p.T) - p.wT) continue;
            a.segbuf[__ldcg(&a.tbase[p.T]) + p.slot] = SegEntry{seg_key(p.gain, p.v), p.c, p.own};
        }
    }
    grid_barrier(a.bar, &a.ctr->err, a.bar_cycles);
    for (int64_t i = gtid; i < nprop; i += gthreads) {
        const Prop p = a.props[i];
        a.tsum[p.T] = 0;
        a.tcnt[p.T] = 0;
        if (a.ssum) a.ssum[p.own] = 0;
    }
    // small segments: one warp each, exact prefix by brute force over <= 32 lanes
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int si = gwarp; si < nseg; si += nwarps) {
        const Seg sg = ldcg_seg(&a.segs[si]);
        if (sg.cnt > 32) continue;
        uint64_t key = ~0ull;
        int32_t c = 0, own = 0;
        if (lane < sg.cnt) {
            const SegEntry e = ldcg_entry(&a.segbuf[sg.base + lane]);
            key = e.key;
            c = e.c;
            own = e.own;
        }
        int64_t pre = 0;
        for (int j = 0; j < sg.cnt; j++) {
            const uint64_t kj = __shfl_sync(0xffffffffu, key, j);
            const int32_t cj = __shfl_sync(0xffffffffu, c, j);
            if (kj <= key) pre += cj;
        }
        if (lane < sg.cnt && (c == 0 || pre < sg.thr)) {
            apply_agg(a, sm.wd, (int32_t)(uint32_t)key, sg.T, own, c);
            moved++;
        }
    }
    // medium segments: one CTA each, staged in shared memory
    for (int si = blockIdx.x; si < nseg; si += gridDim.x) {
        const Seg sg = ldcg_seg(&a.segs[si]);
        if (sg.cnt <= 32 || sg.cnt > a.t.seg_smem) continue;
        const SegEntry *ent = a.segbuf + sg.base;
        stage_segment(ent, sg.cnt, sm.keys, sm.c);
        __syncthreads();
        auto get = [&](int64_t i, uint64_t *key, int32_t *c) {
            *key = sm.keys[i];
            *c = sm.c[i];
        };
        uint64_t kmin, kmax;
        unsigned idmax;
        block_minmax(get, sg.cnt, &kmin, &kmax, &idmax, sm.red);
        const uint64_t K = select_first_reaching(get, sg.cnt, sg.thr, kmin, kmax, idmax, sm.hist,
                                                 &sm.acc, &sm.pf, &sm.done, sm.scan_tmp);
        moved += admit_segment(a, sm.wd, ent, sg.cnt, sm.keys, sm.c, K, sg.T);
        __syncthreads();
    }
    // long segments: the whole grid (the same branch in every CTA)
    const int nbig = __ldcg(&a.ctr->nbig), ntiles = __ldcg(&a.ctr->bigtiles);
    if (nbig > 0 && !(__ldcg(&a.ctr->err) & kErrBig) && nbig <= a.maxbig && ntiles <= a.maxtiles) {
        __syncthreads();
        arbitrate_big(a, sm, nbig, ntiles, moved);
    }
    wd_flush(a, sm.wd);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) moved += __shfl_down_sync(0xffffffffu, moved, d);
    if (lane == 0 && moved) atomicAdd((unsigned long long *)a.moves, (unsigned long long)moved);
}

// ---------------------------------------------------------------- multi-piece rows (hash)

// Rows longer than one piece have their (label, omega) sums merged in a
// global table by the propose kernel; these three kernels select their best
// label in parallel: items of kFin distinct entries, enumerated over all
// multi-piece rows (rows of other sub-rounds are skipped).
constexpr int kFin = 2048;

struct HubItem {
    int64_t li;
    int64_t begin, end;  // distinct-list range of this item
    bool active;
};

__device__ __forceinline__ HubItem hub_item(const LPArgs &a, int64_t t, int round) {
    int64_t lo = 0, hi = a.nL;  // largest li with Hfin[li] <= t
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.Hfin[mid] <= t) lo = mid;
        else hi = mid;
    }
    HubItem it;
    it.li = lo;
    const int64_t c = t - a.Hfin[lo];
    const int64_t ndl = __ldcg(&a.Lndl[lo]);
    it.begin = c * kFin;
    it.end = min64(ndl, it.begin + kFin);
    it.active = colour_of(a, a.Lnodes[lo]) == (uint32_t)a.colour &&
                it.begin < it.end;
    return it;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hub_cand(LPArgs a) {
    if (stopped(a)) return;
    __shared__ unsigned long long red[kThreads / 32];
    const int64_t items = a.Hfin[a.nL];
    for (int64_t t = blockIdx.x; t < items; t += gridDim.x) {
        const HubItem it = hub_item(a, t, a.round);
        if (!it.active) continue;  // uniform over the CTA
        const int32_t v = a.Lnodes[it.li];
        const int32_t own = a.lab[v], c = a.g.vwgt[v];
        const uint64_t h = nhash(a, v);
        const int32_t lb = lbase(a, v);
        const int64_t off = a.Loff[it.li];
        const int32_t *gdl = a.gdl + a.Ldlo[it.li];
        uint32_t mw = 0;
        for (int64_t i = it.begin + threadIdx.x; i < it.end; i += kThreads) {
            const int32_t slot = __ldcg(&gdl[i]);
            const int32_t L = (int32_t)(uint32_t)__ldcg(&a.gkeys[off + slot]);
            const uint32_t w = (uint32_t)__ldcg(&a.gvals[off + slot]);
            if (L == own) a.hown[it.li] = (int32_t)w;
            else if (w > mw && a.W[L] + c <= bnd(a, L)) mw = w;
        }
        mw = __reduce_max_sync(0xffffffffu, mw);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mw;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kThreads / 32; w++) mw = max(mw, (uint32_t)red[w]);
            if (mw) atomicMax(&a.hbest[it.li], (unsigned long long)mw << 32);
        }
        __syncthreads();
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hub_tie(LPArgs a) {
    if (stopped(a)) return;
    const int64_t items = a.Hfin[a.nL];
    for (int64_t t = blockIdx.x; t < items; t += gridDim.x) {
        const HubItem it = hub_item(a, t, a.round);
        if (!it.active) continue;
        const int32_t v = a.Lnodes[it.li];
        const int32_t own = a.lab[v], c = a.g.vwgt[v];
        const uint64_t h = nhash(a, v);
        const int32_t lb = lbase(a, v);
        const int64_t off = a.Loff[it.li];
        const int32_t *gdl = a.gdl + a.Ldlo[it.li];
        // tie hashes only for a row that proposes, only at omega M
        const uint32_t M = (uint32_t)(a.hbest[it.li] >> 32);
        const bool ovl = MODE != kCluster && a.W[own] > bnd(a, own);
        const bool prop = M > 0 && ((int32_t)M > __ldcg(&a.hown[it.li]) || ovl);
        unsigned long long tl = ~0ull;
        for (int64_t i = it.begin + threadIdx.x; i < it.end; i += kThreads) {
            const int32_t slot = __ldcg(&gdl[i]);
            const int32_t L = (int32_t)(uint32_t)__ldcg(&a.gkeys[off + slot]);
            const uint32_t w = (uint32_t)__ldcg(&a.gvals[off + slot]);
            if (prop && L != own && w == M && a.W[L] + c <= bnd(a, L)) {
                const unsigned long long x = ((unsigned long long)tie_of(h, L - lb) << 32) | (uint32_t)L;
                tl = x < tl ? x : tl;
            }
            a.gkeys[off + slot] = kEmpty;
            a.gvals[off + slot] = 0;
        }
        if (__any_sync(0xffffffffu, tl != ~0ull)) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const unsigned long long o = __shfl_xor_sync(0xffffffffu, tl, d);
                tl = o < tl ? o : tl;
            }
            if ((threadIdx.x & 31) == 0) atomicMin(&a.htl[it.li], tl);
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_hub_emit(LPArgs a) {
    if (stopped(a)) return;
    for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < a.nL;
         li += (int64_t)gridDim.x * blockDim.x) {
        if (a.Hfin[li + 1] == a.Hfin[li]) continue;  // single-piece row
        const int32_t v = a.Lnodes[li];
        if (colour_of(a, v) != (uint32_t)a.colour) continue;
        const unsigned long long b = a.hbest[li];  // omega M << 32
        const int32_t own = a.lab[v];
        record_visit(a, v, b, a.hown[li]);
        if (b != 0) {
            const int32_t gain = (int32_t)(b >> 32) - a.hown[li];
            const bool ovl = MODE != kCluster && a.W[own] > bnd(a, own);
            if (gain > 0 || ovl) {
                const int32_t L = (int32_t)(uint32_t)a.htl[li];
                emit<false>(a, v, L, own, gain, a.g.vwgt[v], ovl, a.W[L]);
            }
        }
        a.hbest[li] = 0;
        a.htl[li] = ~0ull;
        a.hown[li] = 0;
        a.Lndl[li] = 0;
    }
}

// ---------------------------------------------------------------- rows of one CTA cluster

// Rows with kChunk < degree <= kHugeDeg (hash modes): a cluster of kHugeCS
// CTAs takes one row at a time.  The row's (label, omega) sums live in one
// open-addressing table spread over the CTAs' shared memory (slot s sits in
// CTA s / T); each CTA reads a contiguous share of the row and inserts into
// the owning CTA's slots through distributed shared memory.  The table has
// >= 2 * degree slots, so an insert always finds room.  Selection: the
// largest eligible omega M and the own label's omega over the cluster, the
// gain rule of Sec. III.A, and, only for a row that proposes, the smallest
// (tie, label) over the labels at omega M (the label of the largest
// cand_key, ties on the key to the smallest label).
// Per-CTA results are written to the CTA's own shared memory and read by the
// others with plain loads after a cluster barrier: only 32-bit CAS and add
// go to another CTA's shared memory.
struct HugeSm {
    uint32_t keys[kHugeSlots];
    int32_t vals[kHugeSlots];
    unsigned long long red[kThreads / 32];
    unsigned long long cbest;  // this CTA's largest eligible omega
    unsigned long long b;      // the cluster's (local copy)
    unsigned long long ctl;    // this CTA's smallest (tie << 32 | label) at omega b
    int32_t cown, bown;        // own label's sum: this CTA's, the cluster's
    int32_t item;              // rank 0: index into this colour's row list
};

__device__ __forceinline__ void huge_insert(cg::cluster_group &cl, HugeSm &sm, uint32_t L,
                                            int32_t w, int tbits, int lbits) {
    const uint32_t tmask = (1u << tbits) - 1;
    uint32_t q = (L * 0x9E3779B1u) >> (32 - tbits);
    for (uint32_t probe = 0; probe <= tmask; probe++) {
        const unsigned owner = q >> lbits;
        const uint32_t loc = q & ((1u << lbits) - 1);
        uint32_t *kp = cl.map_shared_rank(&sm.keys[loc], owner);
        const uint32_t prev = atomicCAS(kp, kEmpty32, L);
        if (prev == kEmpty32 || prev == L) {
            atomicAdd(cl.map_shared_rank(&sm.vals[loc], owner), w);
            return;
        }
        q = (q + 1) & tmask;
    }
}

template <int MODE>
__global__ void __cluster_dims__(kHugeCS, 1, 1) __launch_bounds__(kThreads)
    k_propose_huge(LPArgs a) {
    if (stopped(a)) return;  // the same in every CTA of the cluster
    __shared__ HugeSm sm;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    HugeSm *r0 = cl.map_shared_rank(&sm, 0u);
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kHugeSlots; i += kThreads) {
        sm.keys[i] = kEmpty32;
        sm.vals[i] = 0;
    }
    const int nrows = a.hcnt[a.colour];
    const int32_t *hl = a.hlist + (int64_t)a.colour * a.nL;
    while (true) {
        if (rank == 0 && threadIdx.x == 0) sm.item = atomicAdd(&a.ctr->huge_next, 1);
        cl.sync();
        const int it = r0->item;
        if (it >= nrows) break;  // the same value in every CTA of the cluster
        if (threadIdx.x == 0) {
            sm.ctl = ~0ull;
            sm.cown = 0;
        }
        const int32_t li = hl[it];
        const int32_t v = a.Lnodes[li];
        const int64_t rs = a.g.xadj[v];
        const int64_t deg = a.g.xadj[v + 1] - rs;
        const int32_t own = a.lab[v], c = a.g.vwgt[v];
        const int32_t cpv = (MODE == kCluster && a.cp) ? a.cp[v] : 0;
        const uint64_t h = nhash(a, v);
        const int32_t lb = lbase(a, v);
        int lbits = 6;  // slots per CTA: 2^lbits, total >= 2 * deg
        while (((int64_t)kHugeCS << lbits) < 2 * deg) lbits++;
        if (lbits > 12) {  // rows are routed here only up to kHugeDeg
            lbits = 12;
            if (rank == 0 && threadIdx.x == 0) a.ctr->err = kErrTable;
        }
        const int tbits = lbits + 3;  // kHugeCS == 8
        const int T = 1 << lbits;
        const int64_t e0 = deg * rank / kHugeCS, e1 = deg * (rank + 1) / kHugeCS;
        const int64_t span = e1 - e0;
        const int64_t span_r = (span + 31) & ~31ll;  // whole warps for match_any
        for (int64_t eb = threadIdx.x; eb < span_r; eb += kHugeUnroll * kThreads) {
            int32_t u[kHugeUnroll], w[kHugeUnroll], L[kHugeUnroll];
#pragma unroll
            for (int j = 0; j < kHugeUnroll; j++) {
                const int64_t e = eb + j * kThreads;
                u[j] = e < span ? __ldg(&a.g.adjncy[rs + e0 + e]) : -1;
                w[j] = e < span ? __ldg(&a.g.adjwgt[rs + e0 + e]) : 0;
            }
#pragma unroll
            for (int j = 0; j < kHugeUnroll; j++) {
                if (u[j] >= 0 && MODE == kCluster && a.cp && __ldg(&a.cp[u[j]]) != cpv) u[j] = -1;
                L[j] = u[j] >= 0 ? __ldg(&a.lab[u[j]]) : -1;
            }
#pragma unroll
            for (int j = 0; j < kHugeUnroll; j++) {
                if (eb + j * kThreads >= span_r) break;  // warp-uniform
                // merge equal labels within the warp first
                const unsigned peers = __match_any_sync(0xffffffffu, (unsigned)L[j]);
                const unsigned sum = __reduce_add_sync(peers, (unsigned)w[j]);
                if (L[j] >= 0 && (peers & ((1u << lane) - 1)) == 0)
                    huge_insert(cl, sm, (uint32_t)L[j], (int32_t)sum, tbits, lbits);
            }
        }
        cl.sync();
        // this CTA's slots: the largest eligible omega and the own label's sum
        uint32_t mw = 0;
        for (int i = threadIdx.x; i < T; i += kThreads) {
            const uint32_t L = sm.keys[i];
            if (L == kEmpty32) continue;
            const uint32_t w = (uint32_t)sm.vals[i];
            if ((int32_t)L == own) sm.cown = (int32_t)w;
            else if (w > mw && a.W[L] + c <= bnd(a, (int32_t)L)) mw = w;
        }
        mw = __reduce_max_sync(0xffffffffu, mw);
        if (lane == 0) sm.red[threadIdx.x >> 5] = mw;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < kThreads / 32; i++) mw = max(mw, (uint32_t)sm.red[i]);
            sm.cbest = mw;
        }
        cl.sync();
        if (threadIdx.x == 0) {
            uint32_t M = 0;
            int32_t ownw = 0;
            for (unsigned r = 0; r < kHugeCS; r++) {
                const HugeSm *o = cl.map_shared_rank(&sm, r);
                M = max(M, (uint32_t)o->cbest);
                ownw += o->cown;
            }
            sm.b = M;
            sm.bown = ownw;
        }
        __syncthreads();
        const uint32_t M = (uint32_t)sm.b;
        const int32_t ownw = sm.bown;
        const bool ovl = MODE != kCluster && a.W[own] > bnd(a, own);
        const bool prop = M > 0 && ((int32_t)M > ownw || ovl);
        // tie hashes only when the row proposes, only for labels at omega M:
        // the smallest (tie, label) over the cluster wins
        for (int i = threadIdx.x; i < T; i += kThreads) {
            const uint32_t L = sm.keys[i];
            if (L == kEmpty32) continue;
            if (prop && (uint32_t)sm.vals[i] == M && (int32_t)L != own &&
                a.W[L] + c <= bnd(a, (int32_t)L))
                atomicMin(&sm.ctl, ((unsigned long long)tie_of(h, (int32_t)L - lb) << 32) | L);
            sm.keys[i] = kEmpty32;
            sm.vals[i] = 0;
        }
        cl.sync();
        if (rank == 0 && threadIdx.x == 0) {
            record_visit(a, v, (unsigned long long)M << 32, ownw);
            if (prop) {
                unsigned long long tl = ~0ull;
                for (unsigned r = 0; r < kHugeCS; r++) {
                    const unsigned long long x = cl.map_shared_rank(&sm, r)->ctl;
                    tl = x < tl ? x : tl;
                }
                const int32_t L = (int32_t)(uint32_t)tl;
                emit<false>(a, v, L, own, (int32_t)M - ownw, c, ovl, a.W[L]);
            }
        }
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

struct HubFin {
    const int64_t *xadj;
    const int32_t *Lnodes;
    __device__ int64_t operator()(int64_t i) const {
        const int32_t v = Lnodes[i];
        const int64_t d = xadj[v + 1] - xadj[v];
        return d <= kHugeDeg ? 0 : ceil_div<int64_t>(d, kFin);
    }
};

// ---------------------------------------------------------------- large-node lists

struct LargeFlag {
    const int64_t *xadj;
    __device__ int64_t operator()(int64_t v) const { return xadj[v + 1] - xadj[v] > kMedDeg ? 1 : 0; }
};

// Rows longer than the warp path takes (the pipelined lists' capacity).
struct PipeFlag {
    const int64_t *xadj;
    int64_t med_max;
    __device__ int64_t operator()(int64_t v) const { return xadj[v + 1] - xadj[v] > med_max ? 1 : 0; }
};

__global__ void k_large_compact(DGraph g, const int64_t *pos, int32_t *Lnodes) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (g.xadj[v + 1] - g.xadj[v] > kMedDeg) Lnodes[pos[v]] = (int32_t)v;
}

struct LargePieces {
    const int64_t *xadj;
    const int32_t *Lnodes;
    __device__ int64_t operator()(int64_t i) const {
        const int32_t v = Lnodes[i];
        return ceil_div<int64_t>(xadj[v + 1] - xadj[v], kChunk);
    }
};

// Global table slots of a multi-piece row, 2^ceil(log2(2 deg)); single-piece rows: 0.
struct LargeCap {
    const int64_t *xadj;
    const int32_t *Lnodes;
    __device__ int64_t operator()(int64_t i) const {
        const int32_t v = Lnodes[i];
        const int64_t d = xadj[v + 1] - xadj[v];
        if (d <= kHugeDeg) return 0;
        int64_t c = 1;
        while (c < 2 * d) c <<= 1;
        return c;
    }
};

struct LargeDl {
    const int64_t *xadj;
    const int32_t *Lnodes;
    __device__ int64_t operator()(int64_t i) const {
        const int32_t v = Lnodes[i];
        const int64_t d = xadj[v + 1] - xadj[v];
        return d <= kHugeDeg ? 0 : d;
    }
};

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

// Grid of a CTA-row kernel: resident CTAs per SM times SMs (sets its
// dynamic shared memory limit first).
template <int MODE, typename RS>
static int row_grid(int sms) {
    const size_t smem = sizeof(PropSm<MODE, RS>);
    CK(cudaFuncSetAttribute(k_propose<MODE, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_propose<MODE, RS>, RS::kNT, smem));
    return sms * std::max(1, occ);
}

template <int MODE, typename PS>
static int pipe_grid(int sms) {
    const size_t smem = sizeof(PipeSm<MODE, PS>);
    CK(cudaFuncSetAttribute(k_propose_pipe<MODE, PS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_propose_pipe<MODE, PS>, PS::kNT,
                                                     smem));
    return sms * std::max(1, occ);
}

template <int MODE>
static int stage_grid(int sms) {
    const size_t smem = sizeof(StageSm<MODE>);
    CK(cudaFuncSetAttribute(k_propose_stage<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_propose_stage<MODE>, kStNT, smem));
    return sms * std::max(1, occ);
}

struct RowGrids {
    int big, p[kPipeClasses];
};

template <int MODE>
static RowGrids row_grids(int sms) {
    return RowGrids{row_grid<MODE, BigRows>(sms),
                    {pipe_grid<MODE, PipeA>(sms), pipe_grid<MODE, PipeB>(sms),
                     pipe_grid<MODE, PipeC>(sms), stage_grid<MODE>(sms)}};
}

// Rows above kMedDeg: the pipelined kernels of the two shorter classes and
// then the pieces on stream s, the two longer pipelined classes on s2.
// Classes that the tuning's pipelined bound leaves empty are not launched.
template <int MODE>
static void launch_rows(const LPArgs &a, int k, const RowGrids &rg, cudaStream_t s,
                        cudaStream_t s2) {
    const int mid = a.t.mid_max;
    if (mid > 2048) {
        k_propose_stage<MODE><<<rg.p[3], kStNT, sizeof(StageSm<MODE>), s2>>>(a, k);
        LAUNCHED();
    }
    if (mid > 1024) {
        k_propose_pipe<MODE, PipeC>
            <<<rg.p[2], PipeC::kNT, sizeof(PipeSm<MODE, PipeC>), s2>>>(a, k, 2);
        LAUNCHED();
    }
    k_propose_pipe<MODE, PipeA><<<rg.p[0], PipeA::kNT, sizeof(PipeSm<MODE, PipeA>), s>>>(a, k, 0);
    LAUNCHED();
    if (mid > 512) {
        k_propose_pipe<MODE, PipeB>
            <<<rg.p[1], PipeB::kNT, sizeof(PipeSm<MODE, PipeB>), s>>>(a, k, 1);
        LAUNCHED();
    }
    k_propose<MODE, BigRows><<<rg.big, BigRows::kNT, sizeof(PropSm<MODE, BigRows>), s>>>(a, k);
    LAUNCHED();
}

// Degree-ordered sub-rounds (Sec. III.A visits nodes in increasing degree
// when coarsening): in round r the nodes in (degree asc, high 32 bits of
// h(v, r) asc, v asc) order, the node at position p acting in sub-round
// floor(p S / n).  Keys for the stable sort (v order breaks the last ties):
__global__ void k_degree_keys(DGraph g, uint64_t seed, int32_t round, uint64_t *key,
                              int32_t *val) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t d = (uint64_t)(g.xadj[v + 1] - g.xadj[v]);
        key[v] = (d << 32) | (node_hash(seed, round, (uint32_t)v) >> 32);
        val[v] = (int32_t)v;
    }
}

__global__ void k_degree_colours(int64_t n, int S, const int32_t *order, int32_t *col) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        col[order[p]] = (int32_t)(p * S / n);
}

// End of round r: the errors of its sub-rounds are kept, the rounds done
// counted, and the run stops after a full round without moves.
// The counters of the next round (worklist lengths, sub-round counters) are
// cleared here, after this round's error flags are read.
__global__ void k_round_end(const int64_t *moves_r, Ctr *ctr, int S, int32_t *st, int r,
                            int full, int32_t *wl_cnt, int n_wl) {
    if (st[0]) return;
    __shared__ int32_t err;
    if (threadIdx.x == 0) err = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < S; j += blockDim.x) atomicOr(&err, ctr[j].err);
    __syncthreads();
    if (threadIdx.x == 0) {
        st[2] |= err;
        st[1] = r + 1;
        if (*moves_r == 0 && full) st[0] = 1;
    }
    int32_t *cw = reinterpret_cast<int32_t *>(ctr);
    for (int i = threadIdx.x; i < (int)(S * sizeof(Ctr) / sizeof(int32_t)); i += blockDim.x) cw[i] = 0;
    for (int i = threadIdx.x; i < n_wl; i += blockDim.x) wl_cnt[i] = 0;
}

static std::mutex g_tune_mu;
// built-in defaults; the staged class (mid_max 4096) measured slower than
// the CTA-table kernel on R-MAT rows of 2049..4096 entries, so it is opt-in
static Tuning g_tune{kSmallDeg, kMedDeg, 2048, kSegSmem};
Tuning tuning() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}
bool set_tuning(const Tuning &t) {
    const bool ok = (t.small_max == 4 || t.small_max == 8 || t.small_max == 16 ||
                     t.small_max == 32) &&
                    t.med_max >= t.small_max && t.med_max <= kMedDeg &&
                    (t.mid_max == 512 || t.mid_max == 1024 || t.mid_max == 2048 ||
                     t.mid_max == kMidDeg) &&
                    t.seg_smem >= 64 && t.seg_smem <= kSegSmem;
    if (!ok) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = t;
    return true;
}

static std::atomic<int> g_launch_mode{-1};
int launch_mode() { return g_launch_mode.load(); }
int set_launch_mode(int mode) { return g_launch_mode.exchange(mode < -1 ? -1 : mode > 2 ? 2 : mode); }

// Captures what enqueue(cs) puts on a private stream cs (and on the streams
// it forks from cs) into one CUDA graph and launches it after the work already
// on s; s then waits for the graph.  Returns false, with nothing launched, if
// capture or instantiation is refused (the caller then enqueues directly).
template <class F>
static bool run_captured(cudaStream_t s, F &&enqueue) {
    cudaStream_t cs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        try {
            enqueue(cs);
        } catch (...) {
            ok = false;
        }
        const cudaError_t e = cudaStreamEndCapture(cs, &graph);
        ok = ok && e == cudaSuccess && graph != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaGetLastError();  // a refused capture leaves no sticky error
    bool launched = false;
    if (ok) {
        CK(cudaEventRecord(e0, s));
        CK(cudaStreamWaitEvent(cs, e0, 0));
        CK(cudaGraphLaunch(exec, cs));
        count_graph_launch();
        CK(cudaEventRecord(e1, cs));
        CK(cudaStreamWaitEvent(s, e1, 0));
        CK(cudaStreamSynchronize(cs));
        launched = true;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    return launched;
}

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
    if (S < 1 || S > 32) fail(SCLAP_EINVAL, "subrounds");
    const int mode = !cfg.refine ? kCluster : (cfg.nW <= kDenseMaxK ? kRefineDense : kRefineHash);
    const int k = (int)cfg.nW;

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
    a.Bv = cfg.Bv;
    a.nW = cfg.nW;
    a.cp = cfg.refine ? nullptr : cfg.cp;
    a.seed = cfg.seed;
    a.S = S;
    a.run_of = cfg.run_of;
    a.run_seed = cfg.run_seed;
    a.run_off = cfg.run_off;
    a.run_k = cfg.run_k;
    a.vb = cfg.visit_best;
    a.vo = cfg.visit_own;
    // degree-ordered sub-rounds: sort keys, order and colour per node
    uint64_t *dkey = nullptr;
    int32_t *dord = nullptr, *dcol = nullptr;
    int dbits = 0;
    if (cfg.degree_order) {
        if (cfg.run_of) fail(SCLAP_EINVAL, "degree order with batched runs");
        dkey = sc.get<uint64_t>(g.n);
        dord = sc.get<int32_t>(g.n);
        dcol = sc.get<int32_t>(g.n);
        dbits = 32 + std::max(1, bit_width_u64((uint64_t)graph_totals(g, sc).max_deg));
    }
    a.tsum = sc.zeros<int64_t>(cfg.nW);
    a.tcnt = sc.zeros<int32_t>(cfg.nW);
    a.tbase = sc.get<int64_t>(cfg.nW);
    a.ssum = cfg.refine ? sc.zeros<int64_t>(cfg.nW) : nullptr;
    a.props = sc.get<Prop>(g.n);
    a.segs = sc.get<Seg>(g.n);
    a.segbuf = sc.get<SegEntry>(g.n);
    // every big segment holds more than seg_smem of the <= n proposals
    a.t = tuning();
    a.maxbig = (int32_t)std::min<int64_t>(g.n / (a.t.seg_smem + 1) + 1, cfg.nW);
    a.maxtiles = (int32_t)(g.n / kBigTile + a.maxbig + 1);
    a.big = sc.get<BigSeg>(a.maxbig);
    a.tileseg = sc.get<int32_t>(a.maxtiles);
    a.bhist = sc.zeros<unsigned long long>((size_t)a.maxbig * kBins);
    a.bar = sc.zeros<GridBar>(1);
    a.bar_cycles = kBarCycles;
    int32_t *wl = sc.get<int32_t>((size_t)kClasses * S * g.n);
    // bucket lengths, then piece counts, then cluster-path row counts (per colour)
    const int n_wl = kClasses * S + (2 + kPipeClasses) * S;
    int32_t *wl_cnt = sc.get<int32_t>(n_wl);
    Ctr *ctr = sc.get<Ctr>(S);
    int64_t *d_moves = sc.zeros<int64_t>(cfg.rounds);
    a.wl = wl;
    a.wl_cnt = wl_cnt;
    a.pcnt = wl_cnt + kClasses * S;
    a.hcnt = wl_cnt + kClasses * S + S;
    for (int q = 0; q < kPipeClasses; q++) a.pc[q] = wl_cnt + kClasses * S + (2 + q) * S;
    a.huge_on = mode != kRefineDense;
    a.prof = prof().on ? prof().d_counts : nullptr;

    // nodes of degree > kMedDeg: one list per call, cut into kChunk pieces
    int64_t hub_items = 0;
    {
        int64_t *pos = sc.get<int64_t>(g.n);
        int64_t *d_nL = sc.get<int64_t>(1);
        exclusive_scan(LargeFlag{g.xadj}, g.n, pos, d_nL, sc);
        int64_t nL = 0;
        CK(cudaMemcpyAsync(&nL, d_nL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        a.nL = nL;
        // pipelined lists: room for every row above med_max (the large rows
        // when med_max is kMedDeg)
        int64_t nP = nL;
        if (a.t.med_max < kMedDeg) {
            int64_t *ppos = sc.get<int64_t>(g.n);
            int64_t *d_nP = sc.get<int64_t>(1);
            exclusive_scan(PipeFlag{g.xadj, a.t.med_max}, g.n, ppos, d_nP, sc);
            CK(cudaMemcpyAsync(&nP, d_nP, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
        a.nP = nP;
        if (nP > 0)
            for (int q = 0; q < kPipeClasses; q++) a.pl[q] = sc.get<int32_t>((size_t)S * nP);
        if (nL > 0) {
            int32_t *Lnodes = sc.get<int32_t>(nL);
            k_large_compact<<<sms * 4, 256, 0, s>>>(g, pos, Lnodes);
            LAUNCHED();
            int64_t *Lpre = sc.get<int64_t>(nL + 1);
            exclusive_scan(LargePieces{g.xadj, Lnodes}, nL, Lpre, Lpre + nL, sc);
            a.Lnodes = Lnodes;
            a.Lpre = Lpre;
            CK(cudaMemcpyAsync(&a.Ptot, Lpre + nL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            a.plist = sc.get<int64_t>((size_t)S * (a.Ptot ? a.Ptot : 1));
            a.hlist = sc.get<int32_t>((size_t)S * nL);

            a.Ldone = sc.zeros<int32_t>(nL);
            a.Lndl = sc.zeros<int32_t>(nL);
            if (mode == kRefineDense) {
                a.gacc = sc.zeros<int32_t>((size_t)nL * k);
            } else {
                int64_t *Loff = sc.get<int64_t>(nL + 1);
                int64_t *Ldlo = sc.get<int64_t>(nL + 1);
                exclusive_scan(LargeCap{g.xadj, Lnodes}, nL, Loff, Loff + nL, sc);
                exclusive_scan(LargeDl{g.xadj, Lnodes}, nL, Ldlo, Ldlo + nL, sc);
                int64_t tot[2];
                CK(cudaMemcpyAsync(&tot[0], Loff + nL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                CK(cudaMemcpyAsync(&tot[1], Ldlo + nL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                a.Loff = Loff;
                a.Ldlo = Ldlo;
                int64_t *Hfin = sc.get<int64_t>(nL + 1);
                exclusive_scan(HubFin{g.xadj, Lnodes}, nL, Hfin, Hfin + nL, sc);
                CK(cudaMemcpyAsync(&hub_items, Hfin + nL, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                a.Hfin = Hfin;
                a.hbest = sc.zeros<unsigned long long>(nL);
                a.hown = sc.zeros<int32_t>(nL);
                a.htl = sc.get<unsigned long long>(nL);
                CK(cudaMemsetAsync(a.htl, 0xff, nL * sizeof(unsigned long long), s));
                LAUNCHED();
                a.gkeys = sc.get<unsigned long long>(tot[0]);
                a.gvals = sc.zeros<int32_t>(tot[0]);
                a.gdl = sc.get<int32_t>(tot[1]);
                if (tot[0]) CK(cudaMemsetAsync(a.gkeys, 0xff, tot[0] * sizeof(uint64_t), s));
                CK(cudaStreamSynchronize(s));
            }
        }
    }

    RowGrids rgrids{};
    switch (mode) {
        case kCluster: rgrids = row_grids<kCluster>(sms); break;
        case kRefineHash: rgrids = row_grids<kRefineHash>(sms); break;
        default: rgrids = row_grids<kRefineDense>(sms); break;
    }
    CK(cudaFuncSetAttribute(k_arbitrate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sizeof(ArbSm)));
    // the occupancy below assumes the largest shared-memory carveout
    CK(cudaFuncSetAttribute(k_arbitrate, cudaFuncAttributePreferredSharedMemoryCarveout,
                            (int)cudaSharedmemCarveoutMaxShared));
    const int grid_small = sms * 4;
    int occ_arb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_arb, k_arbitrate, kThreads,
                                                     sizeof(ArbSm)));
    if (occ_arb < 1) fail(SCLAP_ECUDA, "arbitration kernel does not fit on an SM");
    const int grid_arb = sms * std::min(occ_arb, 4);

    cudaStream_t side, side2;
    CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&side2, cudaStreamNonBlocking));
    cudaEvent_t ev_fork, ev_join, ev_join2;
    CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_join2, cudaEventDisableTiming));
    const bool huge = a.huge_on && a.nL > 0;
    const int grid_huge = std::max(kHugeCS, (sms * 4) / kHugeCS * kHugeCS);
    int occ_small = 0;
    switch (mode) {
        case kCluster: CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_small, k_propose_small<kCluster>, kThreads, 0)); break;
        case kRefineHash: CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_small, k_propose_small<kRefineHash>, kThreads, 0)); break;
        default: CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_small, k_propose_small<kRefineDense>, kThreads, 0)); break;
    }
    const int grid_sm = sms * std::max(1, occ_small);

    // Round r: worklists, then S sub-rounds of propose (fork-join over three
    // streams) and arbitration, then the end-of-round test on the device.
    int32_t *d_state = sc.zeros<int32_t>(3);  // [0] stop flag, [1] rounds done, [2] errors
    auto enqueue_round = [&](int r, bool full, cudaStream_t ms) {
        a.round = r;
        a.moves = d_moves + r;
        if (cfg.degree_order) {  // this round's sub-round of every node (stream ms == s)
            k_degree_keys<<<sms * 4, 256, 0, ms>>>(g, cfg.seed, r, dkey, dord);
            LAUNCHED();
            radix_sort_pairs(dkey, dord, g.n, dbits, sc);
            k_degree_colours<<<sms * 4, 256, 0, ms>>>(g.n, S, dord, dcol);
            LAUNCHED();
            a.col = dcol;
        }
        if (r == 0) {  // later rounds: cleared by the previous round's k_round_end
            CK(cudaMemsetAsync(wl_cnt, 0, n_wl * sizeof(int32_t), ms));
            CK(cudaMemsetAsync(ctr, 0, S * sizeof(Ctr), ms));
        }
        k_build_wl<<<sms * 4, kThreads, 0, ms>>>(a, wl, wl_cnt);
        LAUNCHED();
        for (int j = 0; j < S; j++) {
            a.ctr = ctr + j;
            a.colour = j;
            cudaEvent_t pb, pe;
            prof_begin(ms, &pb, &pe);
            // small rows on the side stream, next to the large and medium rows
            CK(cudaEventRecord(ev_fork, ms));
            CK(cudaStreamWaitEvent(side, ev_fork, 0));
            switch (mode) {
                case kCluster: k_propose_small<kCluster><<<grid_sm, kThreads, 0, side>>>(a, k); break;
                case kRefineHash: k_propose_small<kRefineHash><<<grid_sm, kThreads, 0, side>>>(a, k); break;
                default: k_propose_small<kRefineDense><<<grid_sm, kThreads, 0, side>>>(a, k); break;
            }
            LAUNCHED();
            CK(cudaEventRecord(ev_join, side));
            if (a.nP > 0) {
                // rows of one CTA cluster and the 256-thread pipelined
                // rows on a second side stream
                CK(cudaStreamWaitEvent(side2, ev_fork, 0));
                if (huge) {
                    if (mode == kCluster)
                        k_propose_huge<kCluster><<<grid_huge, kThreads, 0, side2>>>(a);
                    else
                        k_propose_huge<kRefineHash><<<grid_huge, kThreads, 0, side2>>>(a);
                    LAUNCHED();
                }
                switch (mode) {
                    case kCluster: launch_rows<kCluster>(a, k, rgrids, ms, side2); break;
                    case kRefineHash: launch_rows<kRefineHash>(a, k, rgrids, ms, side2); break;
                    default: launch_rows<kRefineDense>(a, k, rgrids, ms, side2); break;
                }
                CK(cudaEventRecord(ev_join2, side2));
            }
            CK(cudaStreamWaitEvent(ms, ev_join, 0));
            if (a.nP > 0) CK(cudaStreamWaitEvent(ms, ev_join2, 0));
            prof_end(ms, pb, pe);
            if (hub_items > 0) {
                const int hg = (int)std::min<int64_t>(hub_items, (int64_t)sms * 8);
                switch (mode) {
                    case kCluster:
                        k_hub_cand<kCluster><<<hg, kThreads, 0, ms>>>(a);
                        k_hub_tie<kCluster><<<hg, kThreads, 0, ms>>>(a);
                        k_hub_emit<kCluster><<<sms, kThreads, 0, ms>>>(a);
                        break;
                    default:
                        k_hub_cand<kRefineHash><<<hg, kThreads, 0, ms>>>(a);
                        k_hub_tie<kRefineHash><<<hg, kThreads, 0, ms>>>(a);
                        k_hub_emit<kRefineHash><<<sms, kThreads, 0, ms>>>(a);
                        break;
                }
                LAUNCHED();
                LAUNCHED();
                LAUNCHED();
            }
            if (cfg.refine) {
                k_src<<<(unsigned)(cfg.nW + grid_small), kThreads, 0, ms>>>(a);
                LAUNCHED();
            }
            {
                // cooperative: every CTA resident (the grid barrier needs it),
                // also as a node of a captured graph
                cudaLaunchConfig_t lc = {};
                lc.gridDim = dim3(grid_arb);
                lc.blockDim = dim3(kThreads);
                lc.dynamicSmemBytes = sizeof(ArbSm);
                lc.stream = ms;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeCooperative;
                at[0].val.cooperative = 1;
                lc.attrs = at;
                lc.numAttrs = 1;
                CK(cudaLaunchKernelEx(&lc, k_arbitrate, a));
            }
            LAUNCHED();
        }
        k_round_end<<<1, 128, 0, ms>>>(d_moves + r, ctr, S, d_state, r, full ? 1 : 0, wl_cnt,
                                       n_wl);
        LAUNCHED();
    };

    int done = 0;
    try {
        // degree-ordered rounds sort on the call's stream: one round at a time
        const int lm = cfg.degree_order ? 0
                       : launch_mode() >= 0 ? launch_mode() : (cfg.prefer_capture ? 2 : 0);
        if (cfg.before_round || lm == 0) {
            // one round at a time, the host testing the stop rule after each
            // (always for learned refinement: the host prepares every round's
            // features and gate)
            for (int r = 0; r < cfg.rounds; r++) {
                const uint8_t *act = nullptr;
                const bool full = cfg.before_round ? cfg.before_round(r, &act) : true;
                a.active = act;
                enqueue_round(r, full, s);
                int64_t hmoves = 0;
                CK(cudaMemcpyAsync(&hmoves, d_moves + r, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                done = r + 1;
                if (hmoves == 0 && full) break;
            }
        } else {
            // every round is enqueued ahead: a round without moves sets the
            // stop flag and the kernels of later rounds return at once.  The
            // rounds are captured in one CUDA graph when capture is on (and
            // profiling, which times propose steps with events, is off).
            a.stop = d_state;
            bool ran = false;
            if (lm == 2 && !prof().on)
                ran = run_captured(s, [&](cudaStream_t cs) {
                    for (int r = 0; r < cfg.rounds; r++) enqueue_round(r, true, cs);
                });
            if (!ran)
                for (int r = 0; r < cfg.rounds; r++) enqueue_round(r, true, s);
        }
        int32_t hs[3] = {0, 0, 0};
        CK(cudaMemcpyAsync(hs, d_state, sizeof(hs), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!cfg.before_round && lm != 0) done = hs[1];
        if (hs[2] & kErrTable) fail(SCLAP_ECUDA, "hash table overflow");
        if (hs[2] & kErrBarrier) fail(SCLAP_ETIMEOUT, "grid barrier timed out in arbitration");
        if (hs[2] & kErrBig) fail(SCLAP_ECUDA, "long-segment capacity exceeded");
        if (moves_out && done > 0) {
            moves_out->resize(done);
            CK(cudaMemcpyAsync(moves_out->data(), d_moves, done * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
        }
    } catch (...) {
        cudaStreamSynchronize(side);
        cudaStreamSynchronize(side2);
        cudaEventDestroy(ev_fork);
        cudaEventDestroy(ev_join);
        cudaEventDestroy(ev_join2);
        cudaStreamDestroy(side);
        cudaStreamDestroy(side2);
        throw;
    }
    CK(cudaStreamSynchronize(side));
    CK(cudaStreamSynchronize(side2));
    CK(cudaEventDestroy(ev_fork));
    CK(cudaEventDestroy(ev_join));
    CK(cudaEventDestroy(ev_join2));
    CK(cudaStreamDestroy(side));
    CK(cudaStreamDestroy(side2));
    return done;
}

int barrier_selftest(long long limit_cycles, Scratch &sc) {
    cudaStream_t s = sc.stream();
    GridBar *bar = sc.zeros<GridBar>(1);
    int32_t *err = sc.zeros<int32_t>(1);
    k_barrier_selftest<<<2, 32, 0, s>>>(bar, err, limit_cycles);
    LAUNCHED();
    int32_t h = 0;
    CK(cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return (h & kErrBarrier) ? SCLAP_ETIMEOUT : SCLAP_OK;
}

}  // namespace sclap
