/*
 * sclap.h -- C ABI of libsclap: size-constrained label propagation (SCLaP),
 * cluster contraction, projection and the multilevel driver on one NVIDIA
 * GB300 GPU (sm_103a).
 *
 * Method: Meyerhenke, Sanders, Schulz, "Parallel Graph Partitioning for
 * Complex Networks" (2014).  Problem statement (Sec. II.A): an undirected
 * graph G = (V, E, c, omega) with node weights c >= 0 and edge weights
 * omega > 0; k blocks with c(V_i) <= L_max := (1+eps) * ceil(c(V)/k); the
 * objective is the total weight of cut edges.  A size-constrained clustering
 * bounds every cluster by U (Sec. II.A, Sec. III.A).
 *
 * Deterministic reading used by every entry point (the paper visits nodes
 * sequentially in random order and breaks ties randomly):
 *  - mix64 is the SplitMix64 output function; h(v, r) = mix64(seed ^
 *    ((r + 1) << 32) ^ v) for round r.
 *  - Every round has S synchronous sub-rounds; node v acts in sub-round
 *    (h(v, r) >> 32) mod S and proposes against the state at the start of
 *    that sub-round.
 *  - v's candidates are its neighbours' labels other than its own; label L
 *    is eligible iff W(L) + c(v) <= B (B = U when clustering, L_max when
 *    refining).  The best candidate maximises omega(v, L), then minimises
 *    tie = high 32 bits of mix64(h(v, r) ^ L), then L.  v proposes iff
 *    omega(v, best) - omega(v, own) > 0, or when refining iff its own block
 *    is overloaded (Sec. III.A, last paragraph).
 *  - Departures from an overloaded block are admitted in (gain desc, id asc)
 *    order while the weight already departed is below the excess.  Then each
 *    target T admits its proposals in (gain desc, id asc) order iff c(v) == 0
 *    or the inclusive prefix of c is <= B - W(T).  Admitted moves are applied
 *    together.  A run stops after `rounds` rounds or after a round without
 *    moves.
 *
 * Graph layout (CSR, both directions of every edge stored):
 *   xadj   int64 [n+1]  row offsets, xadj[0] = 0, non-decreasing
 *   adjncy int32 [nnz]  neighbour ids; every row strictly ascending, no
 *                       self-loops
 *   adjwgt int32 [nnz]  omega > 0, symmetric
 *   vwgt   int32 [n]    c >= 0
 * Arrays are device pointers unless an entry point says otherwise; inputs are
 * read-only and caller-owned.  Output arrays are caller-allocated device
 * memory of the stated size; scalar outputs are host pointers (NULL allowed)
 * and are valid when the call returns.  All work is enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and every entry point
 * synchronises that stream before it returns.
 *
 * Errors: every entry point returns SCLAP_OK or one of the codes below; on
 * error no output is valid and `part_inout` arguments are restored.
 */
#ifndef SCLAP_H
#define SCLAP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sclap_status {
    SCLAP_OK = 0,
    SCLAP_EINVAL = 1,     /* bad scalar argument (k < 1, eps < 0, U < max c, ...)   */
    SCLAP_EGRAPH = 2,     /* graph fails validation                                  */
    SCLAP_EOVERFLOW = 3,  /* c(V) or the undirected sum of omega exceeds INT32_MAX   */
    SCLAP_ENOMEM = 4,     /* device allocation failed                                */
    SCLAP_ECUDA = 5,      /* CUDA runtime error                                      */
    SCLAP_ETIMEOUT = 6,   /* a bounded device wait gave up                           */
    SCLAP_ENOTIMPL = 7
};

typedef struct {
    int64_t n, nnz;               /* nodes; nnz = 2m directed entries            */
    const int64_t *xadj;          /* [n+1]                                       */
    const int32_t *adjncy;        /* [nnz]                                       */
    const int32_t *adjwgt;        /* [nnz]                                       */
    const int32_t *vwgt;          /* [n]                                         */
} sclap_graph;

/* A graph whose arrays the library allocated (device memory); release it with
 * sclap_graph_free. */
typedef struct {
    int64_t n, nnz;
    int64_t *xadj;
    int32_t *adjncy, *adjwgt, *vwgt;
} sclap_graph_owned;

/* Multilevel parameters (Sec. IV.E).  sclap_ml_defaults fills the paper's
 * `fast` round counts (l = 3, r = 6, Sec. V.A) with S = 4, n_stop = 2000. */
typedef struct {
    int32_t k;              /* blocks                                            */
    double eps;             /* imbalance                                         */
    int64_t U;              /* cluster bound; <= 0: max(max c(v), c(V)/(10k))    */
    int32_t cluster_rounds; /* l: SCLaP rounds per coarsening level              */
    int32_t refine_rounds;  /* r: SCLaP rounds per uncoarsening level            */
    int32_t subrounds;      /* S                                                 */
    int64_t n_stop;         /* coarsen while the current level has >= n_stop nodes */
    int32_t max_levels;     /* hierarchy depth cap (<= 64; <= 0: 32)             */
    int32_t init_seeds;     /* P individuals in the initial partition           */
    int32_t init_rounds;    /* refinement rounds inside the initial partition   */
    uint64_t seed;
    int32_t degree_order;   /* 1: coarsening in degree-ordered sub-rounds (see
                               sclap_cluster_degree_ordered); 0: by hash       */
} sclap_ml_params;

#define SCLAP_MAX_LEVELS 64
typedef struct {
    int32_t levels;                            /* graphs in the hierarchy        */
    int64_t n[SCLAP_MAX_LEVELS];
    int64_t nnz[SCLAP_MAX_LEVELS];
    int32_t cluster_rounds_done[SCLAP_MAX_LEVELS];
    int32_t refine_rounds_done[SCLAP_MAX_LEVELS];
    int64_t U, lmax;
    int32_t init_best;                         /* chosen individual              */
    int64_t init_cut, init_maxbw;
    int64_t cut, maxbw;                        /* final partition               */
} sclap_ml_stats;

/* Size-constrained clustering, Sec. III.A ("label propagation with size
 * constraints") and Sec. IV.A-B.  Every node starts in its own cluster
 * (label = id); afterwards every cluster weight is <= U.
 *   U               >= max_v c(v), else SCLAP_EINVAL
 *   rounds (l)      >= 0;  subrounds (S) >= 1
 *   constraint_part NULL, or device int32[n]: clusters stay inside the blocks
 *                   of this partition (iterated V-cycles, Sec. IV.D)
 *   labels_out      device int32[n]: cluster id (a node id) per node
 * Nodes without neighbours never move; after the rounds they are packed in id
 * order (per block of constraint_part) into clusters: with U' = U - cmax + 1
 * (cmax: their largest weight) and P(v) the weight of the earlier ones, v
 * joins group floor(P(v) / U') labelled by its smallest id (weight <= U).
 *   rounds_done     host, rounds executed (the last one may have 0 moves)
 * Needs c(V) <= INT32_MAX and sum(adjwgt) / 2 (the undirected total) <=
 * INT32_MAX (SCLAP_EOVERFLOW). */
int sclap_cluster(const sclap_graph *g, int64_t U, int32_t rounds, int32_t subrounds,
                  uint64_t seed, const int32_t *constraint_part, int32_t *labels_out,
                  int32_t *rounds_done, void *stream);

/* sclap_cluster with degree-ordered sub-rounds, the synchronous counterpart
 * of the paper's traversal in increasing degree while coarsening (Sec.
 * III.A): in round r the nodes are ordered by (degree asc, high 32 bits of
 * h(v, r) asc, v asc) and the node at position p acts in sub-round
 * floor(p S / n) (S groups whose sizes differ by at most one, low degrees
 * first).  Tie-breaks still use h(v, r).  With S = 1 it equals
 * sclap_cluster.  Same arguments and errors as sclap_cluster. */
int sclap_cluster_degree_ordered(const sclap_graph *g, int64_t U, int32_t rounds,
                                 int32_t subrounds, uint64_t seed,
                                 const int32_t *constraint_part, int32_t *labels_out,
                                 int32_t *rounds_done, void *stream);

/* SCLaP as local search on a k-partition, Sec. III.A (bound L_max, the
 * overloaded-block rule) and Sec. IV.B (exact block weights).
 *   part_inout  device int32[n], values in [0, k); refined in place
 *   cut_out     host int64: cut of the result (Sec. II.A)
 *   block_w_out host int64[k]: block weights of the result
 * Needs every weighted degree <= INT32_MAX (SCLAP_EOVERFLOW). */
int sclap_refine(const sclap_graph *g, int32_t k, double eps, int32_t rounds,
                 int32_t subrounds, uint64_t seed, int32_t *part_inout, int64_t *cut_out,
                 int64_t *block_w_out, int32_t *rounds_done, void *stream);

/* Same as sclap_refine with an explicit bound B on every one of `nblocks`
 * blocks (used for batched runs over disjoint unions of graphs). */
int sclap_refine_bound(const sclap_graph *g, int32_t nblocks, int64_t B, int32_t rounds,
                       int32_t subrounds, uint64_t seed, int32_t *part_inout,
                       int32_t *rounds_done, void *stream);

/* Cluster contraction, Sec. III ("contracting a clustering") and Sec. IV.C:
 * coarse id q(L) = rank of L among the distinct labels (ascending), f2c(v) =
 * q(label(v)); coarse node weight = cluster weight; coarse edge weight = sum
 * of omega between the two clusters; intra-cluster edges dropped.  Output is
 * canonical: rows ascending, neighbours strictly ascending, symmetric.
 *   labels      device int32[n], values in [0, n)
 *   coarse_out  filled with library-allocated device arrays (free with
 *               sclap_graph_free)
 *   f2c_out     device int32[n] */
int contract_graph(const sclap_graph *g, const int32_t *labels, sclap_graph_owned *coarse_out,
                   int32_t *f2c_out, void *stream);

/* Uncoarsening, Sec. III and Sec. IV.C: fine_part_out[v] = coarse_part[f2c[v]].
 * All three arrays are device memory; no validation beyond n_fine >= 0. */
int project_partition(int64_t n_fine, const int32_t *f2c, const int32_t *coarse_part,
                      int32_t *fine_part_out, void *stream);

/* Cut (Sec. II.A) and block weights of a partition.  The graph is validated
 * like every other entry point's (SCLAP_EGRAPH; see sclap_set_validation).
 *   part        device int32[n] in [0, k); any other id returns SCLAP_EINVAL
 *   cut_out     host int64;  block_w_out host int64[k] (NULL allowed) */
int sclap_cut(const sclap_graph *g, const int32_t *part, int32_t k, int64_t *cut_out,
              int64_t *block_w_out, void *stream);

/* Cut and block weights like sclap_cut, without allocating any memory.  The
 * paper has no counterpart: this exists for callers that cannot let a library
 * allocate device memory, such as loops with a latency budget (cudaMalloc and
 * cudaFree can synchronise the whole device) and programs whose device memory
 * is handed out by their own pool or allocator.  Its accumulators are a
 * file-scope device array of 2 + 65536 int64 values, held by every GPU that
 * loads the library until the process exits; k > 65536 returns SCLAP_EINVAL.
 * The first call on a device looks up that array's device address.  All calls
 * share the array and clear the part they use; calls that overlap on the GPU
 * race.  Same arguments and outputs as sclap_cut; a block id outside [0, k)
 * returns SCLAP_EINVAL (such ids are skipped on the device, never written);
 * no other graph validation. */
int sclap_cut_noalloc(const sclap_graph *g, const int32_t *part, int32_t k, int64_t *cut_out,
                      int64_t *block_w_out, void *stream);

/* Initial partition of a (coarsest) graph; stands in for the paper's
 * evolutionary initial partitioner (Sec. II.C, Sec. IV.E).  P independent
 * individuals: the batched runs of sclap_refine_batched on this graph (bound
 * B on every block) with seeds s_t = mix64(seed ^ (0xD1B54A32D192ED03 *
 * (t + 1))), t = 0..P-1.
 * Best = lowest cut with max block <= B (lowest t on ties), else smallest
 * max block, then cut, then t.
 *   part_out  device int32[n];  cuts_out, maxbw_out host int64[P] (NULL ok);
 *   best_out  host int32 */
int sclap_initial_partition(const sclap_graph *g, int32_t k, int64_t B, int32_t P,
                            int32_t rounds, int32_t subrounds, uint64_t seed,
                            int32_t *part_out, int64_t *cuts_out, int64_t *maxbw_out,
                            int32_t *best_out, void *stream);

/* ---- learned active set (a gate over refinement rounds; the paper has no
 * counterpart: its refinement visits every node, Sec. III.A) ----
 *
 * The scorer is a 6-32-32-1 network of 1313 parameters in this order:
 * W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3 (row-major, output index
 * first).  Inference takes them as bf16 bit patterns; training as float.
 * Features of node v before a round (each rounded to bf16, nearest even),
 * with wdeg its weighted degree and wb / wo the weight to the best eligible
 * other block / to its own block that v's latest visit in this call saw
 * (recorded by the propose step; 0 before the first visit):
 *   1 e + (x - 2^e) / 2^e for x = 1 + deg(v), e = floor(log2 x)
 *   2 W(own) / L_max
 *   3 (wb - wo) / wdeg, the best external gain
 *   4 1 if v moved in the previous round
 *   5 moved neighbours in the previous round / deg(v)
 *   6 wo / wdeg
 * (zeros for nodes without neighbours).  Every output starts from its bias
 * and adds one fmaf per input in index order (float accumulator); hidden
 * outputs pass ReLU and are rounded to bf16; the last output is the logit. */

/* Refinement (as sclap_refine) where a gated round visits only the nodes
 * whose logit is >= z_min; round r is full (every node) when r == 0, when
 * r % full_every == full_every - 1, when r is the last round, or always when
 * net is NULL (then the call equals sclap_refine).  A run stops after a full
 * round without moves.  A gated round reads no edges beyond the rows it
 * visits and those of the nodes that moved in the round before.
 *   net          device uint16[1313] bf16 parameters, or NULL
 *   visited_out  host: nodes with neighbours visited, summed over rounds (NULL ok)
 *   trace_x      device float[rounds][n][6]: the features before each round (NULL ok)
 *   trace_y      device uint8[rounds][n]: 1 if the node moved in that round (NULL ok)
 * Rows of the traces past *rounds_done are left untouched.  Errors as
 * sclap_refine (EINVAL also for full_every < 1); part_inout is restored. */
int sclap_refine_learned(const sclap_graph *g, int32_t k, double eps, int32_t rounds,
                         int32_t subrounds, uint64_t seed, const uint16_t *net, float z_min,
                         int32_t full_every, int32_t *part_inout, int64_t *cut_out,
                         int64_t *block_w_out, int32_t *rounds_done, int64_t *visited_out,
                         float *trace_x, uint8_t *trace_y, void *stream);

/* Logits of N feature rows x (device float[N][6]) with the bf16 network net
 * (device uint16[1313]) into z_out (device float[N]). */
int sclap_mlp_score(const float *x, int64_t N, const uint16_t *net, float *z_out, void *stream);

/* Mean logistic loss log(1 + e^z) - y z over N samples (x device float[N][6],
 * y device uint8[N]) and its gradient (device float[1313], overwritten) with
 * respect to the float parameters params (device float[1313]); *loss_out on
 * the host.  bf16_in = 0: z is the float network's logit.  bf16_in = 1
 * (BF16-in / FP32-accumulate, what training uses): z is the logit inference
 * computes (parameters rounded to bf16, hidden outputs ReLU then bf16, fp32
 * fmaf accumulation in index order), and the gradient is the straight-through
 * one (each rounding passed as the identity).  Summation order not fixed. */
int sclap_mlp_loss_grad(const float *x, const uint8_t *y, int64_t N, const float *params,
                        int32_t bf16_in, float *grad_out, double *loss_out, void *stream);

/* Plain minibatch SGD on the BF16-in loss above (bf16_in = 1; float master
 * parameters): `epochs` passes over the samples in an order shuffled per
 * epoch (sort by SplitMix64 of seed, epoch and index), batches of `batch`,
 * params -= lr * gradient after each.  *loss_out: the BF16-in loss over all
 * samples after training.  1 <= N <= INT32_MAX. */
int sclap_mlp_train(const float *x, const uint8_t *y, int64_t N, float *params, int32_t epochs,
                    int32_t batch, float lr, uint64_t seed, double *loss_out, void *stream);

/* The bf16 network of trained float parameters: net_out[i] = the bf16 bit
 * pattern of params[i] rounded to nearest, ties to even (the same rounding as
 * the features and hidden outputs).  params device float[1313], net_out
 * device uint16[1313]. */
int sclap_mlp_pack_bf16(const float *params, uint16_t *net_out, void *stream);

/* A set of graphs for batched runs (host array of graph views). */
typedef struct {
    int32_t ngraphs;
    const sclap_graph *graphs;
} sclap_batch;

/* Batched SCLaP population: many seeded runs on uneven graphs at once, the
 * stand-in for the paper's population-based initial partitioning of the
 * coarsest graph (Sec. II.C, Sec. IV.E), whose individuals are independent.
 * Run r works on graph run_graph[r] with seed s_r = seeds[r] and k blocks
 * bounded by that graph's L_max = (1+eps) ceil(c(V)/k) (Sec. II.A): it places
 * the nodes in (c desc, h_r(v) asc, v asc) order into the currently lightest
 * block (lowest id on ties), h_r(v) = high 32 bits of mix64(s_r ^ v); then
 * all runs are refined together for `rounds` rounds as one SCLaP refinement
 * over the disjoint union of the runs' graphs, each run's sub-rounds and
 * tie-breaks keyed by s_r with its own node and block ids.  A run's result is
 * therefore the same in any batch and at any position: that start refined by
 * sclap_refine_bound on its graph alone with seed s_r.
 *   run_graph  host int32[nruns], graph index per run
 *   seeds      host uint64[nruns], seed per run
 *   parts_out  device int32[sum of the runs' n], per-run block ids 0..k-1,
 *              concatenated in run order
 *   cuts_out, maxbw_out  host int64[nruns] (NULL allowed)
 * The rounds run as sclap_set_launch_mode says (by default all of them from
 * one captured CUDA graph, launched once).  Needs c(V) <= INT32_MAX per graph and every
 * weighted degree <= INT32_MAX. */
int sclap_refine_batched(const sclap_batch *b, int32_t k, double eps, int32_t rounds,
                         int32_t subrounds, int32_t nruns, const int32_t *run_graph,
                         const uint64_t *seeds, int32_t *parts_out, int64_t *cuts_out,
                         int64_t *maxbw_out, void *stream);

/* The multilevel partitioner, Sec. IV.E: l rounds of clustering and a
 * contraction per level while n >= n_stop (stop also when a level shrinks by
 * less than 5%, when it does not shrink at all, or at max_levels); the
 * initial partition above on the coarsest graph with level seed; then per
 * finer level projection and r rounds of refinement.  Level l uses seed
 * s_l = mix64(seed ^ (0x9E3779B97F4A7C15 * (l + 1))) for both forms.
 *   g         graph arrays may be HOST or DEVICE memory (detected per call;
 *             host arrays are copied to the device inside the call)
 *   part_out  int32[n], host or device (detected), block per node
 *   stats_out host, may be NULL */
int partition_multilevel(const sclap_graph *g, const sclap_ml_params *p, int32_t *part_out,
                         sclap_ml_stats *stats_out, void *stream);

/* One iterated V-cycle (Sec. IV.E: the fast preset runs two cycles, the
 * minimal one a single cycle): the multilevel scheme above seeded by the
 * partition part_inout (k blocks).  Every clustering is restricted to the
 * blocks of that partition (Sec. III.A's constraint; nodes without
 * neighbours are packed per block), each coarse node inherits its members'
 * block, and the coarsest graph's inherited partition, refined with
 * init_rounds rounds, is the initial partition (stats: init_best = -1,
 * init_cut / init_maxbw of that partition after refinement).  With zero
 * refinement rounds the call returns its input.
 *   part_inout  int32[n], host or device (detected): in, the seed partition;
 *               out, the new one
 * EINVAL when a block id is outside 0..k-1; other errors as
 * partition_multilevel. */
int sclap_vcycle(const sclap_graph *g, const sclap_ml_params *p, int32_t *part_inout,
                 sclap_ml_stats *stats_out, void *stream);

void sclap_ml_defaults(sclap_ml_params *p, int32_t k, double eps, uint64_t seed);

/* Failure detection of the library's only in-kernel wait (the paper has no
 * counterpart): the grid barrier of the arbitration kernel gives up after a
 * bounded number of SM clock cycles, sets an error flag and returns, and the
 * calling entry point reports SCLAP_ETIMEOUT.  This runs that barrier in a
 * two-CTA launch where one CTA never arrives, with the bound limit_cycles
 * (>= 0): the wait must run out.  Returns SCLAP_ETIMEOUT when it did and was
 * reported (the expected result), SCLAP_OK if the barrier did not time out,
 * other codes on CUDA errors.  Uses the legacy default stream. */
int sclap_wait_selftest(int64_t limit_cycles);

/* Failure detection of device allocations (the paper has no counterpart):
 * the library's scratch allocations are counted from this call on, and the
 * one that finds the count at `after` (>= 0) fails as if the device were out
 * of memory, so that call returns SCLAP_ENOMEM (with part_inout restored
 * where the entry point documents it); after == -1 turns the injection off.
 * Process-wide; meant for tests.  SCLAP_EINVAL for after < -1. */
int sclap_inject_alloc_failure(int64_t after);

/* Copies a library-owned graph into caller-allocated device arrays of sizes
 * n+1, nnz, nnz and n (enqueued on `stream`, synchronised before return). */
int sclap_graph_copy_out(const sclap_graph_owned *g, int64_t *xadj, int32_t *adjncy,
                         int32_t *adjwgt, int32_t *vwgt, void *stream);

/* Releases the arrays of a graph returned by contract_graph. */
void sclap_graph_free(sclap_graph_owned *g);

const char *sclap_strerror(int code);

/* Graph validation on entry (on by default): monotone xadj, ids in range, rows
 * strictly ascending (hence no duplicates), no self-loops, symmetric equal
 * weights, omega > 0, c >= 0.  Returns the previous setting. */
int sclap_set_validation(int on);

/* How the SCLaP rounds of a call are launched (no effect on results):
 *   0  one round at a time; the host reads the round's move count and stops
 *      the run after a full round without moves
 *   1  every round enqueued ahead; that test runs on the device and sets a
 *      flag after which the kernels of later rounds return at once
 *   2  as 1, the rounds captured in one CUDA graph on a private stream that
 *      joins `stream`; while instrumentation is on, or if the runtime
 *      refuses the capture, the rounds are launched as in 1
 *  -1  (default) 2 for the batched runs (sclap_refine_batched and the
 *      initial partition's individuals), 0 for every other call
 * Learned refinement always runs as 0.  Other values are clamped to -1..2.
 * Returns the previous mode. */
int sclap_set_launch_mode(int mode);

/* Degree-bin and segment thresholds (process-wide; later calls use them).
 * They route rows and contested target segments to kernel paths and change
 * only the speed: every setting gives the same results (each path computes
 * the same selection and arbitration).  The paper has no counterpart.
 * Defaults 32 / 256 / 2048 / 6144; `autotune.py` of the Python package picks
 * them per device and workload by timing candidate sets. */
typedef struct {
    int32_t small_max;  /* rows of <= small_max entries: groups of lanes of one
                           warp (4, 8, 16 or 32)                               */
    int32_t med_max;    /* rows of <= med_max entries: one warp each
                           (small_max .. 256)                                  */
    int32_t mid_max;    /* rows of <= mid_max entries: software-pipelined CTA
                           rows (512, 1024, 2048 or 4096); longer: CTA tables,
                           thread-block clusters and pieces                    */
    int32_t seg_smem;   /* contested segments of <= seg_smem proposals: one CTA
                           (64 .. 6144); longer: the whole grid               */
} sclap_tuning;
int sclap_set_tuning(const sclap_tuning *t);   /* SCLAP_EINVAL outside the ranges */
void sclap_get_tuning(sclap_tuning *t);

/* Instrumentation.  When enabled, the library brackets every launch of the
 * neighbour-aggregation (propose) kernel with CUDA events on its stream and
 * counts the algorithmic bytes it must move (12 B per scanned entry: adjncy,
 * adjwgt, the neighbour-label gather; 24 B per visited node: xadj, label,
 * vwgt, proposal, label write-back).  sclap_prof_read synchronises the device
 * and returns the totals since the last reset.  Meant for one calling thread:
 * while it is enabled, calls from several threads at once are not supported
 * (the event list is not synchronised); the launch counters are atomic. */
typedef struct {
    int64_t propose_launches;
    double propose_ms;            /* sum of event-timed launch durations          */
    double propose_bytes;         /* algorithmic bytes of those launches          */
    int64_t entries_scanned;      /* directed entries aggregated                  */
    int64_t nodes_visited;
    int64_t kernel_launches;      /* every kernel this library launched           */
    int64_t graph_launches;       /* CUDA graphs launched (captured rounds)       */
} sclap_prof;
void sclap_prof_enable(int on);
void sclap_prof_reset(void);
int sclap_prof_read(sclap_prof *out);

#ifdef __cplusplus
}
#endif
#endif
