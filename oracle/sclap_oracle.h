/*
 * sclap_oracle.h -- plain CPU oracle for size-constrained label propagation
 * (SCLaP), cluster contraction, projection and the multilevel driver of
 * Meyerhenke, Sanders and Schulz, "Parallel Graph Partitioning for Complex
 * Networks" (2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The product path
 * (the CUDA library) shares no code, header, table or helper with it.
 *
 * Every routine is written to be read against the paper:
 *   Sec. II.A   definitions (L_max, cut, quotient graph)
 *   Sec. III.A  label propagation with size constraints (both forms)
 *   Sec. IV.B   balance / size constraint
 *   Sec. IV.C   contraction and uncoarsening
 *   Sec. IV.E   the overall multilevel system
 * Where the paper is silent the oracle implements one fixed reading that
 * makes the method deterministic; each reading is stated where it is used.
 */
#ifndef SCLAP_ORACLE_H
#define SCLAP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_EGRAPH = 2, OR_EOVERFLOW = 3, OR_ENOMEM = 4 };

typedef struct {
    int32_t k;            /* number of blocks                              */
    double eps;           /* imbalance parameter                           */
    int64_t U;            /* cluster bound; <= 0: max(max c(v), c(V)/(10k)) */
    int32_t cluster_rounds; /* l (ell): LP rounds per coarsening level      */
    int32_t refine_rounds;  /* r: LP rounds per uncoarsening level          */
    int32_t subrounds;      /* S: synchronous colour classes per round      */
    int64_t n_stop;         /* coarsen while n >= n_stop                    */
    int32_t max_levels;     /* hard cap on hierarchy depth                  */
    int32_t init_seeds;     /* P: initial-partition population size        */
    int32_t init_rounds;    /* refinement rounds inside initial partition   */
    uint64_t seed;
    int32_t degree_order;   /* 1: degree-ordered clustering sub-rounds      */
} or_ml_params;

#define OR_MAX_LEVELS 64
typedef struct {
    int32_t levels;                    /* number of graphs in the hierarchy */
    int64_t n[OR_MAX_LEVELS];
    int64_t nnz[OR_MAX_LEVELS];
    int32_t cluster_rounds_done[OR_MAX_LEVELS];
    int32_t refine_rounds_done[OR_MAX_LEVELS];
    int64_t U, lmax;
    int32_t init_best;
    int64_t init_cut, init_maxbw;
    int64_t cut, maxbw;
} or_ml_stats;

/* Threads of the per-node propose loop (OpenMP builds; default 1).  The
 * results do not depend on it. */
void or_set_threads(int t);
int or_get_threads(void);

uint64_t or_mix64(uint64_t z);
uint32_t or_colour(uint64_t seed, int32_t round, int64_t v, int32_t S);
uint32_t or_tie(uint64_t seed, int32_t round, int64_t v, int64_t L);
int64_t or_lmax(int64_t cV, int32_t k, double eps);

int or_validate(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *adjwgt, const int32_t *vwgt);

int or_cluster(int64_t n, const int64_t *xadj, const int32_t *adjncy,
               const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
               int32_t rounds, int32_t S, uint64_t seed,
               const int32_t *constraint_part, int32_t *labels_out,
               int32_t *rounds_done, int64_t *moves_per_round);

int or_cluster_degree_ordered(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                              const int32_t *adjwgt, const int32_t *vwgt, int64_t U,
                              int32_t rounds, int32_t S, uint64_t seed,
                              const int32_t *constraint_part, int32_t *labels_out,
                              int32_t *rounds_done, int64_t *moves_per_round);
int or_degree_colours(int64_t n, const int64_t *xadj, uint64_t seed, int32_t round, int32_t S,
                      int32_t *colour_out);

int or_refine_bound(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                    const int32_t *adjwgt, const int32_t *vwgt, int32_t nblocks,
                    int64_t B, int32_t rounds, int32_t S, uint64_t seed,
                    int32_t *part_inout, int32_t *rounds_done,
                    int64_t *moves_per_round);

int or_refine(int64_t n, const int64_t *xadj, const int32_t *adjncy,
              const int32_t *adjwgt, const int32_t *vwgt, int32_t k, double eps,
              int32_t rounds, int32_t S, uint64_t seed, int32_t *part_inout,
              int64_t *cut_out, int64_t *block_w_out, int32_t *rounds_done,
              int64_t *moves_per_round);

int or_contract(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                const int32_t *adjwgt, const int32_t *vwgt, const int32_t *labels,
                int64_t *cn, int64_t *cnnz, int64_t **cxadj, int32_t **cadjncy,
                int32_t **cadjwgt, int32_t **cvwgt, int32_t *f2c_out);

void or_free(void *p);

void or_project(int64_t n_fine, const int32_t *f2c, const int32_t *coarse_part,
                int32_t *fine_part_out);

int64_t or_cut(int64_t n, const int64_t *xadj, const int32_t *adjncy,
               const int32_t *adjwgt, const int32_t *part);

void or_block_weights(int64_t n, const int32_t *vwgt, const int32_t *part,
                      int32_t k, int64_t *bw_out);

int or_initial_partition(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                         const int32_t *adjwgt, const int32_t *vwgt, int32_t k,
                         int64_t B, int32_t P, int32_t rounds, int32_t S,
                         uint64_t seed, int32_t *part_out, int64_t *cuts_out,
                         int64_t *maxbw_out, int32_t *best_out);

int or_refine_batched(int32_t ngraphs, const int64_t *ns, const int64_t *const *xadjs,
                      const int32_t *const *adjncys, const int32_t *const *adjwgts,
                      const int32_t *const *vwgts, int32_t k, const int64_t *Bg,
                      int32_t rounds, int32_t S, const uint64_t *seeds, int32_t nruns,
                      const int32_t *run_graph, int32_t *parts_out, int64_t *cuts_out,
                      int64_t *maxbw_out);

int or_lpt_start(int64_t n, const int32_t *vwgt, int32_t k, uint64_t seed, int32_t *part_out);

int or_multilevel(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                  const int32_t *adjwgt, const int32_t *vwgt,
                  const or_ml_params *p, int32_t *part_out, or_ml_stats *st);

int or_vcycle(int64_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
              const int32_t *vwgt, const or_ml_params *p, int32_t *part_inout,
              or_ml_stats *st);

/* learned active set (refinement gate; not in the paper) */
#define OR_MLP_NPARAM 1313
#define OR_MLP_W1 0     /* [32][6] */
#define OR_MLP_B1 192   /* [32] */
#define OR_MLP_W2 224   /* [32][32] */
#define OR_MLP_B2 1248  /* [32] */
#define OR_MLP_W3 1280  /* [32] */
#define OR_MLP_B3 1312  /* [1] */

float or_bf16(float f);
float or_log2_feature(int64_t x);
void or_features(int64_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *adjwgt,
                 const int32_t *lab, const int64_t *W, int64_t Lmax, const uint8_t *moved,
                 const int64_t *vis_best, const int64_t *vis_own, float *x);
float or_mlp_forward(const uint16_t *net, const float *x);
void or_mlp_score(int64_t N, const float *X, const uint16_t *net, float *z);
int or_refine_learned(int64_t n, const int64_t *xadj, const int32_t *adjncy,
                      const int32_t *adjwgt, const int32_t *vwgt, int32_t k, double eps,
                      int32_t rounds, int32_t S, uint64_t seed, const uint16_t *net,
                      float z_min, int32_t full_every, int32_t *part, int32_t *rounds_done,
                      int64_t *moves_per_round, int64_t *visited_out, float *trace_x,
                      uint8_t *trace_y);
double or_mlp_loss_grad_bf16(const float *X, const uint8_t *y, int64_t N, const float *prm,
                             double *grad);
double or_mlp_loss_grad(const float *X, const uint8_t *y, int64_t N, const float *prm,
                        double *grad);

#ifdef __cplusplus
}
#endif
#endif
