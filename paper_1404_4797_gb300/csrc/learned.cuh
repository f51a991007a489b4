// learned.cuh -- the learned active set of refinement (a gate that decides
// which nodes a refinement round visits; it is not in the paper) and the
// kernels that train its scorer.
#pragma once

#include "common.cuh"

namespace sclap {

// Scorer parameters: 1313 values, W1[32][6], b1[32], W2[32][32], b2[32],
// W3[32], b3 (bf16 bit patterns for inference, float for training).
constexpr int kMlpParams = 1313;
constexpr int kMlpW1 = 0, kMlpB1 = 192, kMlpW2 = 224, kMlpB2 = 1248, kMlpW3 = 1280, kMlpB3 = 1312;

// Per-call state of the gate (device arrays sized for the graph).
struct Gate {
    DGraph g;
    const int32_t *lab;
    const int64_t *W;       // block weights of the LP run
    int64_t Lmax;
    const uint16_t *net;    // bf16 parameters or null (no gate: plain rounds)
    float z_min;
    int full_every, rounds;
    float *trace_x;         // [rounds][n][6] or null
    uint8_t *trace_y;       // [rounds][n] or null
    bool unit;              // every edge weight is 1 (then wdeg stays null)
    int64_t *wdeg;          // static weighted degrees
    int32_t *prev;          // labels at the start of the previous round
    uint8_t *moved;         // moved in the previous round
    uint8_t *active;
    int32_t *vb, *vo;           // latest visit: weight to the best eligible other / own block
    int32_t *nmov;              // per round: moved neighbours
    int32_t *movers, *nmovers;  // nodes that moved in the previous round (short rows;
                                // nmovers[0]) and the pieces of long ones (nmovers[1])
    int64_t *pieces;
    unsigned long long *visited;  // device counters: rows visited by gated or traced
                                  // rounds; [1] rows with neighbours
    int nfull = 0;                // full rounds without traces (host count): each
                                  // visits visited[1] rows
};

// Allocates the gate's arrays and computes the weighted degrees.
void gate_init(Gate &gt, Scratch &sc);
// Before round r: moved flags of round r - 1 (into trace_y[r - 1]), features
// (into trace_x[r]), scores and active flags.  Returns whether r is full
// (r == 0, r % full_every == full_every - 1, the last round, or no network).
bool gate_round(Gate &gt, int r, const uint8_t **active, cudaStream_t s);
// After the last executed round: its moved flags into trace_y[rounds_done - 1].
void gate_finish(Gate &gt, int rounds_done, cudaStream_t s);

// Logits of N feature rows with the bf16 scorer.
void mlp_score(const float *x, int64_t N, const uint16_t *net, float *z, cudaStream_t s);
// Mean logistic loss and gradient over samples idx[0, N) (idx null: 0..N-1)
// of float parameters (bf16_in: of the bf16 network inference runs, with the
// straight-through gradient); grad (device, kMlpParams) and *d_loss (device
// double) are accumulated into (zero them first).
void mlp_loss_grad(const float *X, const uint8_t *y, const int64_t *idx, int64_t N,
                   const float *prm, float *grad, double *d_loss, bool bf16_in, cudaStream_t s);
// bf16 bit patterns (nearest even) of the kMlpParams float parameters
void mlp_pack_bf16(const float *prm, uint16_t *net, cudaStream_t s);
// prm -= lr * grad
void mlp_sgd(float *prm, const float *grad, float lr, cudaStream_t s);

}  // namespace sclap
