// lp.cuh -- size-constrained label propagation on the GPU (both forms).
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace sclap {

struct LPConfig {
    DGraph g;
    int32_t *lab;          // device labels (cluster ids or blocks), updated in place
    int64_t nW;            // number of labels: n (clustering) or nblocks (refinement)
    int64_t B;             // U or L_max
    const int64_t *Bv;     // device per-label bounds (batched runs) or null
    bool refine;           // refinement form (overloaded-block rule) vs clustering
    const int32_t *cp;     // V-cycle constraint partition (clustering only) or null
    uint64_t seed;
    int32_t rounds, S;
    // Optional, called on the LP stream before every round (learned
    // refinement): sets *active (device flags per node, null = every node)
    // and returns whether the round is a full one.  A run stops only after a
    // full round without moves.
    std::function<bool(int round, const uint8_t **active)> before_round;
    // Batched runs over a disjoint union (all null / 0 for one graph): run of
    // every node, seed and first node of every run, blocks per run.  A run's
    // sub-rounds and tie-breaks use its seed with its local node and block
    // ids, so it evolves exactly as it would alone.
    const int32_t *run_of = nullptr;
    const uint64_t *run_seed = nullptr;
    const int64_t *run_off = nullptr;
    int32_t run_k = 0;
    bool prefer_capture = false;  // launch mode -1: capture this call's rounds
    // Clustering: sub-rounds by degree quantile (low degrees first) instead
    // of by hash (Sec. III.A's increasing-degree order while coarsening).
    bool degree_order = false;
    // Learned refinement: per node, the weight to the best eligible other
    // label (0 if none) and to its own label that its latest visit saw.
    int32_t *visit_best = nullptr, *visit_own = nullptr;
};

// Runs up to cfg.rounds rounds; returns rounds executed.  moves (optional)
// receives the number of moves of every executed round.  W0 (optional,
// device, nW entries) receives the final label weights.
int lp_run(const LPConfig &cfg, Scratch &sc, std::vector<int64_t> *moves, int64_t *W_out);

// Clustering only: packs the nodes without neighbours into clusters of weight
// <= U in id order (per block of cp when given); see pack_isolated in lp.cu.
void pack_isolated(const DGraph &g, const int32_t *cp, int64_t U, int32_t *lab, Scratch &sc);

// Degree-bin and segment thresholds that route rows and contested segments
// to kernel paths.  Every setting gives the same results (each path computes
// the same selection and arbitration); only the speed differs.  tuning()
// returns the values later calls use; set_tuning returns false (and changes
// nothing) outside the supported ranges.
struct Tuning {
    int32_t small_max;  // rows of <= small_max entries: G-lane groups (4, 8, 16, 32)
    int32_t med_max;    // rows of <= med_max entries: one warp each (small_max..256)
    int32_t mid_max;    // rows of <= mid_max entries: pipelined CTA rows (512 .. 4096)
    int32_t seg_smem;   // contested segments of <= seg_smem entries: one CTA (64..6144)
};
Tuning tuning();
bool set_tuning(const Tuning &t);

// How a call's LP rounds are launched (results do not depend on it): 0 one
// round at a time, the host testing the stop rule; 1 all rounds enqueued
// ahead, a device flag ending them; 2 as 1, captured in one CUDA graph; -1
// (default) 2 for calls that prefer capture (batched runs), else 0.
// set_launch_mode returns the previous mode.
int launch_mode();
int set_launch_mode(int mode);

// Runs the arbitration kernel's bounded grid barrier with one of two CTAs
// absent, so the wait must give up after limit_cycles; returns SCLAP_ETIMEOUT
// when it did (the expected result) and SCLAP_OK if it did not.
int barrier_selftest(long long limit_cycles, Scratch &sc);

}  // namespace sclap
