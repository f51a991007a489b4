// contract.cuh -- cluster contraction, projection and cut on the GPU.
#pragma once

#include "common.cuh"

namespace sclap {

struct CoarseGraph {
    int64_t n = 0, nnz = 0;
    int64_t *xadj = nullptr;
    int32_t *adjncy = nullptr, *adjwgt = nullptr, *vwgt = nullptr;
};

// Contracts the clustering `lab` of g (Sec. III, Sec. IV.C).  Output arrays
// come from out_sc when given, else from cudaMalloc (caller frees).  f2c is
// written for every fine node.
void contract_impl(const DGraph &g, const int32_t *lab, int32_t *f2c, CoarseGraph *out,
                   Scratch *out_sc, Scratch &tmp);

void project_impl(int64_t n_fine, const int32_t *f2c, const int32_t *coarse_part,
                  int32_t *fine_part, cudaStream_t s);

// Cut and block weights.  groups > 1: nodes [goff[t], goff[t+1]) form group t
// (disjoint graphs; goff device int64[groups+1]) and d_cut[t] is its cut.
// Results are device arrays.
void cut_impl(const DGraph &g, const int32_t *part, int64_t nblocks, int64_t groups,
              const int64_t *goff, int64_t *d_cut /* [groups] */, int64_t *d_bw /* [nblocks] */,
              Scratch &sc);

// The same cut and block-weight kernels on caller-provided, zeroed device
// accumulators (d_cut: 1 entry, d_bw: nblocks entries, d_bad: 1 entry that
// counts block ids outside [0, nblocks), which are skipped); allocates nothing.
void cut_launch(const DGraph &g, const int32_t *part, int64_t nblocks, unsigned long long *d_cut,
                unsigned long long *d_bw, unsigned long long *d_bad, cudaStream_t s, int sms);

}  // namespace sclap
