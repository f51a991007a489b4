// api.cu -- the C ABI (include/sclap.h): argument checks, graph validation,
// overflow checks, the initial partitioner and the multilevel driver.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "contract.cuh"
#include "learned.cuh"
#include "lp.cuh"
#include "prims.cuh"

using namespace sclap;

namespace {

std::atomic<bool> g_validate{true};  // process-wide, set from any thread

template <class F>
int guarded(F &&f) {
    try {
        f();
        return SCLAP_OK;
    } catch (const Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return SCLAP_ENOMEM;
    } catch (...) {
        return SCLAP_ECUDA;
    }
}

cudaStream_t as_stream(void *p) { return reinterpret_cast<cudaStream_t>(p); }

DGraph view(const sclap_graph *g) {
    return DGraph{g->n, g->nnz, g->xadj, g->adjncy, g->adjwgt, g->vwgt};
}

// Sec. II.A: L_max = (1 + eps) * ceil(c(V) / k), rounded down.
int64_t lmax_of(int64_t cV, int32_t k, double eps) {
    int64_t avg = (cV + k - 1) / k;
    return (int64_t)std::floor((1.0 + eps) * (double)avg);
}

uint64_t level_seed(uint64_t seed, int l) {
    return mix64(seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(l + 1)));
}

// identity labels (clustering with zero rounds)
__global__ void k_identity(int64_t n, int32_t *lab) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        lab[v] = (int32_t)v;
}

void identity_labels(int64_t n, int32_t *lab, cudaStream_t s) {
    if (n <= 0) return;
    k_identity<<<dev_info().sms * 4, 256, 0, s>>>(n, lab);
    LAUNCHED();
}

// ---------------------------------------------------------------- validation

__global__ void k_validate_nodes(DGraph g, int *bad) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (g.xadj[v + 1] < g.xadj[v] || g.vwgt[v] < 0) atomicOr(bad, 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        if (g.xadj[0] != 0 || g.xadj[g.n] != g.nnz) atomicOr(bad, 1);
}

// Entry checks (xadj already known to be monotone): ids in range, no
// self-loops, omega > 0, rows strictly ascending; symmetry (every (v, u, w)
// has its mirror (u, v, w)) through a fingerprint: the wrapping sums of
// mix64 over (v, u, w) and over (u, v, w) must agree (a mismatch escapes with
// probability about 2^-64).
constexpr int kValTile = 4096;

__device__ __forceinline__ uint64_t entry_fp(uint64_t a, uint64_t b, uint64_t w) {
    return mix64(mix64((a << 32) | b) ^ (w * 0x9E3779B97F4A7C15ull));
}

__global__ void __launch_bounds__(256) k_validate_entries(DGraph g, int *bad,
                                                          unsigned long long *fp /* [2] */) {
    __shared__ int32_t rowof[kValTile];
    __shared__ int32_t tmp[16];
    const int64_t tiles = ceil_div<int64_t>(g.nnz, kValTile);
    unsigned long long f0 = 0, f1 = 0;
    int err = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kValTile;
        const int len = (int)min64(kValTile, g.nnz - e0);
        block_rows<256, 16>(g.xadj, g.n, e0, len, rowof, tmp);
        for (int i = threadIdx.x; i < len; i += 256) {
            const int64_t e = e0 + i;
            const int32_t v = rowof[i];
            const int32_t u = g.adjncy[e];
            const int32_t w = g.adjwgt[e];
            if (u < 0 || u >= g.n || u == v || w <= 0) err = 1;
            if (e > g.xadj[v] && g.adjncy[e - 1] >= u) err = 1;
            f0 += entry_fp((uint32_t)v, (uint32_t)u, (uint32_t)w);
            f1 += entry_fp((uint32_t)u, (uint32_t)v, (uint32_t)w);
        }
        __syncthreads();
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        f0 += __shfl_down_sync(0xffffffffu, f0, d);
        f1 += __shfl_down_sync(0xffffffffu, f1, d);
        err |= __shfl_down_sync(0xffffffffu, err, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&fp[0], f0);
        atomicAdd(&fp[1], f1);
        if (err) atomicOr(bad, 1);
    }
}

void validate_graph(const DGraph &g, Scratch &sc) {
    if (g.n < 0 || g.nnz < 0 || g.n > INT32_MAX) fail(SCLAP_EINVAL, "graph size");
    if (g.n > 0 && (!g.xadj || !g.vwgt)) fail(SCLAP_EINVAL, "null graph array");
    if (g.nnz > 0 && (!g.adjncy || !g.adjwgt)) fail(SCLAP_EINVAL, "null graph array");
    if (!g_validate.load() || g.n == 0) return;
    cudaStream_t s = sc.stream();
    int *bad = sc.zeros<int>(1);
    int grid = dev_info().sms * 8;
    k_validate_nodes<<<grid, 256, 0, s>>>(g, bad);
    LAUNCHED();
    int h = 0;
    CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h) fail(SCLAP_EGRAPH, "xadj / vwgt");
    if (g.nnz > 0) {
        unsigned long long *fp = sc.zeros<unsigned long long>(2);
        const int vgrid = (int)std::min<int64_t>(ceil_div<int64_t>(g.nnz, kValTile), grid);
        k_validate_entries<<<vgrid, 256, 0, s>>>(g, bad, fp);
        LAUNCHED();
        unsigned long long hf[2];
        CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hf, fp, sizeof(hf), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h || hf[0] != hf[1]) fail(SCLAP_EGRAPH, "adjacency");
    }
}

__global__ void k_check_range(int64_t n, const int32_t *a, int64_t hi, int *bad) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (a[v] < 0 || a[v] >= hi) atomicOr(bad, 1);
}

bool in_range(int64_t n, const int32_t *a, int64_t hi, Scratch &sc) {
    if (n == 0) return true;
    cudaStream_t s = sc.stream();
    int *bad = sc.zeros<int>(1);
    k_check_range<<<dev_info().sms * 4, 256, 0, s>>>(n, a, hi, bad);
    LAUNCHED();
    int h = 0;
    CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h == 0;
}

// ---------------------------------------------------------------- initial partition

// Batched runs over the disjoint union of their graphs (run r: nodes off_r + v,
// entries eoff_r + i, blocks r*k .. r*k+k-1).
struct RunDesc {
    const int64_t *xadj;
    const int32_t *adjncy, *adjwgt, *vwgt;
    int64_t n, off, eoff;
    int64_t bound;  // the run's L_max
    uint64_t seed;  // the run's seed (LPT order and SCLaP hashes)
};

__device__ __forceinline__ int64_t run_of(const RunDesc *rd, int64_t nruns, int64_t x, bool entries) {
    int64_t lo = 0, hi = nruns;  // largest r with off_r <= x
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if ((entries ? rd[mid].eoff : rd[mid].off) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t run_of_node(const RunDesc *rd, int64_t nruns, int64_t i) {
    return run_of(rd, nruns, i, false);
}

__global__ void k_union_batch(const RunDesc *rd, int64_t nruns, int64_t un, int64_t unnz,
                              int64_t *ux, int32_t *ua, int32_t *uw, int32_t *uc, int64_t *goff) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < un;
         i += (int64_t)gridDim.x * blockDim.x) {
        const RunDesc &r = rd[run_of(rd, nruns, i, false)];
        const int64_t v = i - r.off;
        ux[i] = r.eoff + r.xadj[v];
        uc[i] = r.vwgt[v];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < unnz;
         i += (int64_t)gridDim.x * blockDim.x) {
        const RunDesc &r = rd[run_of(rd, nruns, i, true)];
        const int64_t e = i - r.eoff;
        ua[i] = (int32_t)(r.adjncy[e] + r.off);
        uw[i] = r.adjwgt[e];
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= nruns;
         r += (int64_t)gridDim.x * blockDim.x)
        goff[r] = r < nruns ? rd[r].off : un;
    if (blockIdx.x == 0 && threadIdx.x == 0) ux[un] = unnz;
}

// LPT order keys: first pass h_r(v) (local v), second pass (r, cmax - c).
__global__ void k_lpt_keys1(const RunDesc *rd, int64_t nruns, int64_t un, uint64_t *key,
                            int32_t *idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < un;
         i += (int64_t)gridDim.x * blockDim.x) {
        const RunDesc &r = rd[run_of(rd, nruns, i, false)];
        key[i] = mix64(r.seed ^ (uint64_t)(i - r.off)) >> 32;
        idx[i] = (int32_t)i;
    }
}

__global__ void k_lpt_keys2(const RunDesc *rd, int64_t nruns, const int32_t *idx,
                            const int32_t *uc, int cb, int64_t cmax, int64_t un, uint64_t *key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < un;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = idx[i];
        const int64_t r = run_of(rd, nruns, u, false);
        key[i] = ((uint64_t)r << cb) | (uint64_t)(cmax - uc[u]);
    }
}

// One warp per run: its nodes in sorted order go to the lightest of its k
// blocks (lowest id on ties).  Sequential by nature: block weights live in
// registers (k <= 32, lane b holds block b) or shared memory, 32 upcoming
// nodes are prefetched per lane, and the argmin is two warp reductions
// (weights fit 32 bits: c(V) <= INT32_MAX is checked).
__global__ void k_lpt_assign(const RunDesc *rd, int32_t k, const int32_t *order,
                             const int32_t *uc, int32_t *upart) {
    extern __shared__ unsigned bw[];
    const int64_t r = blockIdx.x;
    const int lane = threadIdx.x;
    for (int b = lane; b < k; b += 32) bw[b] = 0;
    __syncwarp();
    const int64_t n = rd[r].n;
    const int32_t *ord = order + rd[r].off;
    for (int64_t i0 = 0; i0 < n; i0 += 32) {
        const int64_t i = i0 + lane;
        int32_t u = 0, c = 0;
        if (i < n) {
            u = ord[i];
            c = uc[u];
        }
        const int cnt = (int)min64(32, n - i0);
        if (k <= 32) {
            // k <= 32: lane b keeps block b's weight in a register
            unsigned wb = lane < k ? bw[lane] : 0xffffffffu;
            for (int j = 0; j < cnt; j++) {
                const int32_t uj = __shfl_sync(0xffffffffu, u, j);
                const int32_t cj = __shfl_sync(0xffffffffu, c, j);
                const unsigned gw = __reduce_min_sync(0xffffffffu, wb);
                const unsigned gb = __reduce_min_sync(0xffffffffu, wb == gw ? (unsigned)lane : 32u);
                if (lane == (int)gb) wb += (unsigned)cj;
                if (lane == 0) upart[uj] = (int32_t)(r * k + gb);
            }
            if (lane < k) bw[lane] = wb;
            __syncwarp();
            continue;
        }
        for (int j = 0; j < cnt; j++) {
            const int32_t uj = __shfl_sync(0xffffffffu, u, j);
            const int32_t cj = __shfl_sync(0xffffffffu, c, j);
            unsigned wmin = 0xffffffffu, bmin = 0xffffffffu;
            for (int b = lane; b < k; b += 32)
                if (bw[b] < wmin) { wmin = bw[b]; bmin = (unsigned)b; }
            const unsigned gw = __reduce_min_sync(0xffffffffu, wmin);
            const unsigned gb = __reduce_min_sync(0xffffffffu, wmin == gw ? bmin : 0xffffffffu);
            if (lane == (int)(gb & 31)) bw[gb] += (unsigned)cj;
            if (lane == 0) upart[uj] = (int32_t)(r * k + gb);
            __syncwarp();
        }
    }
}

__global__ void k_run_bounds(const RunDesc *rd, int64_t nruns, int32_t k, int64_t *Bv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nruns * k;
         i += (int64_t)gridDim.x * blockDim.x)
        Bv[i] = rd[i / k].bound;
}

// Run id of every union node, and each run's seed and first node.
__global__ void k_run_map(const RunDesc *rd, int64_t nruns, int64_t un, int32_t *run_of,
                          uint64_t *run_seed, int64_t *run_off) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < un;
         i += (int64_t)gridDim.x * blockDim.x)
        run_of[i] = (int32_t)run_of_node(rd, nruns, i);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nruns;
         r += (int64_t)gridDim.x * blockDim.x) {
        run_seed[r] = rd[r].seed;
        run_off[r] = rd[r].off;
    }
}

__global__ void k_run_max(int64_t nruns, int32_t k, const int64_t *bw, int64_t *maxbw) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nruns;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = 0;
        for (int b = 0; b < k; b++) m = max64(m, bw[r * k + b]);
        maxbw[r] = m;
    }
}

__global__ void k_run_parts(const RunDesc *rd, int64_t nruns, int32_t k, int64_t un,
                            const int32_t *upart, int32_t *parts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < un;
         i += (int64_t)gridDim.x * blockDim.x)
        parts[i] = upart[i] - (int32_t)(run_of(rd, nruns, i, false) * k);
}

struct BatchResult {
    std::vector<int64_t> cuts, maxbw;
    int64_t total_n = 0;
};

// All runs refined together (see sclap_refine_batched).  parts_out: device,
// sum of the runs' node counts.
BatchResult batched_impl(const std::vector<DGraph> &G, const std::vector<int64_t> &bound,
                         const std::vector<int32_t> &run_graph, const std::vector<uint64_t> &seeds,
                         int32_t k, int32_t rounds, int32_t S, int32_t *parts_out, Scratch &sc) {
    cudaStream_t s = sc.stream();
    const int grid = dev_info().sms * 8;
    const int64_t nruns = (int64_t)run_graph.size();
    std::vector<RunDesc> rd(nruns);
    int64_t un = 0, unnz = 0, cmax = 0, cV = 0;
    std::vector<GraphTotals> tot(G.size());
    for (size_t gi = 0; gi < G.size(); gi++) tot[gi] = graph_totals(G[gi], sc, true);
    for (int64_t r = 0; r < nruns; r++) {
        const DGraph &g = G[run_graph[r]];
        rd[r] = RunDesc{g.xadj, g.adjncy, g.adjwgt, g.vwgt, g.n, un, unnz, bound[run_graph[r]],
                        seeds[r]};
        un += g.n;
        unnz += g.nnz;
        cmax = std::max<int64_t>(cmax, tot[run_graph[r]].maxc);
        cV = std::max<int64_t>(cV, tot[run_graph[r]].cV);
        if (tot[run_graph[r]].max_wdeg > INT32_MAX) fail(SCLAP_EOVERFLOW, "weighted degree");
    }
    if (cV > INT32_MAX) fail(SCLAP_EOVERFLOW, "c(V) of a run");
    if (un > INT32_MAX) fail(SCLAP_EINVAL, "batched runs too large");
    BatchResult res;
    res.cuts.assign(nruns, 0);
    res.maxbw.assign(nruns, 0);
    res.total_n = un;
    if (un == 0) return res;
    RunDesc *d_rd = sc.get<RunDesc>(nruns);
    CK(cudaMemcpyAsync(d_rd, rd.data(), nruns * sizeof(RunDesc), cudaMemcpyHostToDevice, s));
    int64_t *ux = sc.get<int64_t>(un + 1);
    int32_t *ua = sc.get<int32_t>(unnz);
    int32_t *uw = sc.get<int32_t>(unnz);
    int32_t *uc = sc.get<int32_t>(un);
    int32_t *up = sc.get<int32_t>(un);
    int64_t *goff = sc.get<int64_t>(nruns + 1);
    k_union_batch<<<grid, 256, 0, s>>>(d_rd, nruns, un, unnz, ux, ua, uw, uc, goff);
    LAUNCHED();
    // LPT start of every run: order (run, c desc, h_r(v) asc, v asc) by two stable sorts
    uint64_t *key = sc.get<uint64_t>(un);
    int32_t *idx = sc.get<int32_t>(un);
    k_lpt_keys1<<<grid, 256, 0, s>>>(d_rd, nruns, un, key, idx);
    LAUNCHED();
    radix_sort_pairs(key, idx, un, 32, sc);
    const int cb = std::max(1, bit_width_u64((uint64_t)cmax));
    const int rb = std::max(1, bit_width_u64((uint64_t)(nruns - 1)));
    k_lpt_keys2<<<grid, 256, 0, s>>>(d_rd, nruns, idx, uc, cb, cmax, un, key);
    LAUNCHED();
    radix_sort_pairs(key, idx, un, cb + rb, sc);
    k_lpt_assign<<<(unsigned)nruns, 32, k * sizeof(unsigned), s>>>(d_rd, k, idx, uc, up);
    LAUNCHED();
    int64_t *Bv = sc.get<int64_t>(nruns * k);
    k_run_bounds<<<grid, 256, 0, s>>>(d_rd, nruns, k, Bv);
    LAUNCHED();
    int32_t *run_of = sc.get<int32_t>(un);
    uint64_t *run_seed = sc.get<uint64_t>(nruns);
    int64_t *run_off = sc.get<int64_t>(nruns);
    k_run_map<<<grid, 256, 0, s>>>(d_rd, nruns, un, run_of, run_seed, run_off);
    LAUNCHED();
    // refine all runs together on the disjoint union
    DGraph ug{un, unnz, ux, ua, uw, uc};
    LPConfig cfg{};
    cfg.g = ug;
    cfg.lab = up;
    cfg.nW = (int64_t)k * nruns;
    cfg.B = 0;
    cfg.Bv = Bv;
    cfg.refine = true;
    cfg.cp = nullptr;
    cfg.seed = 0;  // every run uses its own seed
    cfg.rounds = rounds;
    cfg.S = S;
    cfg.run_of = run_of;
    cfg.run_seed = run_seed;
    cfg.run_off = run_off;
    cfg.run_k = k;
    cfg.prefer_capture = true;
    lp_run(cfg, sc, nullptr, nullptr);
    int64_t *d_cut = sc.get<int64_t>(nruns);
    int64_t *d_bw = sc.get<int64_t>((int64_t)k * nruns);
    int64_t *d_max = sc.get<int64_t>(nruns);
    cut_impl(ug, up, (int64_t)k * nruns, nruns, goff, d_cut, d_bw, sc);
    k_run_max<<<grid, 256, 0, s>>>(nruns, k, d_bw, d_max);
    LAUNCHED();
    if (parts_out) {
        k_run_parts<<<grid, 256, 0, s>>>(d_rd, nruns, k, un, up, parts_out);
        LAUNCHED();
    }
    CK(cudaMemcpyAsync(res.cuts.data(), d_cut, nruns * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(res.maxbw.data(), d_max, nruns * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return res;
}

// Best individual: lowest cut among those with max block <= B (lowest t on
// ties); otherwise smallest max block, then cut, then t.
int32_t pick_best(const std::vector<int64_t> &cuts, const std::vector<int64_t> &mx, int64_t B) {
    int32_t best = -1;
    for (int32_t t = 0; t < (int32_t)cuts.size(); t++) {
        bool better;
        if (best < 0) better = true;
        else {
            const bool fn = mx[t] <= B, fo = mx[best] <= B;
            if (fn != fo) better = fn;
            else if (fn) better = cuts[t] < cuts[best];
            else better = mx[t] < mx[best] || (mx[t] == mx[best] && cuts[t] < cuts[best]);
        }
        if (better) best = t;
    }
    return best;
}

struct InitResult {
    int32_t best;
    std::vector<int64_t> cuts, maxbw;
};

// P individuals on one graph (batched runs) and the best of them.
InitResult initial_impl(const DGraph &g, int32_t k, int64_t B, int32_t P, int32_t rounds,
                        int32_t S, uint64_t seed, int32_t *part_out, Scratch &sc) {
    cudaStream_t s = sc.stream();
    InitResult res;
    int32_t *parts = sc.get<int32_t>((size_t)g.n * P);
    std::vector<uint64_t> seeds(P);
    for (int32_t t = 0; t < P; t++) seeds[t] = mix64(seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(t + 1)));
    BatchResult br = batched_impl({g}, {B}, std::vector<int32_t>(P, 0), seeds, k, rounds, S, parts, sc);
    res.cuts = br.cuts;
    res.maxbw = br.maxbw;
    res.best = g.n > 0 ? pick_best(br.cuts, br.maxbw, B) : 0;
    if (g.n > 0)
        CK(cudaMemcpyAsync(part_out, parts + (int64_t)res.best * g.n, g.n * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s));
    return res;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Every cluster weight is at most c(V); every coarse edge weight and every
// omega(v, L) is a sum over distinct undirected edges, so at most the
// undirected total (half the sum over the directed entries).
void check_totals_cluster(const GraphTotals &t) {
    if (t.cV > INT32_MAX || t.sum_w / 2 > INT32_MAX) fail(SCLAP_EOVERFLOW, "c(V) or sum(omega)");
}

}  // namespace

// ---------------------------------------------------------------- C ABI

namespace {

// Keys of the shuffle of epoch e: SplitMix64 of (seed, epoch, sample).
__global__ void k_shuffle_keys(int64_t N, uint64_t seed, int epoch, uint64_t *keys,
                               int32_t *vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        keys[i] = mix64(seed ^ ((uint64_t)(epoch + 1) << 40) ^ (uint64_t)i);
        vals[i] = (int32_t)i;
    }
}

__global__ void k_widen(int64_t N, const int32_t *a, int64_t *b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

}  // namespace

extern "C" {

const char *sclap_strerror(int code) {
    switch (code) {
        case SCLAP_OK: return "ok";
        case SCLAP_EINVAL: return "invalid argument";
        case SCLAP_EGRAPH: return "graph failed validation";
        case SCLAP_EOVERFLOW: return "weights exceed the 32-bit range";
        case SCLAP_ENOMEM: return "out of device memory";
        case SCLAP_ECUDA: return "CUDA error";
        case SCLAP_ETIMEOUT: return "device wait timed out";
        case SCLAP_ENOTIMPL: return "not implemented";
        default: return "unknown error";
    }
}

int sclap_set_launch_mode(int mode) { return set_launch_mode(mode); }

int sclap_set_tuning(const sclap_tuning *t) {
    if (!t) return SCLAP_EINVAL;
    return set_tuning(Tuning{t->small_max, t->med_max, t->mid_max, t->seg_smem}) ? SCLAP_OK
                                                                                : SCLAP_EINVAL;
}

void sclap_get_tuning(sclap_tuning *t) {
    if (!t) return;
    const Tuning x = tuning();
    t->small_max = x.small_max;
    t->med_max = x.med_max;
    t->mid_max = x.mid_max;
    t->seg_smem = x.seg_smem;
}

int sclap_set_validation(int on) {
    return g_validate.exchange(on != 0) ? 1 : 0;
}

void sclap_ml_defaults(sclap_ml_params *p, int32_t k, double eps, uint64_t seed) {
    std::memset(p, 0, sizeof(*p));
    p->k = k;
    p->eps = eps;
    p->U = 0;
    p->cluster_rounds = 3;
    p->refine_rounds = 6;
    p->subrounds = 4;
    p->n_stop = 2000;
    p->max_levels = 32;
    p->init_seeds = 8;
    p->init_rounds = 6;
    p->seed = seed;
}

static int cluster_call(const sclap_graph *gp, int64_t U, int32_t rounds, int32_t subrounds,
                        uint64_t seed, const int32_t *constraint_part, bool degree_order,
                        int32_t *labels_out, int32_t *rounds_done, void *stream) {
    return guarded([&] {
        if (!gp || (!labels_out && gp->n > 0)) fail(SCLAP_EINVAL, "null");
        if (rounds < 0 || subrounds < 1 || subrounds > 32) fail(SCLAP_EINVAL, "rounds");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);
        GraphTotals t = graph_totals(g, sc);
        if (U < t.maxc) fail(SCLAP_EINVAL, "U < max c(v)");
        check_totals_cluster(t);
        LPConfig cfg{};
        cfg.g = g;
        cfg.lab = labels_out;
        cfg.nW = g.n;
        cfg.B = U;
        cfg.refine = false;
        cfg.cp = constraint_part;
        cfg.seed = seed;
        cfg.rounds = rounds;
        cfg.S = subrounds;
        cfg.degree_order = degree_order;
        int rd = 0;
        if (rounds > 0 && g.n > 0) rd = lp_run(cfg, sc, nullptr, nullptr);
        else identity_labels(g.n, labels_out, s);
        pack_isolated(g, constraint_part, U, labels_out, sc);
        CK(cudaStreamSynchronize(s));
        if (rounds_done) *rounds_done = rd;
    });
}

int sclap_cluster(const sclap_graph *gp, int64_t U, int32_t rounds, int32_t subrounds,
                  uint64_t seed, const int32_t *constraint_part, int32_t *labels_out,
                  int32_t *rounds_done, void *stream) {
    return cluster_call(gp, U, rounds, subrounds, seed, constraint_part, false, labels_out,
                        rounds_done, stream);
}

int sclap_cluster_degree_ordered(const sclap_graph *gp, int64_t U, int32_t rounds,
                                 int32_t subrounds, uint64_t seed,
                                 const int32_t *constraint_part, int32_t *labels_out,
                                 int32_t *rounds_done, void *stream) {
    return cluster_call(gp, U, rounds, subrounds, seed, constraint_part, true, labels_out,
                        rounds_done, stream);
}

int sclap_refine_bound(const sclap_graph *gp, int32_t nblocks, int64_t B, int32_t rounds,
                       int32_t subrounds, uint64_t seed, int32_t *part_inout,
                       int32_t *rounds_done, void *stream) {
    cudaStream_t s = as_stream(stream);
    int32_t *backup = nullptr;
    int rc = guarded([&] {
        if (!gp || (!part_inout && gp->n > 0)) fail(SCLAP_EINVAL, "null");
        if (nblocks < 1 || rounds < 0 || subrounds < 1 || subrounds > 32) fail(SCLAP_EINVAL, "args");
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);
        if (!in_range(g.n, part_inout, nblocks, sc)) fail(SCLAP_EINVAL, "part out of range");
        GraphTotals t = graph_totals(g, sc, true);
        if (t.max_wdeg > INT32_MAX) fail(SCLAP_EOVERFLOW, "weighted degree");
        CK(cudaMalloc(&backup, (g.n ? g.n : 1) * sizeof(int32_t)));
        CK(cudaMemcpyAsync(backup, part_inout, g.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        LPConfig cfg{};
        cfg.g = g;
        cfg.lab = part_inout;
        cfg.nW = nblocks;
        cfg.B = B;
        cfg.refine = true;
        cfg.seed = seed;
        cfg.rounds = rounds;
        cfg.S = subrounds;
        int rd = lp_run(cfg, sc, nullptr, nullptr);
        CK(cudaStreamSynchronize(s));
        if (rounds_done) *rounds_done = rd;
    });
    if (rc != SCLAP_OK && backup && gp) {
        cudaMemcpyAsync(part_inout, backup, gp->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
    }
    if (backup) cudaFree(backup);
    return rc;
}

int sclap_refine(const sclap_graph *gp, int32_t k, double eps, int32_t rounds, int32_t subrounds,
                 uint64_t seed, int32_t *part_inout, int64_t *cut_out, int64_t *block_w_out,
                 int32_t *rounds_done, void *stream) {
    if (!gp || k < 1 || !(eps >= 0)) return SCLAP_EINVAL;
    int64_t cV = 0;
    int rc = guarded([&] {
        Scratch sc(as_stream(stream));
        DGraph g = view(gp);
        validate_graph(g, sc);
        cV = graph_totals(g, sc).cV;
    });
    if (rc) return rc;
    rc = sclap_refine_bound(gp, k, lmax_of(cV, k, eps), rounds, subrounds, seed, part_inout,
                            rounds_done, stream);
    if (rc) return rc;
    if (cut_out || block_w_out) {
        int64_t cut = 0;
        rc = sclap_cut(gp, part_inout, k, &cut, block_w_out, stream);
        if (cut_out) *cut_out = cut;
    }
    return rc;
}

int sclap_refine_learned(const sclap_graph *gp, int32_t k, double eps, int32_t rounds,
                         int32_t subrounds, uint64_t seed, const uint16_t *net, float z_min,
                         int32_t full_every, int32_t *part_inout, int64_t *cut_out,
                         int64_t *block_w_out, int32_t *rounds_done, int64_t *visited_out,
                         float *trace_x, uint8_t *trace_y, void *stream) {
    cudaStream_t s = as_stream(stream);
    int32_t *backup = nullptr;
    int rc = guarded([&] {
        if (!gp || (!part_inout && gp->n > 0)) fail(SCLAP_EINVAL, "null");
        if (k < 1 || !(eps >= 0) || rounds < 0 || subrounds < 1 || subrounds > 32 ||
            full_every < 1)
            fail(SCLAP_EINVAL, "args");
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);
        if (!in_range(g.n, part_inout, k, sc)) fail(SCLAP_EINVAL, "part out of range");
        GraphTotals t = graph_totals(g, sc, true);
        if (t.max_wdeg > INT32_MAX) fail(SCLAP_EOVERFLOW, "weighted degree");
        CK(cudaMalloc(&backup, (g.n ? g.n : 1) * sizeof(int32_t)));
        CK(cudaMemcpyAsync(backup, part_inout, g.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        int64_t *W = sc.get<int64_t>(k);
        Gate gt{};
        gt.g = g;
        gt.lab = part_inout;
        gt.W = W;
        gt.Lmax = lmax_of(t.cV, k, eps);
        gt.net = net;
        gt.z_min = z_min;
        gt.full_every = full_every;
        gt.rounds = rounds;
        gt.trace_x = trace_x;
        gt.trace_y = trace_y;
        gt.unit = t.sum_w == g.nnz;  // weights are >= 1, so a sum of nnz means all are 1
        gate_init(gt, sc);
        LPConfig cfg{};
        cfg.g = g;
        cfg.lab = part_inout;
        cfg.nW = k;
        cfg.B = gt.Lmax;
        cfg.refine = true;
        cfg.seed = seed;
        cfg.rounds = rounds;
        cfg.S = subrounds;
        cfg.before_round = [&](int r, const uint8_t **active) {
            return gate_round(gt, r, active, s);
        };
        cfg.visit_best = gt.vb;
        cfg.visit_own = gt.vo;
        int rd = lp_run(cfg, sc, nullptr, W);
        gate_finish(gt, rd, s);
        unsigned long long vis[2] = {0, 0};
        CK(cudaMemcpyAsync(vis, gt.visited, sizeof(vis), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (rounds_done) *rounds_done = rd;
        if (visited_out) *visited_out = (int64_t)(vis[0] + (unsigned long long)gt.nfull * vis[1]);
    });
    if (rc != SCLAP_OK && backup && gp) {
        cudaMemcpyAsync(part_inout, backup, gp->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
    }
    if (backup) cudaFree(backup);
    if (rc) return rc;
    if (cut_out || block_w_out) {
        int64_t cut = 0;
        rc = sclap_cut(gp, part_inout, k, &cut, block_w_out, stream);
        if (cut_out) *cut_out = cut;
    }
    return rc;
}

int sclap_mlp_score(const float *x, int64_t N, const uint16_t *net, float *z_out, void *stream) {
    return guarded([&] {
        if (N < 0 || (N > 0 && (!x || !net || !z_out))) fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        mlp_score(x, N, net, z_out, s);
        CK(cudaStreamSynchronize(s));
    });
}

int sclap_mlp_loss_grad(const float *x, const uint8_t *y, int64_t N, const float *params,
                        int32_t bf16_in, float *grad_out, double *loss_out, void *stream) {
    return guarded([&] {
        if (N < 0 || !params || !grad_out || (N > 0 && (!x || !y))) fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        double *d_loss = sc.zeros<double>(1);
        CK(cudaMemsetAsync(grad_out, 0, kMlpParams * sizeof(float), s));
        mlp_loss_grad(x, y, nullptr, N, params, grad_out, d_loss, bf16_in != 0, s);
        double l = 0;
        CK(cudaMemcpyAsync(&l, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (loss_out) *loss_out = l;
    });
}

int sclap_mlp_train(const float *x, const uint8_t *y, int64_t N, float *params, int32_t epochs,
                    int32_t batch, float lr, uint64_t seed, double *loss_out, void *stream) {
    return guarded([&] {
        if (N < 1 || N > INT32_MAX || !x || !y || !params || epochs < 0 || batch < 1 || !(lr > 0))
            fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        const int sms = dev_info().sms;
        uint64_t *keys = sc.get<uint64_t>(N);
        int32_t *perm = sc.get<int32_t>(N);
        int64_t *idx = sc.get<int64_t>(N);
        float *grad = sc.get<float>(kMlpParams);
        double *d_loss = sc.zeros<double>(1);
        for (int e = 0; e < epochs; e++) {
            k_shuffle_keys<<<sms * 4, 256, 0, s>>>(N, seed, e, keys, perm);
            LAUNCHED();
            radix_sort_pairs(keys, perm, N, 64, sc);
            k_widen<<<sms * 4, 256, 0, s>>>(N, perm, idx);
            LAUNCHED();
            for (int64_t b0 = 0; b0 < N; b0 += batch) {
                const int64_t nb = std::min<int64_t>(batch, N - b0);
                CK(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s));
                mlp_loss_grad(x, y, idx + b0, nb, params, grad, d_loss, true, s);
                mlp_sgd(params, grad, lr, s);
            }
        }
        CK(cudaMemsetAsync(d_loss, 0, sizeof(double), s));
        CK(cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), s));
        mlp_loss_grad(x, y, nullptr, N, params, grad, d_loss, true, s);
        double l = 0;
        CK(cudaMemcpyAsync(&l, d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (loss_out) *loss_out = l;
    });
}

int sclap_inject_alloc_failure(int64_t after) {
    if (after < -1) return SCLAP_EINVAL;
    set_alloc_failure((long long)after);
    return SCLAP_OK;
}

int sclap_wait_selftest(int64_t limit_cycles) {
    int got = SCLAP_OK;
    const int rc = guarded([&] {
        if (limit_cycles < 0) fail(SCLAP_EINVAL, "limit");
        Scratch sc(nullptr);
        got = barrier_selftest((long long)limit_cycles, sc);
    });
    return rc != SCLAP_OK ? rc : got;
}

int sclap_mlp_pack_bf16(const float *params, uint16_t *net_out, void *stream) {
    return guarded([&] {
        if (!params || !net_out) fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        mlp_pack_bf16(params, net_out, s);
        CK(cudaStreamSynchronize(s));
    });
}

int sclap_cut(const sclap_graph *gp, const int32_t *part, int32_t k, int64_t *cut_out,
              int64_t *block_w_out, void *stream) {
    return guarded([&] {
        if (!gp || (!part && gp->n > 0) || k < 1) fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);  // entry ids index part: checked before the cut kernel
        if (!in_range(g.n, part, k, sc)) fail(SCLAP_EINVAL, "part out of range");
        int64_t *d_cut = sc.get<int64_t>(1);
        int64_t *d_bw = sc.get<int64_t>(k);
        cut_impl(g, part, k, 1, nullptr, d_cut, d_bw, sc);
        int64_t c = 0;
        CK(cudaMemcpyAsync(&c, d_cut, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        if (block_w_out)
            CK(cudaMemcpyAsync(block_w_out, d_bw, k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (cut_out) *cut_out = c;
    });
}

int contract_graph(const sclap_graph *gp, const int32_t *labels, sclap_graph_owned *coarse_out,
                   int32_t *f2c_out, void *stream) {
    return guarded([&] {
        if (!gp || !coarse_out || (gp->n > 0 && (!labels || !f2c_out))) fail(SCLAP_EINVAL, "null");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);
        if (!in_range(g.n, labels, g.n, sc)) fail(SCLAP_EINVAL, "label out of range");
        GraphTotals t = graph_totals(g, sc);
        check_totals_cluster(t);
        CoarseGraph cg;
        contract_impl(g, labels, f2c_out, &cg, nullptr, sc);
        CK(cudaStreamSynchronize(s));
        coarse_out->n = cg.n;
        coarse_out->nnz = cg.nnz;
        coarse_out->xadj = cg.xadj;
        coarse_out->adjncy = cg.adjncy;
        coarse_out->adjwgt = cg.adjwgt;
        coarse_out->vwgt = cg.vwgt;
    });
}

int sclap_graph_copy_out(const sclap_graph_owned *g, int64_t *xadj, int32_t *adjncy,
                         int32_t *adjwgt, int32_t *vwgt, void *stream) {
    return guarded([&] {
        if (!g || !xadj || (g->n > 0 && !vwgt) || (g->nnz > 0 && (!adjncy || !adjwgt)))
            fail(SCLAP_EINVAL, "null");
        cudaStream_t s = as_stream(stream);
        CK(cudaMemcpyAsync(xadj, g->xadj, (g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        if (g->nnz > 0) {
            CK(cudaMemcpyAsync(adjncy, g->adjncy, g->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(adjwgt, g->adjwgt, g->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        }
        if (g->n > 0)
            CK(cudaMemcpyAsync(vwgt, g->vwgt, g->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        CK(cudaStreamSynchronize(s));
    });
}

void sclap_graph_free(sclap_graph_owned *g) {
    if (!g) return;
    cudaFree(g->xadj);
    cudaFree(g->adjncy);
    cudaFree(g->adjwgt);
    cudaFree(g->vwgt);
    std::memset(g, 0, sizeof(*g));
}

int project_partition(int64_t n_fine, const int32_t *f2c, const int32_t *coarse_part,
                      int32_t *fine_part_out, void *stream) {
    return guarded([&] {
        if (n_fine < 0) fail(SCLAP_EINVAL, "n");
        if (n_fine > 0 && (!f2c || !coarse_part || !fine_part_out)) fail(SCLAP_EINVAL, "null");
        cudaStream_t s = as_stream(stream);
        project_impl(n_fine, f2c, coarse_part, fine_part_out, s);
        CK(cudaStreamSynchronize(s));
    });
}

int sclap_initial_partition(const sclap_graph *gp, int32_t k, int64_t B, int32_t P, int32_t rounds,
                            int32_t subrounds, uint64_t seed, int32_t *part_out, int64_t *cuts_out,
                            int64_t *maxbw_out, int32_t *best_out, void *stream) {
    return guarded([&] {
        if (!gp || (!part_out && gp->n > 0) || k < 1 || P < 1 || rounds < 0 || subrounds < 1 ||
            subrounds > 32)
            fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        DGraph g = view(gp);
        validate_graph(g, sc);
        GraphTotals t = graph_totals(g, sc, true);
        if (t.max_wdeg > INT32_MAX) fail(SCLAP_EOVERFLOW, "weighted degree");
        InitResult r = initial_impl(g, k, B, P, rounds, subrounds, seed, part_out, sc);
        if (cuts_out) std::memcpy(cuts_out, r.cuts.data(), P * sizeof(int64_t));
        if (maxbw_out) std::memcpy(maxbw_out, r.maxbw.data(), P * sizeof(int64_t));
        if (best_out) *best_out = r.best;
    });
}

int sclap_refine_batched(const sclap_batch *b, int32_t k, double eps, int32_t rounds,
                         int32_t subrounds, int32_t nruns, const int32_t *run_graph,
                         const uint64_t *seeds, int32_t *parts_out, int64_t *cuts_out,
                         int64_t *maxbw_out, void *stream) {
    return guarded([&] {
        if (!b || b->ngraphs < 1 || !b->graphs || k < 1 || !(eps >= 0) || rounds < 0 ||
            subrounds < 1 || subrounds > 32 || nruns < 1 || !run_graph || !seeds)
            fail(SCLAP_EINVAL, "args");
        cudaStream_t s = as_stream(stream);
        Scratch sc(s);
        std::vector<DGraph> G;
        std::vector<int64_t> bound;
        for (int32_t i = 0; i < b->ngraphs; i++) {
            DGraph g = view(&b->graphs[i]);
            validate_graph(g, sc);
            G.push_back(g);
            bound.push_back(lmax_of(graph_totals(g, sc).cV, k, eps));
        }
        std::vector<int32_t> rg(run_graph, run_graph + nruns);
        int64_t total = 0;
        for (int32_t r : rg) {
            if (r < 0 || r >= b->ngraphs) fail(SCLAP_EINVAL, "run_graph");
            total += G[r].n;
        }
        if (total > 0 && !parts_out) fail(SCLAP_EINVAL, "parts_out");
        BatchResult br = batched_impl(G, bound, rg, std::vector<uint64_t>(seeds, seeds + nruns), k,
                                      rounds, subrounds, parts_out, sc);
        if (cuts_out) std::memcpy(cuts_out, br.cuts.data(), nruns * sizeof(int64_t));
        if (maxbw_out) std::memcpy(maxbw_out, br.maxbw.data(), nruns * sizeof(int64_t));
    });
}

namespace {

// Coarse node c inherits the block of its members (all members of a
// constrained cluster share one block).
__global__ void k_inherit(int64_t n, const int32_t *f2c, const int32_t *fine, int32_t *coarse) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        coarse[f2c[v]] = fine[v];
}

}  // namespace

// The multilevel scheme; with seed_part (host or device int32[n], k blocks)
// one V-cycle seeded by it.
static int multilevel_call(const sclap_graph *gp, const sclap_ml_params *p,
                           const int32_t *seed_part, int32_t *part_out, sclap_ml_stats *st_out,
                           void *stream) {
    return guarded([&] {
        if (!gp || !p || (!part_out && gp->n > 0)) fail(SCLAP_EINVAL, "null");
        if (p->k < 1 || !(p->eps >= 0) || p->cluster_rounds < 0 || p->refine_rounds < 0 ||
            p->subrounds < 1 || p->subrounds > 32 || p->init_seeds < 1 || p->init_rounds < 0)
            fail(SCLAP_EINVAL, "params");
        cudaStream_t s = as_stream(stream);
        Scratch top(s);
        const int64_t n = gp->n, nnz = gp->nnz;
        if (n < 0 || nnz < 0 || n > INT32_MAX) fail(SCLAP_EINVAL, "size");
        DGraph g0 = view(gp);
        if (n > 0 && !is_device_ptr(gp->xadj)) {
            // host input: copy the graph to the device inside the call
            int64_t *x = top.get<int64_t>(n + 1);
            int32_t *a = top.get<int32_t>(nnz);
            int32_t *w = top.get<int32_t>(nnz);
            int32_t *c = top.get<int32_t>(n);
            CK(cudaMemcpyAsync(x, gp->xadj, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            if (nnz) {
                CK(cudaMemcpyAsync(a, gp->adjncy, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
                CK(cudaMemcpyAsync(w, gp->adjwgt, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            }
            CK(cudaMemcpyAsync(c, gp->vwgt, n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            g0 = DGraph{n, nnz, x, a, w, c};
        }
        const bool part_on_device = is_device_ptr(part_out);
        validate_graph(g0, top);
        GraphTotals t0 = graph_totals(g0, top);
        check_totals_cluster(t0);
        const int64_t lmax = lmax_of(t0.cV, p->k, p->eps);
        const int64_t U = p->U > 0 ? p->U : std::max<int64_t>(t0.maxc, t0.cV / (10 * (int64_t)p->k));
        if (U < t0.maxc) fail(SCLAP_EINVAL, "U < max c(v)");
        int maxl = p->max_levels > 0 ? p->max_levels : 32;
        if (maxl > SCLAP_MAX_LEVELS) maxl = SCLAP_MAX_LEVELS;

        sclap_ml_stats st;
        std::memset(&st, 0, sizeof(st));
        std::vector<DGraph> G{g0};
        std::vector<int32_t *> F;   // f2c per level
        std::vector<int32_t *> CP;  // V-cycle: the seed partition on every level
        if (seed_part) {
            int32_t *cp0 = top.get<int32_t>(n ? n : 1);
            CK(cudaMemcpyAsync(cp0, seed_part, n * sizeof(int32_t),
                               is_device_ptr(seed_part) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyHostToDevice, s));
            if (!in_range(n, cp0, p->k, top)) fail(SCLAP_EINVAL, "part out of range");
            CP.push_back(cp0);
        }
        int L = 0;
        while (G[L].n >= p->n_stop && L + 1 < maxl && G[L].n > 0) {
            const DGraph &g = G[L];
            Scratch tmp(s);
            int32_t *lab = tmp.get<int32_t>(g.n);
            LPConfig cfg{};
            cfg.g = g;
            cfg.lab = lab;
            cfg.nW = g.n;
            cfg.B = U;
            cfg.refine = false;
            cfg.seed = level_seed(p->seed, L);
            cfg.rounds = p->cluster_rounds;
            cfg.S = p->subrounds;
            cfg.cp = seed_part ? CP[L] : nullptr;
            cfg.degree_order = p->degree_order != 0;
            int rd = 0;
            if (cfg.rounds > 0) rd = lp_run(cfg, tmp, nullptr, nullptr);
            else identity_labels(g.n, lab, s);
            pack_isolated(g, cfg.cp, U, lab, tmp);
            st.cluster_rounds_done[L] = rd;
            int32_t *f2c = top.get<int32_t>(g.n);
            CoarseGraph cg;
            contract_impl(g, lab, f2c, &cg, &top, tmp);
            if (cg.n == g.n) break;  // no shrink: the level is dropped
            if (seed_part) {
                int32_t *cpc = top.get<int32_t>(cg.n ? cg.n : 1);
                k_inherit<<<dev_info().sms * 4, 256, 0, s>>>(g.n, f2c, CP[L], cpc);
                LAUNCHED();
                CP.push_back(cpc);
            }
            F.push_back(f2c);
            DGraph c{cg.n, cg.nnz, cg.xadj, cg.adjncy, cg.adjwgt, cg.vwgt};
            G.push_back(c);
            L++;
            if (20 * G[L].n > 19 * G[L - 1].n) break;  // stalled (< 5% shrink)
        }
        // initial partition of the coarsest graph
        int32_t *cur = top.get<int32_t>(G[L].n ? G[L].n : 1);
        if (seed_part) {  // the inherited partition, refined like every level
            CK(cudaMemcpyAsync(cur, CP[L], G[L].n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
            Scratch tmp(s);
            LPConfig cfg{};
            cfg.g = G[L];
            cfg.lab = cur;
            cfg.nW = p->k;
            cfg.B = lmax;
            cfg.refine = true;
            cfg.seed = level_seed(p->seed, L);
            cfg.rounds = p->init_rounds;
            cfg.S = p->subrounds;
            if (cfg.rounds > 0) lp_run(cfg, tmp, nullptr, nullptr);
            int64_t *d_c = tmp.get<int64_t>(1);
            int64_t *d_b = tmp.get<int64_t>(p->k);
            cut_impl(G[L], cur, p->k, 1, nullptr, d_c, d_b, tmp);
            std::vector<int64_t> cbw(p->k);
            CK(cudaMemcpyAsync(&st.init_cut, d_c, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(cbw.data(), d_b, p->k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            st.init_best = -1;
            st.init_maxbw = 0;
            for (int64_t x : cbw) st.init_maxbw = std::max(st.init_maxbw, x);
        } else {
            InitResult ir = initial_impl(G[L], p->k, lmax, p->init_seeds, p->init_rounds,
                                         p->subrounds, level_seed(p->seed, L), cur, top);
            st.init_best = ir.best;
            st.init_cut = ir.cuts.empty() ? 0 : ir.cuts[ir.best];
            st.init_maxbw = ir.maxbw.empty() ? 0 : ir.maxbw[ir.best];
        }
        // uncoarsening: projection and r rounds of refinement per level
        for (int l = L - 1; l >= 0; l--) {
            int32_t *fp = top.get<int32_t>(G[l].n);
            project_impl(G[l].n, F[l], cur, fp, s);
            cur = fp;
            Scratch tmp(s);
            LPConfig cfg{};
            cfg.g = G[l];
            cfg.lab = cur;
            cfg.nW = p->k;
            cfg.B = lmax;
            cfg.refine = true;
            cfg.seed = level_seed(p->seed, l);
            cfg.rounds = p->refine_rounds;
            cfg.S = p->subrounds;
            st.refine_rounds_done[l] = lp_run(cfg, tmp, nullptr, nullptr);
        }
        // final cut and balance
        int64_t *d_cut = top.get<int64_t>(1);
        int64_t *d_bw = top.get<int64_t>(p->k);
        cut_impl(g0, cur, p->k, 1, nullptr, d_cut, d_bw, top);
        std::vector<int64_t> bw(p->k);
        CK(cudaMemcpyAsync(&st.cut, d_cut, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(bw.data(), d_bw, p->k * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(part_out, cur, n * sizeof(int32_t),
                           part_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int64_t x : bw) st.maxbw = std::max(st.maxbw, x);
        st.levels = L + 1;
        for (int l = 0; l <= L; l++) {
            st.n[l] = G[l].n;
            st.nnz[l] = G[l].nnz;
        }
        st.U = U;
        st.lmax = lmax;
        if (st_out) *st_out = st;
    });
}

int partition_multilevel(const sclap_graph *gp, const sclap_ml_params *p, int32_t *part_out,
                         sclap_ml_stats *st_out, void *stream) {
    return multilevel_call(gp, p, nullptr, part_out, st_out, stream);
}

int sclap_vcycle(const sclap_graph *gp, const sclap_ml_params *p, int32_t *part_inout,
                 sclap_ml_stats *st_out, void *stream) {
    if (!gp || !p || (!part_inout && gp->n > 0)) return SCLAP_EINVAL;
    return multilevel_call(gp, p, part_inout, part_inout, st_out, stream);
}

// ---------------------------------------------------------------- profiling

void sclap_prof_enable(int on) {
    ProfState &P = prof();
    P.on = on != 0;
    if (P.on && !P.d_counts) {
        cudaMalloc(&P.d_counts, 2 * sizeof(unsigned long long));
        cudaMemset(P.d_counts, 0, 2 * sizeof(unsigned long long));
    }
}

void sclap_prof_reset(void) {
    ProfState &P = prof();
    cudaDeviceSynchronize();
    for (auto &pr : P.pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    P.pending.clear();
    P.propose_launches = 0;
    P.propose_ms = 0;
    if (P.d_counts) cudaMemset(P.d_counts, 0, 2 * sizeof(unsigned long long));
}

int sclap_prof_read(sclap_prof *out) {
    return guarded([&] {
        ProfState &P = prof();
        CK(cudaDeviceSynchronize());
        for (auto &pr : P.pending) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, pr.first, pr.second));
            P.propose_ms += ms;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        P.pending.clear();
        unsigned long long c[2] = {0, 0};
        if (P.d_counts) CK(cudaMemcpy(c, P.d_counts, sizeof(c), cudaMemcpyDeviceToHost));
        out->propose_launches = P.propose_launches;
        out->propose_ms = P.propose_ms;
        out->entries_scanned = (int64_t)c[0];
        out->nodes_visited = (int64_t)c[1];
        out->propose_bytes = 12.0 * (double)c[0] + 24.0 * (double)c[1];
        out->kernel_launches = P.kernel_launches;
        out->graph_launches = P.graph_launches;
    });
}

}  // extern "C"

