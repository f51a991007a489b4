// learned.cu -- the learned active set of refinement (not in the paper: a
// scorer gates which nodes a refinement round visits; every full_every-th
// round and the last one visit all nodes) and the training kernels of its
// 6-32-32-1 scorer.
//
// Inference is bit-reproducible on a CPU: features and hidden outputs are
// rounded to bf16 (nearest, ties to even), every output starts from its bias
// and adds one fmaf per input in index order, and the gate compares the
// logit with z_min (no exponential).
#include "learned.cuh"
#include "prims.cuh"

namespace sclap {

// ---------------------------------------------------------------- bf16 and features

__device__ __forceinline__ float bf16_round(float f) {
    uint32_t u = __float_as_uint(f);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return __uint_as_float(u & 0xFFFF0000u);
}

__device__ __forceinline__ float bf16_value(uint16_t b) {
    return __uint_as_float((uint32_t)b << 16);
}

// log2 of x >= 1 in its piecewise-linear form e + (x - 2^e) / 2^e.
__device__ __forceinline__ float log2_feature(int64_t x) {
    const int e = 63 - __clzll((long long)x);
    const float scale = __uint_as_float((uint32_t)(127 - e) << 23);  // 2^-e, exact
    const float frac = __fmul_rn(__ll2float_rn(x - ((int64_t)1 << e)), scale);
    return __fadd_rn((float)e, frac);
}

// Weighted degree of every row: a warp takes 32 consecutive rows and sums
// each one with its lanes striding over the row's entries (coalesced), then
// one warp reduction per row.  The callers have checked that every weighted
// degree fits 31 bits, so 32-bit lane sums and the reduction cannot wrap.
__global__ void __launch_bounds__(256) k_row_sums(DGraph g, unsigned long long *wdeg) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < g.n;
         base += nw * 32) {
        const int64_t v = base + lane;
        const int64_t rs = v < g.n ? g.xadj[v] : 0, re = v < g.n ? g.xadj[v + 1] : 0;
        uint32_t mine = 0;
        for (int r = 0; r < 32; r++) {
            const int64_t s = __shfl_sync(0xffffffffu, rs, r), e = __shfl_sync(0xffffffffu, re, r);
            uint32_t sum = 0;
            for (int64_t i = s + lane; i < e; i += 32) sum += (uint32_t)__ldg(&g.adjwgt[i]);
            sum = __reduce_add_sync(0xffffffffu, sum);
            if (lane == r) mine = sum;
        }
        if (v < g.n) wdeg[v] = mine;
    }
}

// Movers with longer rows than this are scattered in pieces of this many
// entries, one CTA per piece, so one long row does not hold up the launch.
constexpr int kScatChunk = 2048;

// moved[v] = label changed since the previous call; prev = labels now.  When
// movers is given, the moved nodes with rows of <= kScatChunk entries are
// appended to movers (count in cnt[0]) and the pieces of longer rows to
// pieces as (v << 20) | piece (count in cnt[1]).
__global__ void k_moved(int64_t n, const int64_t *xadj, const int32_t *lab, int32_t *prev,
                        uint8_t *moved, uint8_t *trace_y, bool first, int32_t *movers,
                        int64_t *pieces, int32_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t n_r = (n + 31) & ~31ll;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_r;
         v += (int64_t)gridDim.x * blockDim.x) {
        uint8_t m = 0;
        int64_t deg = 0;
        if (v < n) {
            const int32_t l = lab[v];
            m = first ? 0 : (uint8_t)(l != prev[v]);
            moved[v] = m;
            prev[v] = l;
            if (trace_y) trace_y[v] = m;
            if (m && movers) deg = xadj[v + 1] - xadj[v];
        }
        if (movers) {
            const bool shortrow = m && deg <= kScatChunk;
            const unsigned b = __ballot_sync(0xffffffffu, shortrow);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&cnt[0], __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (shortrow) movers[base + __popc(b & ((1u << lane) - 1))] = (int32_t)v;
            if (m && deg > kScatChunk) {  // rare: one reservation per long row
                const int np = (int)((deg + kScatChunk - 1) / kScatChunk);
                const int pb = atomicAdd(&cnt[1], np);
                for (int q = 0; q < np; q++) pieces[pb + q] = (v << 20) | q;
            }
        }
    }
}

// Moved-neighbour counts: every mover adds 1 to each of its neighbours, so
// the cost follows the movers' rows, not the graph.  Short rows: one warp
// each; pieces of long rows: one CTA each.
__global__ void k_scatter_moved(DGraph g, const int32_t *movers, const int64_t *pieces,
                                const int32_t *cnt, int32_t *nmov) {
    const int nm = cnt[0], np = cnt[1];
    const int lane = threadIdx.x & 31;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nm;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = movers[i];
        for (int64_t e = g.xadj[v] + lane; e < g.xadj[v + 1]; e += 32)
            atomicAdd(&nmov[g.adjncy[e]], 1);
    }
    for (int64_t i = blockIdx.x; i < np; i += gridDim.x) {
        const int64_t it = pieces[i];
        const int64_t v = it >> 20;
        const int64_t e0 = g.xadj[v] + (it & ((1 << 20) - 1)) * kScatChunk;
        const int64_t e1 = min64(g.xadj[v + 1], e0 + kScatChunk);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) atomicAdd(&nmov[g.adjncy[e]], 1);
    }
}

// Scorer forward on one row of six bf16 features; params in shared memory
// (floats holding bf16 values).
__device__ __forceinline__ float mlp_forward(const float *P, const float *x) {
    float h1[32];
#pragma unroll
    for (int j = 0; j < 32; j++) {
        float acc = P[kMlpB1 + j];
#pragma unroll
        for (int i = 0; i < 6; i++) acc = __fmaf_rn(P[kMlpW1 + j * 6 + i], x[i], acc);
        h1[j] = bf16_round(acc > 0.0f ? acc : 0.0f);
    }
    float z = P[kMlpB3];
    for (int j = 0; j < 32; j++) {
        float acc = P[kMlpB2 + j];
#pragma unroll
        for (int i = 0; i < 32; i++) acc = __fmaf_rn(P[kMlpW2 + j * 32 + i], h1[i], acc);
        z = __fmaf_rn(P[kMlpW3 + j], bf16_round(acc > 0.0f ? acc : 0.0f), z);
    }
    return z;
}

// The same forward for two rows at once: every parameter read from shared
// memory (float4 / float2 vectors) feeds both rows, and each row keeps its
// own fmaf chain in index order, so each result equals mlp_forward's.
__device__ __forceinline__ void mlp_forward2(const float *P, const float *xa, const float *xb,
                                             float *za, float *zb) {
    float ha[32], hb[32];
#pragma unroll
    for (int j = 0; j < 32; j++) {
        float aa = P[kMlpB1 + j], ab = aa;
#pragma unroll
        for (int i = 0; i < 6; i += 2) {
            const float2 w = *reinterpret_cast<const float2 *>(&P[kMlpW1 + j * 6 + i]);
            aa = __fmaf_rn(w.x, xa[i], aa);
            ab = __fmaf_rn(w.x, xb[i], ab);
            aa = __fmaf_rn(w.y, xa[i + 1], aa);
            ab = __fmaf_rn(w.y, xb[i + 1], ab);
        }
        ha[j] = bf16_round(aa > 0.0f ? aa : 0.0f);
        hb[j] = bf16_round(ab > 0.0f ? ab : 0.0f);
    }
    float ya = P[kMlpB3], yb = ya;
#pragma unroll 2
    for (int j = 0; j < 32; j++) {
        float aa = P[kMlpB2 + j], ab = aa;
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
            const float4 w = *reinterpret_cast<const float4 *>(&P[kMlpW2 + j * 32 + i]);
            aa = __fmaf_rn(w.x, ha[i], aa);
            ab = __fmaf_rn(w.x, hb[i], ab);
            aa = __fmaf_rn(w.y, ha[i + 1], aa);
            ab = __fmaf_rn(w.y, hb[i + 1], ab);
            aa = __fmaf_rn(w.z, ha[i + 2], aa);
            ab = __fmaf_rn(w.z, hb[i + 2], ab);
            aa = __fmaf_rn(w.w, ha[i + 3], aa);
            ab = __fmaf_rn(w.w, hb[i + 3], ab);
        }
        const float w3 = P[kMlpW3 + j];
        ya = __fmaf_rn(w3, bf16_round(aa > 0.0f ? aa : 0.0f), ya);
        yb = __fmaf_rn(w3, bf16_round(ab > 0.0f ? ab : 0.0f), yb);
    }
    *za = ya;
    *zb = yb;
}
static_assert(kMlpW2 % 4 == 0 && kMlpW1 % 2 == 0, "vector reads of the parameters");

__device__ __forceinline__ void load_net(const uint16_t *net, float *P) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) P[i] = bf16_value(net[i]);
    __syncthreads();
}

// The six features of node v (zeros for a node without neighbours); returns
// its degree.
__device__ __forceinline__ int64_t node_features(const DGraph &g, const int32_t *lab,
                                                 const int64_t *W, int64_t Lmax,
                                                 const uint8_t *moved,
                                                 const unsigned long long *wdeg,
                                                 const int32_t *vb, const int32_t *vo,
                                                 const int32_t *nmov, int64_t v, float *f) {
    const int64_t deg = g.xadj[v + 1] - g.xadj[v];
#pragma unroll
    for (int i = 0; i < 6; i++) f[i] = 0.f;
    if (deg > 0) {
        const int32_t own = lab[v];
        // unit edge weights (wdeg null): the weighted degree is the degree
        const int64_t wb = vb[v], wo = vo[v], wd = wdeg ? (int64_t)wdeg[v] : deg;
        f[0] = bf16_round(log2_feature(1 + deg));
        f[1] = bf16_round(__fdiv_rn(__ll2float_rn(W[own]), __ll2float_rn(Lmax)));
        f[2] = bf16_round(__fdiv_rn(__ll2float_rn(wb - wo), __ll2float_rn(wd)));
        f[3] = moved[v] ? 1.0f : 0.0f;
        f[4] = bf16_round(__fdiv_rn(__int2float_rn(nmov[v]), __ll2float_rn(deg)));
        f[5] = bf16_round(__fdiv_rn(__ll2float_rn(wo), __ll2float_rn(wd)));
    }
    return deg;
}

// Features of every node (written to x when non-null) and, in gated rounds,
// the active flags (logit >= z_min); counts the visited rows.  vb / vo: the
// weight to the best eligible other block / own block that the node's latest
// visit saw (recorded by the propose kernels).  A CTA takes 2 * blockDim
// consecutive nodes per step, each thread two of them (v and v + blockDim).
__global__ void __launch_bounds__(256, 2)
    k_gate(DGraph g, const int32_t *lab, const int64_t *W, int64_t Lmax, const uint8_t *moved,
           const unsigned long long *wdeg, const int32_t *vb, const int32_t *vo,
           const int32_t *nmov, const uint16_t *net, float z_min, bool full, float *x_out,
           uint8_t *active, unsigned long long *visited) {
    __shared__ __align__(16) float P[kMlpParams];
    const bool score = !full && net;
    if (score) load_net(net, P);
    const int lane = threadIdx.x & 31;
    const int64_t chunk = 2 * (int64_t)blockDim.x;
    const int64_t nchunks = ceil_div<int64_t>(g.n, chunk);
    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
        const int64_t v[2] = {ci * chunk + threadIdx.x, ci * chunk + threadIdx.x + blockDim.x};
        float f[2][6];
        int64_t deg[2] = {0, 0};
#pragma unroll
        for (int q = 0; q < 2; q++) {
            if (v[q] < g.n) {
                deg[q] = node_features(g, lab, W, Lmax, moved, wdeg, vb, vo, nmov, v[q], f[q]);
                if (x_out) {
#pragma unroll
                    for (int i = 0; i < 6; i++) x_out[v[q] * 6 + i] = f[q][i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 6; i++) f[q][i] = 0.f;
            }
        }
        bool act[2] = {true, true};
        if (score) {
            float z[2];
            mlp_forward2(P, f[0], f[1], &z[0], &z[1]);
            act[0] = z[0] >= z_min;
            act[1] = z[1] >= z_min;
        }
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            if (v[q] < g.n) {
                active[v[q]] = act[q] ? 1 : 0;
                if (act[q] && deg[q] > 0) cnt++;
            }
        }
        cnt = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
        if (lane == 0 && cnt) atomicAdd(visited, (unsigned long long)cnt);
    }
}

__global__ void k_count_rows(DGraph g, unsigned long long *cnt) {
    const int64_t n_r = (g.n + 31) & ~31ll;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_r;
         v += (int64_t)gridDim.x * blockDim.x) {
        const bool r = v < g.n && g.xadj[v + 1] > g.xadj[v];
        const unsigned b = __ballot_sync(0xffffffffu, r);
        if ((threadIdx.x & 31) == 0 && b) atomicAdd(cnt, (unsigned long long)__popc(b));
    }
}

void gate_init(Gate &gt, Scratch &sc) {
    const int64_t n = gt.g.n;
    cudaStream_t s = sc.stream();
    const int sms = dev_info().sms;
    unsigned long long *wd = gt.unit ? nullptr : sc.zeros<unsigned long long>(n ? n : 1);
    gt.wdeg = (int64_t *)wd;
    gt.prev = sc.get<int32_t>(n ? n : 1);
    gt.moved = sc.zeros<uint8_t>(n ? n : 1);
    gt.active = sc.get<uint8_t>(n ? n : 1);
    gt.vb = sc.zeros<int32_t>(n ? n : 1);
    gt.vo = sc.zeros<int32_t>(n ? n : 1);
    gt.nmov = sc.get<int32_t>(n ? n : 1);
    gt.movers = sc.get<int32_t>(n ? n : 1);
    gt.pieces = sc.get<int64_t>(2 * (gt.g.nnz / kScatChunk) + 1);
    gt.nmovers = sc.get<int32_t>(2);
    gt.visited = sc.zeros<unsigned long long>(2);
    gt.nfull = 0;
    if (gt.g.nnz > 0 && !gt.unit) {
        k_row_sums<<<sms * 4, 256, 0, s>>>(gt.g, wd);
        LAUNCHED();
    }
    if (n > 0) {
        k_count_rows<<<sms * 4, 256, 0, s>>>(gt.g, gt.visited + 1);
        LAUNCHED();
    }
}

bool gate_round(Gate &gt, int r, const uint8_t **active, cudaStream_t s) {
    const int64_t n = gt.g.n;
    const int sms = dev_info().sms;
    const bool full =
        !gt.net || r == 0 || r % gt.full_every == gt.full_every - 1 || r == gt.rounds - 1;
    if (n > 0) {
        CK(cudaMemsetAsync(gt.nmovers, 0, 2 * sizeof(int32_t), s));
        k_moved<<<sms * 4, 256, 0, s>>>(n, gt.g.xadj, gt.lab, gt.prev, gt.moved,
                                        (gt.trace_y && r > 0) ? gt.trace_y + (size_t)(r - 1) * n
                                                               : nullptr,
                                        r == 0, gt.movers, gt.pieces, gt.nmovers);
        LAUNCHED();
    }
    float *x = gt.trace_x ? gt.trace_x + (size_t)r * n * 6 : nullptr;
    if (full && !x) {  // nothing to compute: every row is visited
        gt.nfull++;
        *active = nullptr;
        return true;
    }
    if (n > 0) {
        // neighbours that moved in round r - 1, scattered from its movers
        CK(cudaMemsetAsync(gt.nmov, 0, n * sizeof(int32_t), s));
        if (gt.g.nnz > 0 && r > 0) {
            k_scatter_moved<<<sms * 8, 256, 0, s>>>(gt.g, gt.movers, gt.pieces, gt.nmovers,
                                                    gt.nmov);
            LAUNCHED();
        }
        k_gate<<<sms * 4, 256, 0, s>>>(gt.g, gt.lab, gt.W, gt.Lmax, gt.moved,
                                       (const unsigned long long *)gt.wdeg, gt.vb, gt.vo,
                                       gt.nmov, gt.net, gt.z_min, full, x, gt.active,
                                       gt.visited);
        LAUNCHED();
    }
    *active = full ? nullptr : gt.active;
    return full;
}

void gate_finish(Gate &gt, int rounds_done, cudaStream_t s) {
    if (!gt.trace_y || rounds_done < 1 || gt.g.n == 0) return;
    const int sms = dev_info().sms;
    k_moved<<<sms * 4, 256, 0, s>>>(gt.g.n, gt.g.xadj, gt.lab, gt.prev, gt.moved,
                                    gt.trace_y + (size_t)(rounds_done - 1) * gt.g.n, false,
                                    nullptr, nullptr, nullptr);
    LAUNCHED();
}

// ---------------------------------------------------------------- scoring

__global__ void __launch_bounds__(256)
    k_score(const float *x, int64_t N, const uint16_t *net, float *z) {
    __shared__ float P[kMlpParams];
    load_net(net, P);
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N;
         s += (int64_t)gridDim.x * blockDim.x) {
        float f[6];
#pragma unroll
        for (int i = 0; i < 6; i++) f[i] = x[s * 6 + i];
        z[s] = mlp_forward(P, f);
    }
}

void mlp_score(const float *x, int64_t N, const uint16_t *net, float *z, cudaStream_t s) {
    if (N <= 0) return;
    k_score<<<dev_info().sms * 4, 256, 0, s>>>(x, N, net, z);
    LAUNCHED();
}

// ---------------------------------------------------------------- training

// Warp sum of a float, added by lane 0 to a shared accumulator.
__device__ __forceinline__ void warp_add(float v, float *dst) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(dst, v);
}

// Each lane takes one sample (lanes past the end contribute zeros); every
// gradient term is summed over the warp before one shared atomic; the CTA's
// sums go to grad with one global atomic per parameter.
constexpr int kTrainThreads = 128;

// BF16: the forward of inference (parameters rounded to bf16, hidden outputs
// ReLU then bf16, fp32 fmaf accumulation in index order) and the
// straight-through gradient (each rounding passed as the identity) with
// respect to the float master parameters; else the float network.
template <bool BF16>
__global__ void __launch_bounds__(kTrainThreads)
    k_loss_grad(const float *X, const uint8_t *y, const int64_t *idx, int64_t N, float inv_n,
                const float *prm, float *grad, double *loss) {
    __shared__ float P[kMlpParams];
    __shared__ float G[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        P[i] = BF16 ? bf16_round(prm[i]) : prm[i];
        G[i] = 0.0f;
    }
    __syncthreads();
    double lsum = 0.0;
    const int64_t N_r = (N + 31) & ~31ll;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N_r;
         q += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = q < N;
        const int64_t s = ok ? (idx ? idx[q] : q) : 0;
        float x[6];
#pragma unroll
        for (int i = 0; i < 6; i++) x[i] = ok ? X[s * 6 + i] : 0.0f;
        const float t = ok && y[s] ? 1.0f : 0.0f;
        float a1[32], h1[32], a2[32];
#pragma unroll
        for (int j = 0; j < 32; j++) {
            float acc = P[kMlpB1 + j];
#pragma unroll
            for (int i = 0; i < 6; i++) acc = fmaf(P[kMlpW1 + j * 6 + i], x[i], acc);
            a1[j] = acc;
            h1[j] = BF16 ? bf16_round(acc > 0.0f ? acc : 0.0f) : (acc > 0.0f ? acc : 0.0f);
        }
        float z = P[kMlpB3];
#pragma unroll 4
        for (int j = 0; j < 32; j++) {
            float acc = P[kMlpB2 + j];
#pragma unroll
            for (int i = 0; i < 32; i++) acc = fmaf(P[kMlpW2 + j * 32 + i], h1[i], acc);
            a2[j] = acc;
            const float r = acc > 0.0f ? acc : 0.0f;
            z = fmaf(P[kMlpW3 + j], BF16 ? bf16_round(r) : r, z);
        }
        if (ok) lsum += (double)((z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z))) - t * z);
        const float dz = ok ? (1.0f / (1.0f + expf(-z)) - t) * inv_n : 0.0f;
        warp_add(dz, &G[kMlpB3]);
        float d1[32];
#pragma unroll
        for (int i = 0; i < 32; i++) d1[i] = 0.0f;
        for (int j = 0; j < 32; j++) {
            const float h2 = BF16 ? bf16_round(a2[j] > 0.0f ? a2[j] : 0.0f)
                                  : (a2[j] > 0.0f ? a2[j] : 0.0f);
            warp_add(dz * h2, &G[kMlpW3 + j]);
            const float d2 = a2[j] > 0.0f ? dz * P[kMlpW3 + j] : 0.0f;
            warp_add(d2, &G[kMlpB2 + j]);
#pragma unroll
            for (int i = 0; i < 32; i++) {
                warp_add(d2 * h1[i], &G[kMlpW2 + j * 32 + i]);
                d1[i] = fmaf(d2, P[kMlpW2 + j * 32 + i], d1[i]);
            }
        }
#pragma unroll
        for (int j = 0; j < 32; j++) {
            const float dj = a1[j] > 0.0f ? d1[j] : 0.0f;
            warp_add(dj, &G[kMlpB1 + j]);
#pragma unroll
            for (int i = 0; i < 6; i++) warp_add(dj * x[i], &G[kMlpW1 + j * 6 + i]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x)
        if (G[i] != 0.0f) atomicAdd(&grad[i], G[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, d);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum * (double)inv_n);
}

void mlp_loss_grad(const float *X, const uint8_t *y, const int64_t *idx, int64_t N,
                   const float *prm, float *grad, double *d_loss, bool bf16_in, cudaStream_t s) {
    if (N <= 0) return;
    const int64_t blocks = std::min<int64_t>(ceil_div<int64_t>(N, kTrainThreads),
                                             (int64_t)dev_info().sms * 4);
    if (bf16_in)
        k_loss_grad<true><<<(unsigned)blocks, kTrainThreads, 0, s>>>(X, y, idx, N, 1.0f / (float)N,
                                                                     prm, grad, d_loss);
    else
        k_loss_grad<false><<<(unsigned)blocks, kTrainThreads, 0, s>>>(
            X, y, idx, N, 1.0f / (float)N, prm, grad, d_loss);
    LAUNCHED();
}

// bf16 bit patterns of float parameters, nearest even (the rounding of the
// scorer's features and hidden outputs).
__global__ void k_pack_bf16(const float *prm, uint16_t *net) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x)
        net[i] = (uint16_t)(__float_as_uint(bf16_round(prm[i])) >> 16);
}

void mlp_pack_bf16(const float *prm, uint16_t *net, cudaStream_t s) {
    k_pack_bf16<<<ceil_div(kMlpParams, 256), 256, 0, s>>>(prm, net);
    LAUNCHED();
}

__global__ void k_sgd(float *prm, const float *grad, float lr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x)
        prm[i] -= lr * grad[i];
}

void mlp_sgd(float *prm, const float *grad, float lr, cudaStream_t s) {
    k_sgd<<<ceil_div(kMlpParams, 256), 256, 0, s>>>(prm, grad, lr);
    LAUNCHED();
}

}  // namespace sclap
