// noalloc.cu -- cut and block weights of a partition without any device
// allocation.  Some callers cannot let a library allocate: loops with a
// latency budget (cudaMalloc and cudaFree can synchronise the whole device),
// and programs whose device memory is handed out by their own pool or
// allocator, which would not see or account for memory a library takes on
// its own.  This entry point keeps its accumulators in a file-scope device
// array instead of taking memory per call.
#include <cstring>
#include <mutex>

#include "contract.cuh"

namespace {

constexpr int kNoAllocMaxK = 65536;

// [0] cut accumulator, [1] count of block ids outside [0, k), [2 .. 2 + k)
// block weights (k <= kNoAllocMaxK).  Every GPU that loads the library holds
// this array until the process exits; all calls share it, so calls that
// overlap on the GPU race.
static __device__ __align__(256) unsigned long long g_cut_scratch[2 + kNoAllocMaxK];

std::mutex g_mu;
unsigned long long *g_ptr[64];
int g_sms[64];
bool g_ready[64];

// Device address of g_cut_scratch for the current device (the host-side name
// is only a stand-in).  Looked up once per device, with that device current.
int scratch_for_current_device(unsigned long long **ptr, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SCLAP_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cut_scratch) != cudaSuccess) return SCLAP_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SCLAP_ECUDA;
        g_ptr[dev] = static_cast<unsigned long long *>(p);
        g_sms[dev] = n;
        g_ready[dev] = true;
    }
    *ptr = g_ptr[dev];
    *sms = g_sms[dev];
    return SCLAP_OK;
}

}  // namespace

extern "C" int sclap_cut_noalloc(const sclap_graph *gp, const int32_t *part, int32_t k,
                                 int64_t *cut_out, int64_t *block_w_out, void *stream) {
    if (!gp || k < 1 || gp->n < 0 || gp->nnz < 0) return SCLAP_EINVAL;
    if (k > kNoAllocMaxK) return SCLAP_EINVAL;  // beyond the static accumulator
    if (gp->n > 0 && !part) return SCLAP_EINVAL;
    unsigned long long *acc = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&acc, &sms);
    if (rc != SCLAP_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    try {
        // The array keeps the previous call's sums: clear what this call uses.
        // Clearing 2 + k slots is enough because the block-weight kernel skips
        // (and counts in slot 1) every id outside [0, k), so its writes stay
        // inside slots [2, 2 + k).
        CK(cudaMemsetAsync(acc, 0, (2 + (size_t)k) * sizeof(unsigned long long), s));
        sclap::DGraph g{gp->n, gp->nnz, gp->xadj, gp->adjncy, gp->adjwgt, gp->vwgt};
        sclap::cut_launch(g, part, k, acc, acc + 2, acc + 1, s, sms);
        unsigned long long c[2] = {0, 0};
        CK(cudaMemcpyAsync(c, acc, sizeof(c), cudaMemcpyDeviceToHost, s));
        if (block_w_out)
            CK(cudaMemcpyAsync(block_w_out, acc + 2, (size_t)k * sizeof(int64_t),
                               cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (c[1]) return SCLAP_EINVAL;  // a block id outside [0, k)
        if (cut_out) *cut_out = (int64_t)c[0];
    } catch (const sclap::Error &e) {
        return e.code;
    }
    return SCLAP_OK;
}
