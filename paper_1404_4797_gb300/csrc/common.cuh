// common.cuh -- shared definitions of the CUDA path (device helpers, error
// handling, stream-ordered scratch memory, launch accounting).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <vector>

#include "sclap.h"

namespace sclap {

// ---------------------------------------------------------------- errors

struct Error {
    int code;
    const char *what;
};

[[noreturn]] inline void fail(int code, const char *what) { throw Error{code, what}; }

inline void cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(SCLAP_ENOMEM, what);
    fail(SCLAP_ECUDA, what);
}
#define CK(x) ::sclap::cuda_check((x), #x)

// ---------------------------------------------------------------- launch accounting

void count_launch();
void count_graph_launch();
// After every kernel launch: record it and surface launch-configuration errors.
#define LAUNCHED() do { ::sclap::count_launch(); CK(cudaGetLastError()); } while (0)

// ---------------------------------------------------------------- device helpers

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output function (Steele, Lea, Flood 2014).
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t node_hash(uint64_t seed, int32_t round, uint32_t v) {
    return mix64(seed ^ ((uint64_t)(uint32_t)(round + 1) << 32) ^ (uint64_t)v);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

template <typename T>
__host__ __device__ __forceinline__ T ceil_div(T a, T b) { return (a + b - 1) / b; }

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------- scratch memory

// Stream-ordered device scratch taken from a private memory pool that keeps
// freed blocks cached (so repeated calls do not pay for cudaMalloc).
void *scratch_alloc(size_t bytes, cudaStream_t s);
void set_alloc_failure(long long after);
void scratch_free(void *p, cudaStream_t s);

// RAII list of scratch blocks released (stream-ordered) when it goes out of scope.
class Scratch {
   public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    ~Scratch() { release(); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    template <typename T>
    T *get(size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        void *p = scratch_alloc((bytes + 255) & ~size_t(255), s_);
        blocks_.push_back(p);
        return static_cast<T *>(p);
    }
    template <typename T>
    T *zeros(size_t count) {
        T *p = get<T>(count);
        CK(cudaMemsetAsync(p, 0, (count ? count : 1) * sizeof(T), s_));
        return p;
    }
    void release() {
        for (void *p : blocks_) scratch_free(p, s_);
        blocks_.clear();
    }
    cudaStream_t stream() const { return s_; }

   private:
    cudaStream_t s_;
    std::vector<void *> blocks_;
};

// Device properties cached per process.
struct DevInfo {
    int device;
    int sms;
};
const DevInfo &dev_info();

// ---------------------------------------------------------------- graph view

struct DGraph {
    int64_t n, nnz;
    const int64_t *xadj;
    const int32_t *adjncy, *adjwgt, *vwgt;
};

// ---------------------------------------------------------------- profiling

struct ProfState {
    bool on = false;
    int64_t propose_launches = 0;
    int64_t kernel_launches = 0;
    int64_t graph_launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;  // recorded, not yet read
    double propose_ms = 0;
    // device-side counters of entries / nodes processed by the timed kernel
    unsigned long long *d_counts = nullptr;  // [2]: entries, nodes
};
ProfState &prof();
void prof_begin(cudaStream_t s, cudaEvent_t *b, cudaEvent_t *e);
void prof_end(cudaStream_t s, cudaEvent_t b, cudaEvent_t e);

}  // namespace sclap
