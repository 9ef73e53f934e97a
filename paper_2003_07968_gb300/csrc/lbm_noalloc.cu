// lbm_noalloc.cu -- lbm_mass_noalloc: the FP64 mass reduction of the
// library for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or anything that allocates) at the
// point where they need a mass check: applications that reserve all device
// memory up front through their own allocator and forbid later
// allocations, or real-time loops that must not take the allocator's locks.
// For them this entry point reduces FP32 values they already own (a density
// field, say) into a result buffer they already own, and keeps its
// per-block partial sums in a fixed array in device global memory that
// belongs to the library module itself (kNoallocPartials doubles = 2 MiB per
// GPU that loads the library, held until the process exits).
//
// The reduction is the same two-level scheme as the handle's mass kernels:
// every block adds a fixed chunk of the input in FP64 and writes one
// partial; a second kernel adds the partials in block order, so the result
// does not depend on timing.  Every partial the second kernel reads was
// written by the first kernel of the same call, so nothing has to be cleared
// between calls.  All calls share the one array: calls whose kernels overlap
// on the GPU (different streams, or different host threads without ordering)
// race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pplbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int64_t kChunk = (int64_t)kThreads * kPerThread;  // values per block
constexpr int kNoallocPartials = LBM_NOALLOC_MAX_COUNT / kChunk;
static_assert((int64_t)kNoallocPartials * kChunk == LBM_NOALLOC_MAX_COUNT, "scratch size");

// The scratch array: module-scope device memory, no allocation per call.
static __device__ __align__(256) double g_partials[kNoallocPartials];

__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const float* __restrict__ v,
                                                              int64_t count, double* partials) {
    const int64_t begin = (int64_t)blockIdx.x * kChunk;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = begin + (int64_t)k * kThreads + threadIdx.x;
        if (i < count) acc += (double)__ldg(v + i);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < kThreads / 32 ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) partials[blockIdx.x] = acc;
    }
}

// Adds the partials in block order: each thread a strided share, then a
// fixed-order combination of the per-thread sums.
__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double* partials, int n,
                                                            double offset, double* out) {
    __shared__ double s[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc += partials[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = offset;
        for (int i = 0; i < kThreads; ++i) m += s[i];
        *out = m;
    }
}

// Device address of g_partials per device, looked up once with that device
// current (host code only sees a host-side stand-in for the symbol) and kept
// for the life of the process: a device reset would leave it stale, which
// the header states as a limit of the entry point.
std::mutex g_mu;
double* g_addr[128] = {nullptr};

}  // namespace

extern "C" int lbm_mass_noalloc(const float* values, int64_t count, double offset,
                                double* mass_out, void* stream) {
    if (!values || !mass_out || count < 1) return LBM_ERR_ARG;
    if (count > (int64_t)LBM_NOALLOC_MAX_COUNT) return LBM_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return LBM_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
                cudaGetLastError();
                return LBM_ERR_CUDA;
            }
            g_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_addr[dev];
    }
    const int nb = (int)((count + kChunk - 1) / kChunk);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_partial<<<nb, kThreads, 0, st>>>(values, count, scratch);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    k_noalloc_final<<<1, kThreads, 0, st>>>(scratch, nb, offset, mass_out);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
