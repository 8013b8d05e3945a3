// Allocation-free degraded volume average.
//
// Some callers cannot call cudaMalloc: code running under an allocator it
// does not own (a host framework that forbids raw device allocations, or a
// pre-sized memory pool), code that must not allocate once a run is under
// way (real-time or long-running jobs that pre-size everything), or drivers
// that cannot tolerate the implicit synchronisation of cudaMalloc/cudaFree.
// For them this file offers one reduction that allocates nothing: its
// per-block partial sums live in a fixed array of device memory compiled into
// the library, and the caller supplies inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "fatiguefft.h"

namespace {

constexpr int kNaBlocks = 304;   // 2 blocks per SM of a 152-SM GB300
constexpr int kNaMaxComp = 81;   // enough for the 81 entries of a tangent
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// Scratch shared by every call on a device: kNaMaxComp x kNaBlocks partial
// sums (194,688 bytes).  Every slot a call reads is written earlier in the
// same call, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_na_partials[kNaMaxComp * kNaBlocks];

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {nullptr};

__global__ void k_na_partials(const double* X, const double* phi, size_t N, double k_res,
                              double* part) {
    __shared__ double sh[32];
    const int c = blockIdx.y;
    double a = 0.0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
        const double om = 1.0 - phi[v];
        a += (om * om + k_res) * X[(size_t)c * N + v];
    }
    const double s = fatfft::block_sum<kNaThreads>(a, sh);
    if (threadIdx.x == 0) part[(size_t)c * kNaBlocks + blockIdx.x] = s;
}

__global__ void k_na_finish(const double* part, double scale, double* out) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int i = threadIdx.x; i < kNaBlocks; i += blockDim.x)
        a += part[(size_t)blockIdx.x * kNaBlocks + i];
    const double s = fatfft::block_sum<kNaThreads>(a, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s * scale;
}

}  // namespace

extern "C" fft_status degraded_average_noalloc(const double* X, int ncomp, const double* phi,
                                               size_t N, double k_res, double* out,
                                               void* cuda_stream) {
    if (!X || !phi || !out || N == 0) return FFT_ERR_ARG;
    if (ncomp < 1 || ncomp > kNaMaxComp) return FFT_ERR_ARG;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return FFT_ERR_CUDA;
    double* part = nullptr;
    {
        // First call on this device: look up the device address of the
        // scratch array (its name is only a placeholder in host code).  The
        // address is kept for the life of the process; it does not survive
        // a reset of the device (cudaDeviceReset, a re-created primary
        // context), after which the module is loaded again elsewhere.
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_partials) != cudaSuccess || !p)
                return FFT_ERR_CUDA;
            g_na_ptr[dev] = (double*)p;
        }
        part = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_na_partials<<<dim3(kNaBlocks, ncomp), kNaThreads, 0, s>>>(X, phi, N, k_res, part);
    k_na_finish<<<ncomp, kNaThreads, 0, s>>>(part, 1.0 / (double)N, out);
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}
