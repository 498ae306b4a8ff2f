// dp_power_noalloc: the FP64 switching-power reduction (Eq. 1) over
// caller-supplied device arrays, for callers that cannot allocate device
// memory.  Its scratch (one FP64 partial sum per block) lives in a file-scope
// __device__ array instead of a cudaMalloc'd buffer.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "diffpower.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 32;
constexpr int64_t kChunk = (int64_t)kThreads * kPerThread;  // nets reduced by one block
constexpr int kMaxBlocks = 4096;                             // partial sums the scratch holds
constexpr int kMaxDevices = 64;

// Shared by every call on a device and kept until the library is unloaded.
// Each call overwrites partials [0, blocks) before reading them, so nothing
// needs clearing; two calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_partials[kMaxBlocks];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// block b sums alpha_n C_n over nets [b * kChunk, (b + 1) * kChunk) in a fixed order
__global__ void __launch_bounds__(kThreads) k_partials(const float *__restrict__ tr, const float *__restrict__ beta,
                                                       const float *__restrict__ cload, int64_t n,
                                                       double *partials) {
    const int64_t base = (int64_t)blockIdx.x * kChunk;
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < kPerThread; i++) {
        const int64_t k = base + (int64_t)i * kThreads + threadIdx.x;
        if (k < n) {
            double a = (double)tr[k];
            if (beta) a *= (double)beta[k];
            s += a * (double)cload[k];
        }
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_final(const double *__restrict__ partials, int nb, double K,
                                                    double *watts) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *watts = K * s;
}

}  // namespace

extern "C" dp_status dp_power_noalloc(int device, const float *tr, const float *beta, const float *cload, int64_t n,
                                      double vdd, double fclk, double *watts, void *cuda_stream) {
    if (n < 0 || !watts || (n > 0 && (!tr || !cload))) return DP_EINVAL;
    if (!(vdd > 0) || !(fclk > 0) || !std::isfinite(vdd) || !std::isfinite(fclk)) return DP_EINVAL;
    if (n > (int64_t)kMaxBlocks * kChunk) return DP_EUNSUPPORTED;  // beyond the scratch capacity
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return DP_ECUDA;
    if (device < 0 || device >= ndev || device >= kMaxDevices) return DP_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return DP_ECUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return DP_ECUDA;
    dp_status st = DP_OK;
    double *scratch = nullptr;
    {
        // once per device, with that device current: the device address of the scratch
        // array (its name in host code only stands in for it)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch[device]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess) {
                st = DP_ECUDA;
            } else {
                g_scratch[device] = static_cast<double *>(p);
            }
        }
        scratch = g_scratch[device];
    }
    if (st == DP_OK) {
        // Each launch's own status decides the result.  An error the caller left pending on
        // this thread is neither reported as this call's nor cleared, so the caller still
        // finds it with cudaGetLastError().
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        const int nb = (int)((n + kChunk - 1) / kChunk);
        const double K = 0.5 * vdd * vdd * fclk * 1e-15;
        if (nb > 0) {
            void *args[] = {(void *)&tr, (void *)&beta, (void *)&cload, (void *)&n, (void *)&scratch};
            if (cudaLaunchKernel((const void *)k_partials, dim3(nb), dim3(kThreads), args, 0, s) != cudaSuccess)
                st = DP_ECUDA;
        }
        if (st == DP_OK) {
            const double *partials = scratch;
            int nblocks = nb;
            void *args[] = {(void *)&partials, (void *)&nblocks, (void *)&K, (void *)&watts};
            if (cudaLaunchKernel((const void *)k_final, dim3(1), dim3(kThreads), args, 0, s) != cudaSuccess)
                st = DP_ECUDA;
        }
    }
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}
