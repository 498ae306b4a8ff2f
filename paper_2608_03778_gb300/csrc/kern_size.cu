// Gradient-weighted sizing score (Eq. 8) and its top-k ranking.
//
// For cell line u with output net y:  S_u = |dP/dP_sw| * P_sw,
//   P_sw = K * alpha_y * C_load,y   (alpha: TR_model, or the hybrid TR after a hybrid reverse pass)
//   mode 0: dP/dP_sw read as the SP adjoint of y (the global sensitivity the reverse pass leaves);
//   mode 1: the chain rule through Eq. 2, adjoint / (2 - 4 SP_y), |2 - 4 SP_y| floored at 1e-6.
// Scores are non-negative floats, so their bit patterns order like unsigned
// integers: the k-th largest is found by a radix select over 8-bit digits,
// most significant first (integer histograms, so the counts and the threshold
// are exact), and the cells at or above the threshold are collected for the
// final ordering on the host.
#include "kern_common.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void k_scores(const int32_t *__restrict__ cell_of_user, const float4 *__restrict__ pq,
                         const float *__restrict__ alpha, const float *__restrict__ gnet,
                         const float *__restrict__ cload, int64_t ns, int64_t nc, float K, int mode, float *out) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nc) return;
    const int64_t y = ns + cell_of_user[u];
    const float psw = K * alpha[y] * cload[y];
    float sens = fabsf(gnet[y]);
    if (mode == 1) {
        // 2 - 4 SP = 2 (P(net=0) - P): from the float-float pair, without the cancellation
        // of forming 2 - 4 SP from a rounded SP near SP = 0.5
        float d = 2.f * pair_qmp(pq[y]);
        if (fabsf(d) < 1e-6f) d = d < 0.f ? -1e-6f : 1e-6f;
        sens = fabsf(gnet[y] / d);
    }
    const float s = sens * psw;
    out[u] = s > 0.f ? s : 0.f;   // +0 for zero, negative zero or NaN: the bits then order like the values
}

__global__ void k_radix_hist(const float *__restrict__ s, int64_t n, uint32_t prefix, uint32_t mask, int shift,
                             unsigned *hist) {
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = __float_as_uint(s[i]);
        if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

__global__ void k_radix_collect(const float *__restrict__ s, int64_t n, uint32_t thr, int32_t *idx,
                                unsigned *count, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || __float_as_uint(s[i]) < thr) return;
    const unsigned at = atomicAdd(count, 1u);
    if ((int64_t)at < cap) idx[at] = (int32_t)i;
}

}  // namespace

void launch_scores(const DevDesign &d, bool hybrid, float K, int mode, float *out, cudaStream_t s) {
    if (d.n_cells == 0) return;
    k_scores<<<(unsigned)cdiv(d.n_cells, 256), 256, 0, s>>>(d.cell_of_user, d.pq, hybrid ? d.trh : d.tr, d.gnet,
                                                           d.cload, d.n_start, d.n_cells, K, mode, out);
}

void launch_radix_hist(const float *scores, int64_t n, uint32_t prefix, uint32_t mask, int shift, unsigned *hist,
                       cudaStream_t s) {
    const int64_t blocks = cdiv(n > 0 ? n : 1, 256);
    k_radix_hist<<<(unsigned)(blocks < 1216 ? blocks : 1216), 256, 0, s>>>(scores, n, prefix, mask, shift, hist);
}

void launch_radix_collect(const float *scores, int64_t n, uint32_t thr, int32_t *idx, unsigned *count, int64_t cap,
                          cudaStream_t s) {
    if (n > 0) k_radix_collect<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(scores, n, thr, idx, count, cap);
}

}  // namespace dp
