// Forward pass (Sec. III-B, Algorithm 2, Eq. 2), loads and power (Eq. 1),
// capacitance gradients and output gathers.
#include "kern_common.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// startpoints: (P, Q) = (SP, 1 - SP); TR = input TR (tr_mode 0) or 2PQ (tr_mode 1)
__global__ void k_init_start(const float *__restrict__ sp_in, const float *__restrict__ tr_in, float4 *pq, float *tr,
                             int64_t ns, int tr_mode, const uint32_t *epoch) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const pair_ff a = pair_of(sp_in[k]);
    pq[k] = pair_store(a, epoch[0] & 1u);
    tr[k] = tr_mode ? pair_tr(a) : tr_in[k];
}

// one thread per cell of one level: gather the fanin (P, Q) pairs, evaluate
// the cell's pair, write it and TR_model = 2PQ (Eq. 2) for its output net
__global__ void k_fwd_level(const uint4 *__restrict__ fanin, float4 *pq, float *tr, int32_t c0, int32_t c1,
                            int64_t ns, OpTable ops, const uint32_t *epoch) {
    int32_t c = c0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= c1) return;
    const uint4 r = fanin[c];
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    pair_ff x[4];
    gather_ff<false>(pq, r, k, x);
    const pair_ff o = cell_pair(k, op_tt(ops, op), x);
    pq[ns + c] = pair_store(o, epoch[0] & 1u);
    tr[ns + c] = pair_tr(o);
}

// Eq. 1 loads: C_load = wire + DFF D caps + sum of the input pin caps of the driven cells
__global__ void k_cload(const float *__restrict__ base, const int32_t *__restrict__ fptr,
                        const int32_t *__restrict__ fedge, const float *__restrict__ pincap, float *cload, int64_t nn) {
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    float c = base[n];
    for (int32_t e = fptr[n]; e < fptr[n + 1]; e++) c += pincap[fedge[e] >> 2];
    cload[n] = c;
}

__global__ void k_set_pincap(const int32_t *__restrict__ cells, const float *__restrict__ caps,
                             const int32_t *__restrict__ cell_of_user, float *pincap, int32_t n, int64_t nc) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t u = cells ? cells[i] : i;   // no index list: cells in cell-line order
    if (u >= 0 && u < nc) pincap[cell_of_user[u]] = caps[i];
}

__device__ __forceinline__ double warp_sum(double v) { return warp_sum_f64(v); }

// power partials: a fixed grid and a fixed per-thread stride make the FP64
// summation order independent of timing, so the result is reproducible
__global__ void __launch_bounds__(kPowerThreads) k_power_partials(const float *__restrict__ tr,
                                                                  const float *__restrict__ beta,
                                                                  const float *__restrict__ cload, double *partials,
                                                                  int64_t nn) {
    // each term alpha C rounded once to binary32 (rel. 6e-8), the sum in FP64: one
    // conversion and one FP64 add per net, on a part whose FP64 pipe is narrow
    double s = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += (int64_t)gridDim.x * blockDim.x) {
        const float a = beta ? __fmul_rn(tr[n], beta[n]) : tr[n];
        s += (double)__fmul_rn(a, cload[n]);
    }
    __shared__ double sh[kPowerThreads / 32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kPowerThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kPowerThreads) k_power_final(const double *__restrict__ partials, int nb, double K,
                                                               double *out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partials[i];
    __shared__ double sh[kPowerThreads / 32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < kPowerThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) *out = K * t;
    }
}

// The output gradients that do not go through the adjoint, in one launch: blocks [0, bp) take
// d P / d pincap (user cell order: K times the alpha of the cell's inputs), the next bc blocks
// d P / d C_load (user net order: K alpha), the rest d P / d TR_in (startpoint order: K beta
// C_load when the startpoint TR is an input, tr_mode 0).  alpha: TR_model, or the hybrid TR
// beta * TR_model as k_hybrid stores it.  The block's role is uniform over the block.
__global__ void k_cap_grads(const uint4 *__restrict__ fanin, const float *__restrict__ alpha,
                            const float *__restrict__ beta, const float *__restrict__ cload,
                            const int32_t *__restrict__ net_of_user, const int32_t *__restrict__ cell_of_user, float K,
                            int tr_mode, float *gpin, float *gcl, float *gtr, int64_t nc, int64_t nn, int64_t ns,
                            unsigned bp, unsigned bc, OpTable ops) {
    const unsigned b = blockIdx.x;
    if (b < bp) {
        const int64_t u = (int64_t)b * blockDim.x + threadIdx.x;
        if (u < nc) gpin[u] = grad_pincap_of(fanin, alpha, cell_of_user, K, u, ops);
    } else if (b < bp + bc) {
        const int64_t u = (int64_t)(b - bp) * blockDim.x + threadIdx.x;
        if (u < nn) gcl[u] = grad_cload_of(alpha, net_of_user, K, u);
    } else {
        const int64_t k = (int64_t)(b - bp - bc) * blockDim.x + threadIdx.x;
        if (k < ns) gtr[k] = grad_tr_in_of(beta, cload, K, tr_mode, k);
    }
}

__global__ void k_gather_f32(const float *__restrict__ src, const int32_t *__restrict__ idx, float *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}
__global__ void k_gather_u32(const uint32_t *__restrict__ src, const int32_t *__restrict__ idx, uint32_t *dst,
                             int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}
__global__ void k_sp_user(const float4 *__restrict__ pq, const int32_t *__restrict__ idx, float *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = untag(pq[idx[i]].x);
}
__global__ void k_trh_user(const float *__restrict__ tr, const float *__restrict__ beta,
                           const int32_t *__restrict__ idx, float *dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { int32_t m = idx[i]; dst[i] = beta[m] * tr[m]; }
}

}  // namespace

// 1-D grids for per-level kernels: blocks small enough that a level spreads
// over all SMs (the level, not the GPU, is the unit of parallel work)
static inline int level_block(int64_t n) {
    int b = 256;
    while (b > 32 && n < (int64_t)b * 304) b >>= 1;
    return b;
}

void launch_init_start(const DevDesign &d, int tr_mode, cudaStream_t s) {
    if (d.n_start == 0) return;
    k_init_start<<<(unsigned)cdiv(d.n_start, 256), 256, 0, s>>>(d.sp_in, d.tr_in, d.pq, d.tr, d.n_start, tr_mode,
                                                                 d.epoch);
}

void launch_fwd_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, cudaStream_t s) {
    if (c1 <= c0) return;
    int b = level_block(c1 - c0);
    k_fwd_level<<<(unsigned)cdiv(c1 - c0, b), b, 0, s>>>(d.fanin, d.pq, d.tr, c0, c1, d.n_start, ops, d.epoch);
}

void launch_cload(const DevDesign &d, cudaStream_t s) {
    if (d.n_nets == 0) return;
    k_cload<<<(unsigned)cdiv(d.n_nets, 256), 256, 0, s>>>(d.base_cap, d.fout_ptr, d.fout_edge, d.pincap, d.cload,
                                                          d.n_nets);
}

void launch_set_pincap(const DevDesign &d, const int32_t *cells, const float *caps, int32_t n, cudaStream_t s) {
    if (n <= 0) return;
    k_set_pincap<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(cells, caps, d.cell_of_user, d.pincap, n, d.n_cells);
}

void launch_power(const DevDesign &d, bool hybrid, double K, int slot, cudaStream_t s) {
    k_power_partials<<<kPowerBlocks, kPowerThreads, 0, s>>>(d.tr, hybrid ? d.beta : nullptr, d.cload, d.partials,
                                                            d.n_nets);
    k_power_final<<<1, kPowerThreads, 0, s>>>(d.partials, kPowerBlocks, K, d.power + slot);
}

void launch_cap_grads(const DevDesign &d, const OpTable &ops, bool hybrid, int tr_mode, double K,
                          float *grad_cload, float *grad_pincap, float *grad_tr_in, cudaStream_t s) {
    const float *beta = hybrid ? d.beta : nullptr;
    const float *alpha = hybrid ? d.trh : d.tr;   // trh = beta * TR_model, the same binary32 product
    const unsigned bp = grad_pincap ? (unsigned)cdiv(d.n_cells, 256) : 0u;
    const unsigned bc = grad_cload ? (unsigned)cdiv(d.n_nets, 256) : 0u;
    const unsigned bt = grad_tr_in ? (unsigned)cdiv(d.n_start, 256) : 0u;
    if (bp + bc + bt)
        k_cap_grads<<<bp + bc + bt, 256, 0, s>>>(d.fanin, alpha, beta, d.cload, d.net_of_user, d.cell_of_user,
                                                 (float)K, tr_mode, grad_pincap, grad_cload, grad_tr_in, d.n_cells,
                                                 d.n_nets, d.n_start, bp, bc, ops);
}

void launch_gather_f32(const float *src, const int32_t *idx, float *dst, int64_t n, cudaStream_t s) {
    if (n) k_gather_f32<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(src, idx, dst, n);
}
void launch_gather_u32(const uint32_t *src, const int32_t *idx, uint32_t *dst, int64_t n, cudaStream_t s) {
    if (n) k_gather_u32<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(src, idx, dst, n);
}
void launch_sp_user(const DevDesign &d, float *dst, cudaStream_t s) {
    if (d.n_nets) k_sp_user<<<(unsigned)cdiv(d.n_nets, 256), 256, 0, s>>>(d.pq, d.net_of_user, dst, d.n_nets);
}
void launch_trh_user(const DevDesign &d, float *dst, cudaStream_t s) {
    if (d.n_nets) k_trh_user<<<(unsigned)cdiv(d.n_nets, 256), 256, 0, s>>>(d.tr, d.beta, d.net_of_user, dst, d.n_nets);
}

}  // namespace dp
