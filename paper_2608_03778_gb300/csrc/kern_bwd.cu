// Reverse pass (Sec. III-E, Eq. 7; Eq. 6 for the paper's hybrid rule).
// Nets are visited in reverse level order.  A net's adjoint is the sum of the
// contributions its fanout cells left on their input edges plus its local
// term; a cell then writes one contribution per input edge.  Edge
// contributions are stored in fanout-CSR order (each cell knows the fanout
// position of its input edges), so a net sums one contiguous range.  Every
// fanout cell of a level-l net sits on a level above l, so the range is
// complete when the net is visited: a gather replaces atomic scatters, and
// the result is reproducible bit for bit.
#include "kern_common.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ float fanout_sum(const int32_t *__restrict__ fptr, const float *__restrict__ gfo,
                                            int64_t n) {
    return fanout_sum_l2(gfo, fptr[n], fptr[n + 1]);
}

// grad_mode 0: g = acc + local; 1: g = beta (acc + local) (Eq. 6); 2: g = acc + beta local
__device__ __forceinline__ float combine(int grad_mode, float acc, float local, const float *beta, int64_t n) {
    return adj_combine(grad_mode, acc, local, grad_mode ? beta[n] : 1.f);
}

__global__ void k_bwd_level(const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr,
                            const int4 *__restrict__ efpos, const float4 *__restrict__ pq,
                            const float *__restrict__ cload, const float *__restrict__ beta, float *gnet,
                            float *gfo, int32_t c0, int32_t c1, int64_t ns, int grad_mode, float K, OpTable ops) {
    int32_t c = c0 + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= c1) return;
    const int64_t n = ns + c;
    const float acc = fanout_sum(fptr, gfo, n);
    // local term: d(K C 2P(1-P))/dP = K C (2 - 4P) = 2 K C (Q - P)
    const float g = combine(grad_mode, acc, adj_local(K, cload[n], pair_qmp(pq[n])), beta, n);
    gnet[n] = g;
    const uint4 r = fanin[c];
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    float p[4], q[4], d[4];
    gather_pairs(pq, r, k, p, q);
    cell_partials(k, op_tt(ops, op), p, q, d);
    const int4 ep = efpos[c];
    if (k > 0) gfo[ep.x] = g * d[0];
    if (k > 1) gfo[ep.y] = g * d[1];
    if (k > 2) gfo[ep.z] = g * d[2];
    if (k > 3) gfo[ep.w] = g * d[3];
}

__global__ void k_bwd_start(const int32_t *__restrict__ fptr, const float4 *__restrict__ pq,
                            const float *__restrict__ cload, const float *__restrict__ beta, float *gnet,
                            const float *gfo, int64_t ns, int grad_mode, int tr_mode, float K, float *out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const float acc = fanout_sum(fptr, gfo, k);
    // a startpoint has a local SP term only when its TR is derived from its SP (tr_mode 1)
    const float local = tr_mode ? adj_local(K, cload[k], pair_qmp(pq[k])) : 0.f;
    const float g = combine(grad_mode, acc, local, beta, k);
    gnet[k] = g;
    if (out) out[k] = g;
}

}  // namespace

static inline int level_block(int64_t n) {
    int b = 256;
    while (b > 32 && n < (int64_t)b * 304) b >>= 1;
    return b;
}

void launch_bwd_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, int grad_mode, float K,
                      cudaStream_t s) {
    if (c1 <= c0) return;
    int b = level_block(c1 - c0);
    k_bwd_level<<<(unsigned)cdiv(c1 - c0, b), b, 0, s>>>(d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos, d.pq,
                                                         d.cload, d.beta, d.gnet, d.gfo, c0, c1, d.n_start,
                                                         grad_mode, K, ops);
}

void launch_bwd_start(const DevDesign &d, int grad_mode, int tr_mode, float K, float *grad_sp_in, cudaStream_t s) {
    if (d.n_start == 0) return;
    int b = level_block(d.n_start);
    k_bwd_start<<<(unsigned)cdiv(d.n_start, b), b, 0, s>>>(d.fout_ptr, d.pq, d.cload, d.beta, d.gnet, d.gfo,
                                                           d.n_start, grad_mode, tr_mode, K, grad_sp_in);
}

}  // namespace dp
