// Lag-one mode of the batched path (tr_mode 2): every net carries SP and
// T = P(x_t != x_{t+1}) of a stationary two-state process, so two consecutive
// values follow q(a, b) with q(1,1) = P - T/2, q(0,0) = P(net=0) - T/2,
// q(0,1) = q(1,0) = T/2.  Under spatial independence a cell's output toggles
// with probability
//     T_y = sum over input pairs (a, b) of prod_i q_i(a_i, b_i) [f(a) != f(b)],
// its exact toggle probability on fanout-free circuits (an extension of Eq. 2,
// which it equals when every startpoint has T = 2P(1-P)).  SP is the
// multilinear pair of the other modes.  The power is K sum_n T_n C_n (Eq. 1).
//
// T_y is a fold over the 4^k joint input states, input 0 innermost: leaf m
// (digit i of m in base 4 = 2 a_i + b_i) holds [f(a) != f(b)], and each input
// folds four sub-results with its weights q_i.  Its derivatives are the same
// fold with one input's weights replaced by dq/dP = (-1, 0, 0, 1) or
// dq/dT = (-1/2, 1/2, 1/2, -1/2).  The reverse pass carries two adjoints per
// net (of P and of T); edge contributions are float2 in fanout-CSR order, so a
// net sums one contiguous range, without atomics, as in the other modes.
#include "kern_batch.cuh"

namespace dp {
namespace {

// q weights of a stored pair and its T
__device__ __forceinline__ void lag1_weights(const float2 &pv, float t, float (&w)[4]) {
    const pair_ff a = pair_get(pv);
    const float h = 0.5f * t;
    w[0] = (a.q.hi + a.q.lo) - h;
    w[1] = h;
    w[2] = h;
    w[3] = (a.p.hi + a.p.lo) - h;
}

// the fold, with input `sub` (if 0 <= sub < K) weighted by dv instead of its own weights
template <int K>
__device__ __forceinline__ float lag1_fold(uint32_t tt, const float (&w)[4][4], int sub, const float (&dv)[4]) {
    constexpr int M = 1 << (2 * K);
    float v[M];
#pragma unroll
    for (int m = 0; m < M; m++) {
        int a = 0, b = 0;
#pragma unroll
        for (int i = 0; i < K; i++) {
            const int dgt = (m >> (2 * i)) & 3;
            a |= (dgt >> 1) << i;
            b |= (dgt & 1) << i;
        }
        v[m] = (((tt >> a) ^ (tt >> b)) & 1u) ? 1.f : 0.f;
    }
#pragma unroll
    for (int i = 0; i < K; i++) {
        float c[4];
#pragma unroll
        for (int d = 0; d < 4; d++) c[d] = i == sub ? dv[d] : w[i][d];
#pragma unroll
        for (int m = 0; m < (M >> (2 * (i + 1))); m++)
            v[m] = fmaf(c[3], v[4 * m + 3], fmaf(c[2], v[4 * m + 2], fmaf(c[1], v[4 * m + 1], c[0] * v[4 * m])));
    }
    return v[0];
}

__device__ __forceinline__ float lag1_t(int k, uint32_t tt, const float (&w)[4][4], int sub, const float (&dv)[4]) {
    switch (k) {
        case 0: return 0.f;   // a constant never toggles
        case 1: return lag1_fold<1>(tt, w, sub, dv);
        case 2: return lag1_fold<2>(tt, w, sub, dv);
        case 3: return lag1_fold<3>(tt, w, sub, dv);
        default: return lag1_fold<4>(tt, w, sub, dv);
    }
}

__device__ __forceinline__ void gather_lag1(const float2 *pq, const float *tq, const uint4 &r, int k, int64_t S,
                                            int64_t s, pair_ff (&x)[4], float (&w)[4][4]) {
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
    float2 v[4];
    float t[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v[j] = j < k ? pq[(int64_t)n[j] * S + s] : make_float2(0.f, 0.f);
        t[j] = j < k ? tq[(int64_t)n[j] * S + s] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        x[j] = pair_get(v[j]);
        lag1_weights(v[j], t[j], w[j]);
    }
}

__global__ void k_fwdl_start(const float *__restrict__ sp_in, const float *__restrict__ tr_in, float2 *pq, float *tq,
                             int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pq[i] = make_float2(sp_in[i], 0.f);
    tq[i] = tr_in[i];
}

__global__ void k_fwdl_level(const uint4 *__restrict__ fanin, float2 *pq, float *tq, int32_t c0, int32_t c1,
                             int64_t ns, int64_t S, OpTable ops) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    const float none[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    const int64_t cf = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    const uint4 rf = cf < c1 ? fanin[cf] : make_uint4(0, 0, 0, 0);   // static: before the wait
    pdl_wait();
    for (int64_t c = cf; c < c1; c += step) {
        const uint4 r = c == cf ? rf : fanin[c];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        const uint32_t tt = op_tt(ops, op);
        pair_ff x[4];
        float w[4][4];
        gather_lag1(pq, tq, r, k, S, s, x, w);
        pq[(ns + c) * S + s] = cell_p(k, tt, x);
        tq[(ns + c) * S + s] = lag1_t(k, tt, w, -1, none);
    }
}

// reverse level: the net's adjoints (gP from its fanout range, gT from its range
// plus the direct term K_s C), then per input edge the contributions
// (gP dP/dP_j + gT dT/dP_j, gT dT/dT_j)
__global__ void k_bwdl_level(const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr,
                             const int4 *__restrict__ efpos, const float2 *__restrict__ pq,
                             const float *__restrict__ tq, const float *__restrict__ cload,
                             const float *__restrict__ dcl, const float *__restrict__ ks, float2 *gfo2, int32_t c0,
                             int32_t c1, int64_t ns, int64_t S, OpTable ops) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    pdl_wait();
    const float Ks = ks[s];
    const float dP[4] = {-1.f, 0.f, 0.f, 1.f};
    const float dT[4] = {-0.5f, 0.5f, 0.5f, -0.5f};
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t c = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y; c < c1; c += step) {
        const int64_t n = ns + c;
        float gp = 0.f, gt = 0.f;
        for (int32_t e = fptr[n]; e < fptr[n + 1]; e++) {
            const float2 g = gfo2[(int64_t)e * S + s];
            gp += g.x;
            gt += g.y;
        }
        gt += Ks * cl_of(cload, dcl, n, S, s);
        const uint4 r = fanin[c];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        const uint32_t tt = op_tt(ops, op);
        pair_ff x[4];
        float w[4][4], p[4], q[4], d[4];
        gather_lag1(pq, tq, r, k, S, s, x, w);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            p[j] = x[j].p.hi + x[j].p.lo;
            q[j] = x[j].q.hi + x[j].q.lo;
        }
        cell_partials(k, tt, p, q, d);
        const int4 ep = efpos[c];
        const int pos[4] = {ep.x, ep.y, ep.z, ep.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (j >= k) break;
            const float dtp = lag1_t(k, tt, w, j, dP), dtt = lag1_t(k, tt, w, j, dT);
            gfo2[(int64_t)pos[j] * S + s] = make_float2(fmaf(gp, d[j], gt * dtp), gt * dtt);
        }
    }
}

__global__ void k_bwdl_start(const int32_t *__restrict__ fptr, const float *__restrict__ cload,
                             const float *__restrict__ dcl, const float *__restrict__ ks,
                             const float2 *__restrict__ gfo2, float *gsp, float *gtr, int64_t ns, int64_t S) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    pdl_wait();
    const float Ks = ks[s];
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t k = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; k < ns; k += step) {
        float gp = 0.f, gt = 0.f;
        for (int32_t e = fptr[k]; e < fptr[k + 1]; e++) {
            const float2 g = gfo2[(int64_t)e * S + s];
            gp += g.x;
            gt += g.y;
        }
        gsp[k * S + s] = gp;
        gtr[k * S + s] = gt + Ks * cl_of(cload, dcl, k, S, s);
    }
}

}  // namespace

void launch_fwdl(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl, BatchShape sh,
                 cudaStream_t s) {
    const int64_t S = b.S;
    if (d.n_start)
        k_fwdl_start<<<(unsigned)bcdiv(d.n_start * S, 256), 256, 0, s>>>(b.sp_in, b.tr_in, b.pq, b.tq, d.n_start * S);
    sh = fit_shape(sh, S);
    const dim3 blk((unsigned)sh.bx, (unsigned)sh.by);
    for (int l = 1; l <= d.n_levels; l++) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        if (c1 > c0)
            launch_pdl(k_fwdl_level, bgrid(S, sh, c1 - c0), blk, s, d.fanin, b.pq, b.tq, c0, c1, d.n_start, S, ops);
    }
}

void launch_bwdl(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl, BatchShape sh,
                 cudaStream_t s) {
    const int64_t S = b.S;
    sh = fit_shape(sh, S);
    const dim3 blk((unsigned)sh.bx, (unsigned)sh.by);
    for (int l = d.n_levels; l >= 1; l--) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        if (c1 > c0)
            launch_pdl(k_bwdl_level, bgrid(S, sh, c1 - c0), blk, s, d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos,
                       b.pq, b.tq, d.cload, b.dcl, b.ks, b.gfo2, c0, c1, d.n_start, S, ops);
    }
    if (d.n_start)
        launch_pdl(k_bwdl_start, bgrid(S, sh, d.n_start), blk, s, d.fout_ptr, d.cload, b.dcl, b.ks, b.gfo2, b.gsp,
                   b.gtr, d.n_start, S);
}

}  // namespace dp
