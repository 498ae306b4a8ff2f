// Device helpers shared by the batched kernels (kern_batch.cu, kern_lag1.cu):
// per-net state is stored scenario-innermost, value[n * S + s].
#pragma once
#include "kern_common.cuh"

namespace dp {

__host__ __device__ inline int64_t bcdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// the stored float-float P of a net and its pair (P, 1 - P)
__device__ __forceinline__ pair_ff pair_get(const float2 &v) {
    const ff p{v.x, v.y};
    const ff t = fast_two_sum(1.f, -v.x);   // exact: 0 <= P.hi <= 1
    return pair_ff{p, fast_two_sum(t.hi, __fsub_rn(t.lo, v.y))};
}
__device__ __forceinline__ float2 p_set(const pair_ff &a) { return make_float2(a.p.hi, a.p.lo); }

__device__ __forceinline__ void gather_ffb(const float2 *pq, const uint4 &r, int k, int64_t S, int64_t s,
                                           pair_ff (&x)[4]) {
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
    float2 v[4];
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = j < k ? pq[(int64_t)n[j] * S + s] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; j++) x[j] = pair_get(v[j]);
}

// P(out = 1) of a cell alone: the multilinear extension of its truth table over
// the fanin pairs, folded in float-float.  The batched path stores only P and
// re-derives each fanin's Q = 1 - P where it is read, so every pair sums to 1
// to about 4e-15 afresh and no drift of P + Q can build up along paths: the
// complementary sum and the renormalisation of the single-scenario path would
// be thrown away here.
template <int K>
__device__ __forceinline__ ff ml_p(uint32_t tt, const pair_ff (&x)[4]) {
    ff v[1 << K];
    // input 0 over a pair of table entries (f(0), f(1)): 0, Q, P, or exactly 1
#pragma unroll
    for (int m = 0; m < (1 << (K - 1)); m++) {
        const bool a1 = (tt >> (2 * m)) & 1u, b1 = (tt >> (2 * m + 1)) & 1u;
        v[m] = a1 ? (b1 ? ff_make(1.f) : x[0].q) : (b1 ? x[0].p : ff_make(0.f));
    }
#pragma unroll
    for (int i = 1; i < K; i++) {
#pragma unroll
        for (int m = 0; m < (1 << (K - 1 - i)); m++) v[m] = fold_pq(x[i], v[2 * m], v[2 * m + 1]);
    }
    return v[0];
}

__device__ __forceinline__ float2 cell_p(int k, uint32_t tt, const pair_ff (&x)[4]) {
    ff p;
    switch (k) {
        case 0: p = ff_make((tt & 1u) ? 1.f : 0.f); break;
        case 1: p = ml_p<1>(tt, x); break;
        case 2: p = ml_p<2>(tt, x); break;
        case 3: p = ml_p<3>(tt, x); break;
        default: p = ml_p<4>(tt, x); break;
    }
    return make_float2(p.hi, p.lo);
}

// binary32 (P, Q) of a cell's inputs for the partial derivatives
__device__ __forceinline__ void gather32(const float2 *pq, const uint4 &r, int k, int64_t S, int64_t s,
                                         float (&p)[4], float (&q)[4]) {
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
    float2 v[4];
#pragma unroll
    for (int j = 0; j < 4; j++) v[j] = j < k ? pq[(int64_t)n[j] * S + s] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const pair_ff a = pair_get(v[j]);
        p[j] = a.p.hi + a.p.lo;
        q[j] = a.q.hi + a.q.lo;
    }
}

// Q - P of a stored net, rounded once to binary32
__device__ __forceinline__ float qmp32(const float2 &v) {
    const pair_ff a = pair_get(v);
    const ff d = ff_add(a.q, ff{-a.p.hi, -a.p.lo});
    return d.hi + d.lo;
}

// switching activity of net n in scenario s: the input TR at a startpoint in
// tr_mode 0, else TR_model = 2 P Q (Eq. 2) rounded once to binary32.  In the
// lag-one mode (tr_mode 2) every net's TR is stored, and the callers pass that
// array in tr_in's place.
__device__ __forceinline__ float alpha32(const float2 *pq, const float *tr_in, int64_t n, int64_t ns, int64_t S,
                                         int64_t s, int tr_mode) {
    if (tr_mode == 2 || (n < ns && tr_mode == 0)) return tr_in[n * S + s];
    return pair_tr(pair_get(pq[n * S + s]));
}

// the load of net n in scenario s: C_load plus the scenario's sizing delta (if any)
__device__ __forceinline__ float cl_of(const float *cload, const float *dcl, int64_t n, int64_t S, int64_t s) {
    return dcl ? cload[n] + dcl[n * S + s] : cload[n];
}


// Programmatic dependent launch of the level chains: a level kernel lets the
// next kernel's blocks be scheduled as soon as all of its own blocks have
// started (they fill the SMs during its tail), and waits for the previous
// kernel in the stream to complete, with its writes visible, before reading
// anything but static design structures.  Kernels launched without the
// attribute are unaffected: the wait returns at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);   // errors surface via cudaGetLastError
}

// A shape for S scenarios: when S is below the shape's scenario width, the width
// shrinks to the power of two covering S and the block takes more cells instead
// (same threads per block), so a small batch does not leave most lanes of every
// warp idle.  Each (cell, scenario) is computed the same way in any shape.
inline BatchShape fit_shape(BatchShape sh, int64_t S) {
    if (S <= 0 || S >= sh.bx) return sh;
    int bx = 1;
    while (bx < S) bx <<= 1;
    if (bx >= sh.bx) return sh;   // a width that is no power of two (set by hand) and S above its half
    return BatchShape{bx, sh.bx * sh.by / bx, sh.v};
}

// scenarios per thread a shape gets for S scenarios: its v where S is a multiple of it, else 1
inline int scen_per_thread(BatchShape sh, int64_t S) { return (sh.v == 2 || sh.v == 4) && S % sh.v == 0 ? sh.v : 1; }

inline dim3 bgrid(int64_t S, BatchShape sh, int64_t rows) {
    const int64_t gy = bcdiv(rows > 0 ? rows : 1, sh.by);
    return dim3((unsigned)bcdiv(S, sh.bx), (unsigned)(gy < 65535 ? gy : 65535));
}

}  // namespace dp
