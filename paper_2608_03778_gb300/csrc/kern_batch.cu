// Batched scenarios: S input-activity scenarios of one design per launch.
// Every per-net value is stored scenario-innermost (value[n * S + s]), so the
// S values of one fanin are contiguous: a warp covering 32 scenarios of one
// cell reads each fanin as 256 consecutive bytes.  A block is bx scenarios x
// by cells; blockIdx.y walks the cells of a level.  Each thread computes one
// (cell, scenario) independently of the block shape, so every shape gives
// bitwise identical results and the shape is free for the autotuner.
//
// Each cell evaluates P(out = 1) as the multilinear extension of its truth
// table in float-float (the same reading of Eq. 2 as the single-scenario
// path), and only P is stored, as a float-float value (8 bytes per net and
// scenario): Q is re-derived as 1 - P in float-float, exact to about 1e-14
// absolute, wherever it is read.  That loses Q's relative accuracy only for nets within about 1e-9
// of 1, which matters for the hybrid beta (Eq. 5, single-scenario only) and
// not for the model power, SP, TR or gradients at their tolerances; it halves
// the bytes every gather moves.  The gradient is the model gradient (Sec. III-E,
// Eq. 7) in binary32, scaled per scenario by a seed K * w_s so that a caller
// can back-propagate any weighted sum of the scenario powers.
#include "kern_batch.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__global__ void k_fwdb_start(const float *__restrict__ sp_in, float2 *pq, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pq[i] = make_float2(sp_in[i], 0.f);
}

// the same, four values per thread (n a multiple of 4): one 16-byte load, two 16-byte stores
__global__ void k_fwdb_start4(const float *__restrict__ sp_in, float2 *pq, int64_t n) {
    const int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const float4 a = *reinterpret_cast<const float4 *>(sp_in + i);
    reinterpret_cast<float4 *>(pq + i)[0] = make_float4(a.x, 0.f, a.y, 0.f);
    reinterpret_cast<float4 *>(pq + i)[1] = make_float4(a.z, 0.f, a.w, 0.f);
}

__global__ void k_fwdb_level(const uint4 *__restrict__ fanin, float2 *pq, int32_t c0, int32_t c1, int64_t ns,
                             int64_t S, OpTable ops) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    const int64_t cf = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    uint4 r = cf < c1 ? fanin[cf] : make_uint4(0, 0, 0, 0);   // static: before the wait
    pdl_wait();
    for (int64_t c = cf; c < c1; c += step) {
        if (c != cf) r = fanin[c];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        pair_ff x[4];
        gather_ffb(pq, r, k, S, s, x);
        pq[(ns + c) * S + s] = cell_p(k, op_tt(ops, op), x);
    }
}

// Eq. 1 per scenario: chunk b of the nets -> partials[s * nchunks + b], then
// the chunks of each scenario summed in FP64 in a fixed order (reproducible).
// Within a chunk a thread forms each term alpha * C in binary32 (TR = 2 P Q
// with Q from the float-float pair, so it keeps its relative accuracy near
// P = 1; about 1e-7 relative per term) and adds it with TwoSum into a
// float-float sum (about 48 significant bits), so the FP64 pipe, slow on this
// part, sees one conversion per chunk instead of several operations per term.
__global__ void k_powerb_partials(const float2 *__restrict__ pq, const float *__restrict__ tr_in,
                                  const float *__restrict__ cload, const float *__restrict__ dcl, double *partials,
                                  int64_t nn, int64_t ns,
                                  int64_t S, int64_t chunk, int nchunks, int tr_mode) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t n0 = (int64_t)blockIdx.y * chunk, n1 = n0 + chunk < nn ? n0 + chunk : nn;
    ff acc = ff_make(0.f);
    for (int64_t n = n0; n < n1; n += 4) {
        float a[4], c[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t m = n + i;
            a[i] = 0.f;
            c[i] = 0.f;
            if (m < n1) {
                if (tr_mode == 2 || (m < ns && tr_mode == 0)) {
                    a[i] = tr_in[m * S + s];
                } else {
                    const pair_ff pr = pair_get(pq[m * S + s]);
                    a[i] = 2.f * (pr.p.hi + pr.p.lo) * (pr.q.hi + pr.q.lo);
                }
                c[i] = cl_of(cload, dcl, m, S, s);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const ff t = two_sum(acc.hi, a[i] * c[i]);
            acc = fast_two_sum(t.hi, t.lo + acc.lo);
        }
    }
    partials[s * nchunks + blockIdx.y] = (double)acc.hi + (double)acc.lo;
}

// The same partial sums with four consecutive scenarios per thread (S a
// multiple of 4): one 32-byte load of their P per net, four accumulators, each
// scenario's terms added in the same net order as above (bitwise the same).
__global__ void k_powerb_partials4(const float2 *__restrict__ pq, const float *__restrict__ tr_in,
                                   const float *__restrict__ cload, const float *__restrict__ dcl, double *partials,
                                   int64_t nn, int64_t ns, int64_t S, int64_t chunk, int nchunks, int tr_mode) {
    const int64_t s = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (s >= S) return;
    const int64_t n0 = (int64_t)blockIdx.y * chunk, n1 = n0 + chunk < nn ? n0 + chunk : nn;
    ff acc[4] = {ff_make(0.f), ff_make(0.f), ff_make(0.f), ff_make(0.f)};
    for (int64_t n = n0; n < n1; n += 2) {
        float a[2][4], c[2][4];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int64_t m = n + i;
#pragma unroll
            for (int v = 0; v < 4; v++) a[i][v] = c[i][v] = 0.f;
            if (m < n1) {
                if (tr_mode == 2 || (m < ns && tr_mode == 0)) {
                    const float4 t = *reinterpret_cast<const float4 *>(tr_in + m * S + s);
                    a[i][0] = t.x;
                    a[i][1] = t.y;
                    a[i][2] = t.z;
                    a[i][3] = t.w;
                } else {
                    const float4 u0 = reinterpret_cast<const float4 *>(pq + m * S + s)[0];
                    const float4 u1 = reinterpret_cast<const float4 *>(pq + m * S + s)[1];
                    const float2 w[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                         make_float2(u1.z, u1.w)};
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        const pair_ff pr = pair_get(w[v]);
                        a[i][v] = 2.f * (pr.p.hi + pr.p.lo) * (pr.q.hi + pr.q.lo);
                    }
                }
                if (dcl) {
                    const float4 t = *reinterpret_cast<const float4 *>(dcl + m * S + s);
                    c[i][0] = cload[m] + t.x;
                    c[i][1] = cload[m] + t.y;
                    c[i][2] = cload[m] + t.z;
                    c[i][3] = cload[m] + t.w;
                } else {
#pragma unroll
                    for (int v = 0; v < 4; v++) c[i][v] = cload[m];
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const ff t = two_sum(acc[v].hi, a[i][v] * c[i][v]);
                acc[v] = fast_two_sum(t.hi, t.lo + acc[v].lo);
            }
    }
#pragma unroll
    for (int v = 0; v < 4; v++) partials[(s + v) * nchunks + blockIdx.y] = (double)acc[v].hi + (double)acc[v].lo;
}

// one warp per scenario: lane l sums chunks l, l + 32, ... in order, then a fixed shuffle tree
__global__ void k_sumb_final(const double *__restrict__ partials, int nchunks, int64_t S, double K, double *out) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= S) return;
    double acc = 0.0;
    for (int b = lane; b < nchunks; b += 32) acc += partials[s * nchunks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[s] = K * acc;
}

__global__ void k_seedb(float *ks, const double *__restrict__ w, double K, int64_t S) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) ks[s] = (float)(w ? K * w[s] : K);
}
// The same level with V consecutive scenarios per thread (V = 2 or 4, S a
// multiple of V): each fanin gather is V / 2 16-byte loads of those scenarios'
// P, so a warp keeps V times the bytes in flight; every (cell, scenario) is
// computed exactly as above.
template <int V>
__global__ void k_fwdb_levelv(const uint4 *__restrict__ fanin, float2 *pq, int32_t c0, int32_t c1, int64_t ns,
                              int64_t S, OpTable ops) {
    const int64_t s = V * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    pdl_trigger();
    if (s >= S) return;
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    const int64_t cf = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    uint4 r = cf < c1 ? fanin[cf] : make_uint4(0, 0, 0, 0);   // static: before the wait
    pdl_wait();
    for (int64_t c = cf; c < c1; c += step) {
        if (c != cf) r = fanin[c];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        const uint32_t tt = op_tt(ops, op);
        const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
        float4 v[4][V / 2];
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int h = 0; h < V / 2; h++)
                v[j][h] = j < k ? reinterpret_cast<const float4 *>(pq + (int64_t)n[j] * S + s)[h]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 out[V / 2];
#pragma unroll
        for (int h = 0; h < V / 2; h++) {
            pair_ff x[4], y[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                x[j] = pair_get(make_float2(v[j][h].x, v[j][h].y));
                y[j] = pair_get(make_float2(v[j][h].z, v[j][h].w));
            }
            const float2 a = cell_p(k, tt, x), b = cell_p(k, tt, y);
            out[h] = make_float4(a.x, a.y, b.x, b.y);
        }
#pragma unroll
        for (int h = 0; h < V / 2; h++) reinterpret_cast<float4 *>(pq + (ns + c) * S + s)[h] = out[h];
    }
}

// reverse level: each net's adjoint is its fanout range summed in index order
// plus its local term d(K_s C 2PQ)/dP = 2 K_s C (Q - P); the cell then writes
// one contribution per input edge (no atomics)
__global__ void k_bwdb_level(const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr,
                             const int4 *__restrict__ efpos, const float2 *__restrict__ pq,
                             const float *__restrict__ cload, const float *__restrict__ dcl,
                             const float *__restrict__ ks, float *gfo, int32_t c0, int32_t c1, int64_t ns, int64_t S,
                             OpTable ops) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    const int64_t cf = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    uint4 rf = cf < c1 ? fanin[cf] : make_uint4(0, 0, 0, 0);   // static: before the wait
    pdl_wait();
    const float Ks = ks[s];
    for (int64_t c = cf; c < c1; c += step) {
        const int64_t n = ns + c;
        // everything that does not depend on the fanout sum goes out first, so its loads
        // overlap the fanout range's
        const uint4 r = c == cf ? rf : fanin[c];
        const int4 ep = efpos[c];
        const int32_t e0 = fptr[n], e1 = fptr[n + 1];
        const float2 self = pq[n * S + s];
        const float cl = cl_of(cload, dcl, n, S, s);
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        float p[4], q[4], d[4];
        gather32(pq, r, k, S, s, p, q);
        float acc = 0.f;
        for (int32_t e = e0; e < e1; e++) acc += gfo[(int64_t)e * S + s];
        const float g = acc + 2.f * Ks * cl * qmp32(self);
        cell_partials(k, op_tt(ops, op), p, q, d);
        if (k > 0) gfo[(int64_t)ep.x * S + s] = g * d[0];
        if (k > 1) gfo[(int64_t)ep.y * S + s] = g * d[1];
        if (k > 2) gfo[(int64_t)ep.z * S + s] = g * d[2];
        if (k > 3) gfo[(int64_t)ep.w * S + s] = g * d[3];
    }
}

// The same reverse level with V consecutive scenarios per thread (V = 2 or 4,
// S a multiple of V): 16-byte loads of those scenarios' P, 8- or 16-byte loads
// and stores of their edge adjoints; every (cell, scenario) is computed
// exactly as above.
template <int V>
__global__ void k_bwdb_levelv(const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr,
                              const int4 *__restrict__ efpos, const float2 *__restrict__ pq,
                              const float *__restrict__ cload, const float *__restrict__ dcl,
                              const float *__restrict__ ks, float *gfo, int32_t c0, int32_t c1, int64_t ns, int64_t S,
                              OpTable ops) {
    const int64_t s = V * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    pdl_trigger();
    if (s >= S) return;
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    const int64_t cf = c0 + (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    uint4 rf = cf < c1 ? fanin[cf] : make_uint4(0, 0, 0, 0);   // static: before the wait
    pdl_wait();
    float Ks[V];
#pragma unroll
    for (int i = 0; i < V; i++) Ks[i] = ks[s + i];
    for (int64_t c = cf; c < c1; c += step) {
        const int64_t n = ns + c;
        const uint4 r = c == cf ? rf : fanin[c];
        const int4 ep = efpos[c];
        const int32_t e0 = fptr[n], e1 = fptr[n + 1];
        float2 self[V];
#pragma unroll
        for (int h = 0; h < V / 2; h++) {
            const float4 t = reinterpret_cast<const float4 *>(pq + n * S + s)[h];
            self[2 * h] = make_float2(t.x, t.y);
            self[2 * h + 1] = make_float2(t.z, t.w);
        }
        float cl[V];
#pragma unroll
        for (int i = 0; i < V; i++) cl[i] = dcl ? cload[n] + dcl[n * S + s + i] : cload[n];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        const uint32_t tt = op_tt(ops, op);
        const uint32_t nid[4] = {r.x & kMask24, r.y, r.z, r.w};
        float4 v[4][V / 2];
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int h = 0; h < V / 2; h++)
                v[j][h] = j < k ? reinterpret_cast<const float4 *>(pq + (int64_t)nid[j] * S + s)[h]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        float acc[V];
#pragma unroll
        for (int i = 0; i < V; i++) acc[i] = 0.f;
        for (int32_t e = e0; e < e1; e++) {
            const float *src = gfo + (int64_t)e * S + s;
            if (V == 4) {
                const float4 t = *reinterpret_cast<const float4 *>(src);
                acc[0] += t.x;
                acc[1 % V] += t.y;
                acc[2 % V] += t.z;
                acc[3 % V] += t.w;
            } else {
                const float2 t = *reinterpret_cast<const float2 *>(src);
                acc[0] += t.x;
                acc[1 % V] += t.y;
            }
        }
        float g[V], d[V][4];
#pragma unroll
        for (int i = 0; i < V; i++) {
            float p[4], q[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float4 &w = v[j][i / 2];
                const pair_ff a = pair_get((i & 1) ? make_float2(w.z, w.w) : make_float2(w.x, w.y));
                p[j] = a.p.hi + a.p.lo;
                q[j] = a.q.hi + a.q.lo;
            }
            g[i] = acc[i] + 2.f * Ks[i] * cl[i] * qmp32(self[i]);
            cell_partials(k, tt, p, q, d[i]);
        }
        const int pos[4] = {ep.x, ep.y, ep.z, ep.w};
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (j >= k) break;
            float *dst = gfo + (int64_t)pos[j] * S + s;
            if (V == 4) *reinterpret_cast<float4 *>(dst) = make_float4(g[0] * d[0][j], g[1 % V] * d[1 % V][j],
                                                                       g[2 % V] * d[2 % V][j], g[3 % V] * d[3 % V][j]);
            else *reinterpret_cast<float2 *>(dst) = make_float2(g[0] * d[0][j], g[1 % V] * d[1 % V][j]);
        }
    }
}

// startpoints: fanout sum, plus the local term when their TR derives from their SP (tr_mode 1)
__global__ void k_bwdb_start(const int32_t *__restrict__ fptr, const float2 *__restrict__ pq,
                             const float *__restrict__ cload, const float *__restrict__ dcl,
                             const float *__restrict__ ks,
                             const float *__restrict__ gfo, float *gsp, int64_t ns, int64_t S, int tr_mode) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    pdl_trigger();
    if (s >= S) return;
    pdl_wait();
    const float Ks = ks[s];
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t k = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; k < ns; k += step) {
        const int32_t e0 = fptr[k], e1 = fptr[k + 1];
        float acc = 0.f;
        for (int32_t e = e0; e < e1; e++) acc += gfo[(int64_t)e * S + s];
        float g = acc;
        if (tr_mode) g += 2.f * Ks * cl_of(cload, dcl, k, S, s) * qmp32(pq[k * S + s]);
        gsp[k * S + s] = g;
    }
}

// The same with four consecutive scenarios per thread (S a multiple of 4): 16-byte
// loads of the edge adjoints, eight edges' loads in flight before they are added in
// index order (the same order as above, so bitwise the same).
__global__ void k_bwdb_start4(const int32_t *__restrict__ fptr, const float2 *__restrict__ pq,
                              const float *__restrict__ cload, const float *__restrict__ dcl,
                              const float *__restrict__ ks, const float *__restrict__ gfo, float *gsp, int64_t ns,
                              int64_t S, int tr_mode) {
    const int64_t s = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    pdl_trigger();
    if (s >= S) return;
    pdl_wait();
    const float4 Ks = *reinterpret_cast<const float4 *>(ks + s);
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t k = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; k < ns; k += step) {
        const int32_t e0 = fptr[k], e1 = fptr[k + 1];
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int32_t e = e0; e < e1; e += 8) {
            float4 t[8];
#pragma unroll
            for (int i = 0; i < 8; i++)
                t[i] = e + i < e1 ? *reinterpret_cast<const float4 *>(gfo + (int64_t)(e + i) * S + s)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int i = 0; i < 8; i++)
                if (e + i < e1) {
                    acc.x += t[i].x;
                    acc.y += t[i].y;
                    acc.z += t[i].z;
                    acc.w += t[i].w;
                }
        }
        float g[4] = {acc.x, acc.y, acc.z, acc.w};
        if (tr_mode) {
            const float ksv[4] = {Ks.x, Ks.y, Ks.z, Ks.w};
            const float4 u0 = reinterpret_cast<const float4 *>(pq + k * S + s)[0];
            const float4 u1 = reinterpret_cast<const float4 *>(pq + k * S + s)[1];
            const float2 w[4] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                 make_float2(u1.z, u1.w)};
#pragma unroll
            for (int v = 0; v < 4; v++) g[v] += 2.f * ksv[v] * cl_of(cload, dcl, k, S, s + v) * qmp32(w[v]);
        }
        *reinterpret_cast<float4 *>(gsp + k * S + s) = make_float4(g[0], g[1], g[2], g[3]);
    }
}

// dP_s/dC_n = K_s alpha_n(s); dP_s/dpincap_c = K_s sum_j alpha_{fanin j}(s)
// (one pin cap per cell, loading each of its fanin nets); dP_s/dTR_k = K_s C_k
// at a startpoint in tr_mode 0, else 0
__global__ void k_gradb_rows(const uint4 *__restrict__ fanin, const float2 *__restrict__ pq,
                             const float *__restrict__ tr_in, const float *__restrict__ cload,
                             const float *__restrict__ dcl,
                             const int32_t *__restrict__ net_of_user, const int32_t *__restrict__ cell_of_user,
                             const float *__restrict__ ks, const float *__restrict__ gtr_lag1, float *gcl,
                             float *gpin, float *gtr, int64_t nn, int64_t nc, int64_t ns, int64_t S, int tr_mode,
                             OpTable ops) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const float Ks = ks[s];
    const int64_t rows = (gcl ? nn : 0) + (gpin ? nc : 0) + (gtr ? ns : 0);
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t r = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; r < rows; r += step) {
        int64_t u = r;
        if (gcl) {
            if (u < nn) {
                gcl[u * S + s] = Ks * alpha32(pq, tr_in, net_of_user[u], ns, S, s, tr_mode);
                continue;
            }
            u -= nn;
        }
        if (gpin) {
            if (u < nc) {
                const uint4 f = fanin[cell_of_user[u]];
                const int k = op_arity(ops, f.x >> 24);
                const uint32_t n[4] = {f.x & kMask24, f.y, f.z, f.w};
                float a = 0.f;
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (j < k) a += alpha32(pq, tr_in, n[j], ns, S, s, tr_mode);
                gpin[u * S + s] = Ks * a;
                continue;
            }
            u -= nc;
        }
        gtr[u * S + s] = tr_mode == 2 ? gtr_lag1[u * S + s] : (tr_mode ? 0.f : Ks * cl_of(cload, dcl, u, S, s));
    }
}

// Cap gradients summed over the scenarios in FP64: one warp per row, lane l
// takes scenarios l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void k_gradb_reduce(const uint4 *__restrict__ fanin, const float2 *__restrict__ pq,
                               const float *__restrict__ tr_in, const int32_t *__restrict__ net_of_user,
                               const int32_t *__restrict__ cell_of_user, const float *__restrict__ ks, float *gcl,
                               float *gpin, int64_t nn, int64_t nc, int64_t ns, int64_t S, int tr_mode, OpTable ops) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = (gcl ? nn : 0) + (gpin ? nc : 0);
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < rows; r += W) {
        int64_t u = r;
        const bool is_cl = gcl && u < nn;
        if (gcl && !is_cl) u -= nn;
        uint32_t n[4] = {0, 0, 0, 0};
        int k = 1;
        if (is_cl) {
            n[0] = (uint32_t)net_of_user[u];
        } else {
            const uint4 f = fanin[cell_of_user[u]];
            k = op_arity(ops, f.x >> 24);
            n[0] = f.x & kMask24;
            n[1] = f.y;
            n[2] = f.z;
            n[3] = f.w;
        }
        double acc = 0.0;
        for (int64_t s = lane; s < S; s += 32) {
            float a = 0.f;
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (j < k) a += alpha32(pq, tr_in, n[j], ns, S, s, tr_mode);
            acc += (double)(ks[s] * a);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            if (is_cl) gcl[u] = (float)acc;
            else gpin[u] = (float)acc;
        }
    }
}

__global__ void k_netb_user(const float2 *__restrict__ pq, const float *__restrict__ tr_in,
                            const int32_t *__restrict__ net_of_user, float *sp_out, float *tr_out, int64_t nn,
                            int64_t ns, int64_t S, int tr_mode) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t step = (int64_t)gridDim.y * blockDim.y;
    for (int64_t u = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; u < nn; u += step) {
        const int64_t n = net_of_user[u];
        if (sp_out) {
            const float2 v = pq[n * S + s];
            sp_out[u * S + s] = v.x + v.y;
        }
        if (tr_out) tr_out[u * S + s] = alpha32(pq, tr_in, n, ns, S, s, tr_mode);
    }
}

__global__ void k_ascent(float *x, const float *__restrict__ g, int64_t n, float eta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = __fadd_rn(x[i], __fmul_rn(eta, g[i]));
    x[i] = fminf(fmaxf(v, 0.f), 1.f);
}

// ---- Eq. 3: P_virus of the thresholded vectors ----
// words of net n: [2W] with W = ceil(S / 64); word w < W holds v0 of scenarios
// 64 w .. 64 w + 63, word W + w holds v1 = not v0 of the same scenarios
__global__ void k_virus_start(const float *__restrict__ sp, uint64_t *words, uint8_t *v0, int64_t ns, int64_t S,
                              int64_t W) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns * W) return;
    const int64_t k = i / W, w = i - k * W;
    uint64_t b0 = 0, valid = 0;
    for (int b = 0; b < 64; b++) {
        const int64_t s = w * 64 + b;
        if (s >= S) break;
        const bool one = sp[k * S + s] >= 0.5f;
        if (v0) v0[k * S + s] = one ? 1 : 0;
        b0 |= (uint64_t)one << b;
        valid |= 1ull << b;
    }
    words[k * 2 * W + w] = b0;
    words[k * 2 * W + W + w] = ~b0 & valid;
}

__global__ void k_virus_level(const uint4 *__restrict__ fanin, uint64_t *words, int32_t c0, int32_t c1, int64_t ns,
                              int64_t W2, OpTable ops) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)(c1 - c0) * W2) return;
    const int64_t c = c0 + i / W2, w = i % W2;
    const uint4 r = fanin[c];
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
    uint64_t x[4];
#pragma unroll
    for (int j = 0; j < 4; j++) x[j] = j < k ? words[(int64_t)n[j] * W2 + w] : 0ull;
    words[(ns + c) * W2 + w] = cell_bits(k, op_tt(ops, op), x);
}

__global__ void k_virus_partials(const uint64_t *__restrict__ words, const float *__restrict__ cload,
                                 double *partials, int64_t nn, int64_t S, int64_t W, int64_t chunk, int nchunks) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t w = s >> 6;
    const int b = (int)(s & 63);
    const int64_t n0 = (int64_t)blockIdx.y * chunk, n1 = n0 + chunk < nn ? n0 + chunk : nn;
    double acc = 0.0;
    for (int64_t n = n0; n < n1; n++) {
        const uint64_t d = words[n * 2 * W + w] ^ words[n * 2 * W + W + w];
        if ((d >> b) & 1ull) acc += (double)cload[n];
    }
    partials[s * nchunks + blockIdx.y] = acc;
}

// out[c * ldo + r] = in[r * C + c] for an R x C block, through 32 x 32 tiles in shared memory
__global__ void k_transpose(const float *__restrict__ in, float *out, int64_t R, int64_t C, int64_t ldo) {
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[c * ldo + r] = t[threadIdx.x][i];
    }
}


int nchunks_of(int64_t nn, int64_t *chunk) {
    const int64_t m = nn > 0 ? nn : 1;
    *chunk = cdiv(m, kBatchPowerChunks);
    return (int)cdiv(m, *chunk);
}

}  // namespace

void launch_fwdb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl, int tr_mode,
                 BatchShape sh, cudaStream_t s) {
    if (tr_mode == 2) {
        launch_fwdl(d, b, ops, lvl, sh, s);
        return;
    }
    const int64_t S = b.S;
    if (d.n_start && (d.n_start * S) % 4 == 0)
        k_fwdb_start4<<<(unsigned)cdiv(d.n_start * S / 4, 256), 256, 0, s>>>(b.sp_in, b.pq, d.n_start * S);
    else if (d.n_start)
        k_fwdb_start<<<(unsigned)cdiv(d.n_start * S, 256), 256, 0, s>>>(b.sp_in, b.pq, d.n_start * S);
    const int v = scen_per_thread(sh, S);
    sh = fit_shape(sh, S / v);
    const dim3 blk((unsigned)sh.bx, (unsigned)sh.by);
    for (int l = 1; l <= d.n_levels; l++) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        if (c1 <= c0) continue;
        const dim3 g = bgrid(S / v, sh, c1 - c0);
        if (v == 4) launch_pdl(k_fwdb_levelv<4>, g, blk, s, d.fanin, b.pq, c0, c1, d.n_start, S, ops);
        else if (v == 2) launch_pdl(k_fwdb_levelv<2>, g, blk, s, d.fanin, b.pq, c0, c1, d.n_start, S, ops);
        else launch_pdl(k_fwdb_level, g, blk, s, d.fanin, b.pq, c0, c1, d.n_start, S, ops);
    }
}

void launch_powerb(const DevDesign &d, const BatchBufs &b, int tr_mode, double K, cudaStream_t s) {
    const int64_t S = b.S;
    int64_t chunk = 0;
    const int nch = nchunks_of(d.n_nets, &chunk);
    if (S % 4 == 0)
        k_powerb_partials4<<<dim3((unsigned)cdiv(S / 4, 128), (unsigned)nch), 128, 0, s>>>(
            b.pq, tr_mode == 2 ? b.tq : b.tr_in, d.cload, b.dcl, b.partials, d.n_nets, d.n_start, S, chunk, nch,
            tr_mode);
    else
        k_powerb_partials<<<dim3((unsigned)cdiv(S, 128), (unsigned)nch), 128, 0, s>>>(
            b.pq, tr_mode == 2 ? b.tq : b.tr_in, d.cload, b.dcl, b.partials, d.n_nets, d.n_start, S, chunk, nch,
            tr_mode);
    k_sumb_final<<<(unsigned)cdiv(S * 32, 256), 256, 0, s>>>(b.partials, nch, S, K, b.power);
}

void launch_seedb(const BatchBufs &b, double K, const double *weights, cudaStream_t s) {
    k_seedb<<<(unsigned)cdiv(b.S, 128), 128, 0, s>>>(b.ks, weights, K, b.S);
}

void launch_bwdb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl, int tr_mode,
                 BatchShape sh, cudaStream_t s) {
    if (tr_mode == 2) {
        launch_bwdl(d, b, ops, lvl, sh, s);
        return;
    }
    const int64_t S = b.S;
    const int v = scen_per_thread(sh, S);   // scenarios per thread in the cell levels
    const BatchShape sh1 = fit_shape(sh, S);
    sh = fit_shape(sh, S / v);
    const dim3 blk((unsigned)sh.bx, (unsigned)sh.by);
    for (int l = d.n_levels; l >= 1; l--) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        if (c1 <= c0) continue;
        const dim3 g = bgrid(S / v, sh, c1 - c0);
        if (v == 4)
            launch_pdl(k_bwdb_levelv<4>, g, blk, s, d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos, b.pq, d.cload,
                       b.dcl, b.ks, b.gfo, c0, c1, d.n_start, S, ops);
        else if (v == 2)
            launch_pdl(k_bwdb_levelv<2>, g, blk, s, d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos, b.pq, d.cload,
                       b.dcl, b.ks, b.gfo, c0, c1, d.n_start, S, ops);
        else
            launch_pdl(k_bwdb_level, g, blk, s, d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos, b.pq, d.cload,
                       b.dcl, b.ks, b.gfo, c0, c1, d.n_start, S, ops);
    }
    if (d.n_start && S % 4 == 0) {
        const BatchShape s4 = fit_shape(BatchShape{128, 1, 4}, S / 4);
        launch_pdl(k_bwdb_start4, bgrid(S / 4, s4, d.n_start), dim3((unsigned)s4.bx, (unsigned)s4.by), s, d.fout_ptr,
                   b.pq, d.cload, b.dcl, b.ks, b.gfo, b.gsp, d.n_start, S, tr_mode);
    } else if (d.n_start) {
        launch_pdl(k_bwdb_start, bgrid(S, sh1, d.n_start), dim3((unsigned)sh1.bx, (unsigned)sh1.by), s, d.fout_ptr,
                   b.pq, d.cload, b.dcl, b.ks, b.gfo, b.gsp, d.n_start, S, tr_mode);
    }
}

void launch_gradb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, int tr_mode, bool reduce, float *gtr,
                  float *gpin, float *gcl, cudaStream_t s) {
    const int64_t S = b.S;
    if (reduce) {
        const int64_t rows = (gcl ? d.n_nets : 0) + (gpin ? d.n_cells : 0);
        if (rows) {
            const int64_t blocks = cdiv(rows, 8);
            k_gradb_reduce<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(
                d.fanin, b.pq, tr_mode == 2 ? b.tq : b.tr_in, d.net_of_user, d.cell_of_user, b.ks, gcl, gpin,
                d.n_nets, d.n_cells, d.n_start, S, tr_mode, ops);
        }
        gcl = gpin = nullptr;
    }
    const int64_t rows = (gcl ? d.n_nets : 0) + (gpin ? d.n_cells : 0) + (gtr ? d.n_start : 0);
    if (rows == 0) return;
    const BatchShape sh = fit_shape(BatchShape{S >= 128 ? 128 : 32, S >= 128 ? 1 : 4}, S);
    k_gradb_rows<<<bgrid(S, sh, rows), dim3((unsigned)sh.bx, (unsigned)sh.by), 0, s>>>(
        d.fanin, b.pq, tr_mode == 2 ? b.tq : b.tr_in, d.cload, b.dcl, d.net_of_user, d.cell_of_user, b.ks,
        b.gtr, gcl, gpin, gtr, d.n_nets, d.n_cells, d.n_start, S, tr_mode, ops);
}

void launch_netb_user(const DevDesign &d, const BatchBufs &b, int tr_mode, float *sp, float *tr, cudaStream_t s) {
    if (!d.n_nets || (!sp && !tr)) return;
    const BatchShape sh = fit_shape(BatchShape{b.S >= 128 ? 128 : 32, b.S >= 128 ? 1 : 4}, b.S);
    k_netb_user<<<bgrid(b.S, sh, d.n_nets), dim3((unsigned)sh.bx, (unsigned)sh.by), 0, s>>>(
        b.pq, tr_mode == 2 ? b.tq : b.tr_in, d.net_of_user, sp, tr, d.n_nets, d.n_start, b.S, tr_mode);
}

void launch_transpose(const float *in, float *out, int64_t R, int64_t C, cudaStream_t s) {
    if (R <= 0 || C <= 0) return;
    const int64_t gy = cdiv(R, 32);
    for (int64_t y0 = 0; y0 < gy; y0 += 65535) {   // grid.y limit: the rows go in slabs
        const int64_t rows = (gy - y0 < 65535 ? gy - y0 : 65535) * 32;
        const int64_t rr = R - y0 * 32 < rows ? R - y0 * 32 : rows;
        k_transpose<<<dim3((unsigned)cdiv(C, 32), (unsigned)cdiv(rr, 32)), dim3(32, 8), 0, s>>>(
            in + y0 * 32 * C, out + y0 * 32, rr, C, R);
    }
}

void launch_ascent(float *x, const float *g, int64_t n, float eta, cudaStream_t s) {
    if (n) k_ascent<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(x, g, n, eta);
}

void launch_virus(const DevDesign &d, const OpTable &ops, const int32_t *lvl, const float *sp, int64_t S,
                  uint64_t *words, uint8_t *v0, double *partials, double *out, cudaStream_t s) {
    const int64_t W = cdiv(S, 64), W2 = 2 * W;
    if (d.n_start)
        k_virus_start<<<(unsigned)cdiv(d.n_start * W, 128), 128, 0, s>>>(sp, words, v0, d.n_start, S, W);
    for (int l = 1; l <= d.n_levels; l++) {
        const int64_t m = (int64_t)(lvl[l] - lvl[l - 1]) * W2;
        if (m)
            k_virus_level<<<(unsigned)cdiv(m, 256), 256, 0, s>>>(d.fanin, words, lvl[l - 1], lvl[l], d.n_start, W2,
                                                                 ops);
    }
    int64_t chunk = 0;
    const int nch = nchunks_of(d.n_nets, &chunk);
    k_virus_partials<<<dim3((unsigned)cdiv(S, 128), (unsigned)nch), 128, 0, s>>>(words, d.cload, partials, d.n_nets,
                                                                                S, W, chunk, nch);
    k_sumb_final<<<(unsigned)cdiv(S * 32, 256), 256, 0, s>>>(partials, nch, S, 1.0, out);
}

}  // namespace dp
