// Device helpers shared by the kernels: cell evaluation on probabilities and
// on bit-packed words, and the Philox4x32-10 counter generator.
#pragma once
#include <cstdint>

#include "kernels.h"

namespace dp {

constexpr uint32_t kMask24 = 0xFFFFFFu;

__device__ __forceinline__ int op_arity(const OpTable &t, uint32_t op) { return (int)((t.e[op] >> 16) & 0xFFu); }
__device__ __forceinline__ uint32_t op_lut(const OpTable &t, uint32_t op) { return t.e[op] >> 24; }
__device__ __forceinline__ uint32_t op_tt(const OpTable &t, uint32_t op) { return t.e[op] & 0xFFFFu; }

// ---- float-float arithmetic (an unevaluated sum hi + lo of two binary32
// values, about 44 significant bits), built from error-free transforms on the
// FP32 pipes.  The _rn intrinsics are never contracted into FMAs, which the
// transforms rely on.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_make(float a) { return ff{a, 0.f}; }
// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
// Dekker's FastTwoSum, valid when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);   // exact product error
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const ff r = ff_add(a, ff_mul(ff_make(-q1), b));
    return fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// Probabilities of a net are carried as the pair (P, Q) = (P(net=1), P(net=0)),
// each a float-float value, stored as float4 (P.hi, P.lo, Q.hi, Q.lo).  Q is
// never formed as 1 - P: deep reconvergent netlists have many nets within
// 1e-15 of 0 or 1, where that subtraction would destroy the relative accuracy
// of TR_model = 2PQ (Eq. 2), and the hybrid beta (Eq. 5) multiplies the
// paper's gradient at every net (Eq. 6), so its error compounds along paths.
//
// The output pair of a cell with K inputs is the multilinear extension of its
// truth table and of the complemented table (Sec. III-B; exact under input
// independence, equal to the stack interpreter of Algorithm 2 on read-once
// cells), folded input by input as v = Q_i v[.., 0] + P_i v[.., 1]: every
// term is non-negative, so both P and Q keep full relative accuracy.  The pair
// is then divided by its sum (1 in exact arithmetic) so that rounding cannot
// accumulate along the exponentially many paths of a reconvergent netlist.
struct pair_ff {
    ff p, q;
};
// Storage tag: P.hi and Q.hi are never negative, so their sign bits carry the
// parity of the forward pass that wrote them (a counter in device memory,
// advanced once per pass).  A reader of the dataflow schedule knows a pair is
// from the current pass when both tags match; every reader masks the tags.
__device__ __forceinline__ float untag(float v) { return __int_as_float(__float_as_int(v) & 0x7FFFFFFF); }
__device__ __forceinline__ float4 pq_decode(float4 v) { return make_float4(untag(v.x), v.y, untag(v.z), v.w); }
__device__ __forceinline__ pair_ff pair_load(const float4 &v) {
    return pair_ff{ff{untag(v.x), v.y}, ff{untag(v.z), v.w}};
}
__device__ __forceinline__ float4 pair_store(const pair_ff &a, uint32_t parity) {
    const int t = (int)(parity << 31);
    return make_float4(__int_as_float(__float_as_int(a.p.hi) | t), a.p.lo, __int_as_float(__float_as_int(a.q.hi) | t),
                       a.q.lo);
}
// writes a tagged pair as two 8-byte halves (P.hi, P.lo) and (Q.hi, Q.lo), each
// single-copy atomic, so a concurrent reader never sees a half torn
__device__ __forceinline__ void pair_put(float4 *dst, const pair_ff &a, uint32_t parity) {
    const float4 v = pair_store(a, parity);
    const unsigned long long h0 = (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
    const unsigned long long h1 = (unsigned long long)__float_as_uint(v.z) | ((unsigned long long)__float_as_uint(v.w) << 32);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(dst), "l"(h0), "l"(h1) : "memory");
}

// (P, 1 - P) of a binary32 probability, exactly
__device__ __forceinline__ pair_ff pair_of(float p) { return pair_ff{ff_make(p), two_sum(1.f, -p)}; }

// TR_model = 2PQ rounded once to binary32
__device__ __forceinline__ float pair_tr(const pair_ff &a) {
    const ff t = ff_mul(a.p, a.q);
    return 2.f * (t.hi + t.lo);
}

// The pair divided by its sum s = P + Q.  In float-float s differs from 1 only
// by accumulated rounding, d = s - 1 of order 1e-13, so x / s = x (1 - d) up
// to d^2 (far below the format's 2^-44): one binary32 product and a
// FastTwoSum per value instead of two float-float divisions.
__device__ __forceinline__ pair_ff pair_renorm(const ff &p, const ff &q) {
    const ff s = ff_add(p, q);
    const float d = __fadd_rn(__fsub_rn(s.hi, 1.f), s.lo);   // s.hi - 1 is exact near 1
    return pair_ff{fast_two_sum(p.hi, __fsub_rn(p.lo, __fmul_rn(p.hi, d))),
                   fast_two_sum(q.hi, __fsub_rn(q.lo, __fmul_rn(q.hi, d)))};
}

// one fold step, q v0 + p v1 (all terms non-negative): the two products' rounding
// errors and every low-part product are gathered in one binary32 sum, then a
// single renormalisation
__device__ __forceinline__ ff fold_pq(const pair_ff &x, const ff &v0, const ff &v1) {
    const float a = __fmul_rn(x.q.hi, v0.hi), b = __fmul_rn(x.p.hi, v1.hi);
    const float ea = fmaf(x.q.hi, v0.hi, -a), eb = fmaf(x.p.hi, v1.hi, -b);
    const ff s = two_sum(a, b);
    float lo = __fadd_rn(s.lo, __fadd_rn(ea, eb));
    lo = fmaf(x.q.hi, v0.lo, lo);
    lo = fmaf(x.q.lo, v0.hi, lo);
    lo = fmaf(x.p.hi, v1.lo, lo);
    lo = fmaf(x.p.lo, v1.hi, lo);
    return fast_two_sum(s.hi, lo);
}

template <int K>
__device__ __forceinline__ pair_ff ml_pair(uint32_t tt, const pair_ff (&x)[4]) {
    ff v1[1 << K], v0[1 << K];
    // first fold: leaves are 0/1, so each term is 0, Q_0, P_0, or Q_0 + P_0 = 1
#pragma unroll
    for (int m = 0; m < (1 << (K - 1)); m++) {
        const bool a1 = (tt >> (2 * m)) & 1u, b1 = (tt >> (2 * m + 1)) & 1u;
        const ff z = ff_make(0.f), o = ff_make(1.f);
        v1[m] = a1 ? (b1 ? o : x[0].q) : (b1 ? x[0].p : z);
        v0[m] = a1 ? (b1 ? z : x[0].p) : (b1 ? x[0].q : o);
    }
#pragma unroll
    for (int i = 1; i < K; i++) {
#pragma unroll
        for (int m = 0; m < (1 << (K - 1 - i)); m++) {
            v1[m] = fold_pq(x[i], v1[2 * m], v1[2 * m + 1]);
            v0[m] = fold_pq(x[i], v0[2 * m], v0[2 * m + 1]);
        }
    }
    return pair_renorm(v1[0], v0[0]);
}

__device__ __forceinline__ pair_ff cell_pair(int k, uint32_t tt, const pair_ff (&x)[4]) {
    switch (k) {
        case 0: return (tt & 1u) ? pair_ff{ff_make(1.f), ff_make(0.f)} : pair_ff{ff_make(0.f), ff_make(1.f)};
        case 1: return ml_pair<1>(tt, x);
        case 2: return ml_pair<2>(tt, x);
        case 3: return ml_pair<3>(tt, x);
        default: return ml_pair<4>(tt, x);
    }
}

// gathers the (P, Q) pairs of a cell's inputs (unused slots: P = 0, Q = 1)
template <bool L2>
__device__ __forceinline__ void gather_ff(const float4 *pq, const uint4 &r, int k, pair_ff (&x)[4]) {
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
        x[j] = pair_ff{ff_make(0.f), ff_make(1.f)};
        if (j < k) x[j] = pair_load(L2 ? __ldcg(pq + n[j]) : pq[n[j]]);
    }
}

// (Q - P) of a stored pair, rounded once to binary32
__device__ __forceinline__ float pair_qmp(const float4 &t) {
    const float4 v = pq_decode(t);
    const ff d = ff_add(ff{v.z, v.w}, ff{-v.x, -v.y});
    return d.hi + d.lo;
}

// binary32 (P, Q) of a cell's inputs, for the partial derivatives
__device__ __forceinline__ void gather_pairs(const float4 *pq, const uint4 &r, int k, float (&p)[4], float (&q)[4]) {
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
        p[j] = 0.f;
        q[j] = 1.f;
        if (j < k) {
            const float4 v = pq_decode(pq[n[j]]);
            p[j] = v.x + v.y;
            q[j] = v.z + v.w;
        }
    }
}

// d P / d a_J: the multilinear extension, over the other inputs, of the
// difference table f(.., a_J = 1, ..) - f(.., a_J = 0, ..) (entries in {-1,0,1}).
template <int K, int J>
__device__ __forceinline__ float ml_partial(uint32_t tt, const float (&p)[4], const float (&q)[4]) {
    constexpr int M = 1 << (K - 1);
    float v[M];
#pragma unroll
    for (int m = 0; m < M; m++) {
        const int lo = m & ((1 << J) - 1);
        const int hi = (m >> J) << (J + 1);
        const int m0 = hi | lo, m1 = m0 | (1 << J);
        v[m] = (float)((tt >> m1) & 1u) - (float)((tt >> m0) & 1u);
    }
#pragma unroll
    for (int i = 0; i < K; i++) {
        if (i == J) continue;
        const int f = i < J ? i : i - 1;  // folds already done
#pragma unroll
        for (int m = 0; m < (M >> (f + 1)); m++) v[m] = fmaf(p[i], v[2 * m + 1], q[i] * v[2 * m]);
    }
    return v[0];
}

// all partials of a cell into d[0..3] (unused slots 0)
__device__ __forceinline__ void cell_partials(int k, uint32_t tt, const float (&p)[4], const float (&q)[4],
                                              float (&d)[4]) {
    d[0] = d[1] = d[2] = d[3] = 0.f;
    switch (k) {
        case 0: break;
        case 1: d[0] = ml_partial<1, 0>(tt, p, q); break;
        case 2: d[0] = ml_partial<2, 0>(tt, p, q); d[1] = ml_partial<2, 1>(tt, p, q); break;
        case 3:
            d[0] = ml_partial<3, 0>(tt, p, q); d[1] = ml_partial<3, 1>(tt, p, q); d[2] = ml_partial<3, 2>(tt, p, q);
            break;
        default:
            d[0] = ml_partial<4, 0>(tt, p, q); d[1] = ml_partial<4, 1>(tt, p, q);
            d[2] = ml_partial<4, 2>(tt, p, q); d[3] = ml_partial<4, 3>(tt, p, q);
            break;
    }
}

// The gradients that do not go through the adjoint, one element each (alpha: TR_model, or the
// hybrid TR; K in binary32): d P / d C_load of user net u, d P / d pincap of user cell u (K times
// the alpha of the cell's input nets), d P / d TR_in of startpoint k (K beta C_load in tr_mode 0).
__device__ __forceinline__ float grad_cload_of(const float *alpha, const int32_t *net_of_user, float K, int64_t u) {
    return K * alpha[net_of_user[u]];
}
__device__ __forceinline__ float grad_pincap_of(const uint4 *fanin, const float *alpha, const int32_t *cell_of_user,
                                                float K, int64_t u, const OpTable &ops) {
    const uint4 r = fanin[cell_of_user[u]];
    const int k = op_arity(ops, r.x >> 24);
    const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++)
        if (j < k) s += alpha[n[j]];
    return K * s;
}
__device__ __forceinline__ float grad_tr_in_of(const float *beta, const float *cload, float K, int tr_mode, int64_t k) {
    return tr_mode ? 0.f : K * (beta ? beta[k] : 1.f) * cload[k];
}

// butterfly sum of one double per lane over the warp (every lane gets the sum); the power
// reductions use this one function, so their order is the same wherever they run
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// The adjoint's local term 2 K C (Q - P) (the derivative of K C 2PQ with respect to P) and its
// combination with the fanout sum acc -- grad_mode 0: acc + local; 1: beta (acc + local)
// (Eq. 6); 2: acc + beta local.  Every operation is rounded on its own (no contraction into
// an FMA, which the compiler may or may not form depending on the surrounding code), so every
// schedule gives the same bits.
__device__ __forceinline__ float adj_local(float K, float cl, float qmp) {
    return __fmul_rn(__fmul_rn(__fmul_rn(2.f, K), cl), qmp);
}
__device__ __forceinline__ float adj_combine(int grad_mode, float acc, float local, float b) {
    if (grad_mode == 1) return __fmul_rn(b, __fadd_rn(acc, local));
    if (grad_mode == 2) return __fadd_rn(acc, __fmul_rn(b, local));
    return __fadd_rn(acc, local);
}

// Sum of a net's edge adjoints gfo[e0..e1) in index order (the order every
// schedule uses, so results match bit for bit).  Loads go out in batches of
// 8 before the additions, so a high-fanout net costs one L2 round trip per
// batch instead of one per edge.
__device__ __forceinline__ float fanout_sum_l2(const float *gfo, int32_t e0, int32_t e1) {
    float acc = 0.f;
    for (int32_t e = e0; e < e1; e += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = e + i < e1 ? __ldcg(gfo + e + i) : 0.f;
#pragma unroll
        for (int i = 0; i < 8; i++)
            if (e + i < e1) acc += v[i];
    }
    return acc;
}

// The cell's Boolean function on 64 lanes at once: a multiplexer tree over
// the truth table, selecting on input 0 first (one LOP3 per mux and half word).
template <int K>
__device__ __forceinline__ uint64_t bits_eval(uint32_t tt, const uint64_t (&x)[4]) {
    uint64_t v[1 << K];
#pragma unroll
    for (int m = 0; m < (1 << K); m++) v[m] = ((tt >> m) & 1u) ? ~0ull : 0ull;
#pragma unroll
    for (int i = 0; i < K; i++) {
#pragma unroll
        for (int m = 0; m < (1 << (K - 1 - i)); m++) v[m] = (x[i] & v[2 * m + 1]) | (~x[i] & v[2 * m]);
    }
    return v[0];
}

__device__ __forceinline__ uint64_t cell_bits(int k, uint32_t tt, const uint64_t (&x)[4]) {
    switch (k) {
        case 0: return (tt & 1u) ? ~0ull : 0ull;
        case 1: return bits_eval<1>(tt, x);
        case 2: return bits_eval<2>(tt, x);
        case 3: return bits_eval<3>(tt, x);
        default: return bits_eval<4>(tt, x);
    }
}

// One LOP3 (any 3-input Boolean function, table as an immediate) per 32 bits.
template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}

// Two 64-bit words of a cell with at most 3 inputs: the cell's 8-bit LOP3
// table selects, through one warp-uniform indirect branch, the LOP3
// instruction carrying that table, applied to (x2, x1, x0).
__device__ __forceinline__ void cell_bits_lop3(uint32_t lut, const uint64_t (&x0)[4], const uint64_t (&x1)[4],
                                               uint64_t &w0, uint64_t &w1) {
    const uint32_t a0 = (uint32_t)x0[2], b0 = (uint32_t)x0[1], c0 = (uint32_t)x0[0];
    const uint32_t a1 = (uint32_t)(x0[2] >> 32), b1 = (uint32_t)(x0[1] >> 32), c1 = (uint32_t)(x0[0] >> 32);
    const uint32_t a2 = (uint32_t)x1[2], b2 = (uint32_t)x1[1], c2 = (uint32_t)x1[0];
    const uint32_t a3 = (uint32_t)(x1[2] >> 32), b3 = (uint32_t)(x1[1] >> 32), c3 = (uint32_t)(x1[0] >> 32);
    uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    switch (lut) {
#define DP_LOP3_CASE(N)                  \
    case N:                              \
        r0 = lop3<N>(a0, b0, c0);        \
        r1 = lop3<N>(a1, b1, c1);        \
        r2 = lop3<N>(a2, b2, c2);        \
        r3 = lop3<N>(a3, b3, c3);        \
        break;
#define DP_LOP3_4(N) DP_LOP3_CASE(N) DP_LOP3_CASE(N + 1) DP_LOP3_CASE(N + 2) DP_LOP3_CASE(N + 3)
#define DP_LOP3_16(N) DP_LOP3_4(N) DP_LOP3_4(N + 4) DP_LOP3_4(N + 8) DP_LOP3_4(N + 12)
#define DP_LOP3_64(N) DP_LOP3_16(N) DP_LOP3_16(N + 16) DP_LOP3_16(N + 32) DP_LOP3_16(N + 48)
        DP_LOP3_64(0) DP_LOP3_64(64) DP_LOP3_64(128) DP_LOP3_64(192)
#undef DP_LOP3_64
#undef DP_LOP3_16
#undef DP_LOP3_4
#undef DP_LOP3_CASE
        default: break;
    }
    w0 = (uint64_t)r0 | ((uint64_t)r1 << 32);
    w1 = (uint64_t)r2 | ((uint64_t)r3 << 32);
}

// Four 64-bit words of a cell (x[j][i] = word i of input j): two LOP3 pairs
// for up to 3 inputs, the multiplexer tree for 4.
__device__ __forceinline__ void cell_words4(int k, uint32_t tt, uint32_t lut, const uint64_t (&x)[4][4],
                                            uint64_t (&w)[4]) {
    if (k <= 3) {
        const uint64_t a0[4] = {x[0][0], x[1][0], x[2][0], 0}, a1[4] = {x[0][1], x[1][1], x[2][1], 0};
        const uint64_t b0[4] = {x[0][2], x[1][2], x[2][2], 0}, b1[4] = {x[0][3], x[1][3], x[2][3], 0};
        cell_bits_lop3(lut, a0, a1, w[0], w[1]);
        cell_bits_lop3(lut, b0, b1, w[2], w[3]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint64_t xi[4] = {x[0][i], x[1][i], x[2][i], x[3][i]};
            w[i] = bits_eval<4>(tt, xi);
        }
    }
}

// both words of a cell, LOP3 for up to 3 inputs, multiplexer tree for 4
__device__ __forceinline__ void cell_bits2(int k, uint32_t tt, uint32_t lut, const uint64_t (&x0)[4],
                                           const uint64_t (&x1)[4], uint64_t &w0, uint64_t &w1) {
    if (k <= 3) {
        cell_bits_lop3(lut, x0, x1, w0, w1);
    } else {
        w0 = bits_eval<4>(tt, x0);
        w1 = bits_eval<4>(tt, x1);
    }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): per round the two even
// words are multiplied by the round constants, the high halves are xored with
// the odd words and the key, and the key advances by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

}  // namespace dp
