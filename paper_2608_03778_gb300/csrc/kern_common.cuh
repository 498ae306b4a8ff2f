// Device helpers shared by the kernels: cell evaluation on probabilities and
// on bit-packed words, and the Philox4x32-10 counter generator.
#pragma once
#include <cstdint>

#include "kernels.h"

namespace dp {

constexpr uint32_t kMask24 = 0xFFFFFFu;

__device__ __forceinline__ int op_arity(const OpTable &t, uint32_t op) { return (int)(t.e[op] >> 16); }
__device__ __forceinline__ uint32_t op_tt(const OpTable &t, uint32_t op) { return t.e[op] & 0xFFFFu; }

// SP of a cell with K inputs: the multilinear extension of its truth table,
// sum_m f(m) prod_i (m_i ? a_i : 1 - a_i), evaluated as nested linear
// interpolations along inputs 0, 1, ... (exact under input independence,
// Sec. III-B; equals the stack interpreter of Algorithm 2 on read-once cells).
template <int K>
__device__ __forceinline__ float ml_eval(uint32_t tt, const float (&a)[4]) {
    float v[1 << K];
#pragma unroll
    for (int m = 0; m < (1 << K); m++) v[m] = (float)((tt >> m) & 1u);
#pragma unroll
    for (int i = 0; i < K; i++) {
#pragma unroll
        for (int m = 0; m < (1 << (K - 1 - i)); m++) v[m] = fmaf(a[i], v[2 * m + 1] - v[2 * m], v[2 * m]);
    }
    return v[0];
}

// d SP / d a_J: the multilinear extension, over the other inputs, of the
// difference table f(.., a_J = 1, ..) - f(.., a_J = 0, ..) (entries in {-1,0,1},
// so no cancellation between two large values).
template <int K, int J>
__device__ __forceinline__ float ml_partial(uint32_t tt, const float (&a)[4]) {
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
        for (int m = 0; m < (M >> (f + 1)); m++) v[m] = fmaf(a[i], v[2 * m + 1] - v[2 * m], v[2 * m]);
    }
    return v[0];
}

__device__ __forceinline__ float cell_sp(int k, uint32_t tt, const float (&a)[4]) {
    switch (k) {
        case 0: return (float)(tt & 1u);
        case 1: return ml_eval<1>(tt, a);
        case 2: return ml_eval<2>(tt, a);
        case 3: return ml_eval<3>(tt, a);
        default: return ml_eval<4>(tt, a);
    }
}

// all partials of a cell into d[0..3] (unused slots 0)
__device__ __forceinline__ void cell_partials(int k, uint32_t tt, const float (&a)[4], float (&d)[4]) {
    d[0] = d[1] = d[2] = d[3] = 0.f;
    switch (k) {
        case 0: break;
        case 1: d[0] = ml_partial<1, 0>(tt, a); break;
        case 2: d[0] = ml_partial<2, 0>(tt, a); d[1] = ml_partial<2, 1>(tt, a); break;
        case 3:
            d[0] = ml_partial<3, 0>(tt, a); d[1] = ml_partial<3, 1>(tt, a); d[2] = ml_partial<3, 2>(tt, a);
            break;
        default:
            d[0] = ml_partial<4, 0>(tt, a); d[1] = ml_partial<4, 1>(tt, a);
            d[2] = ml_partial<4, 2>(tt, a); d[3] = ml_partial<4, 3>(tt, a);
            break;
    }
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
