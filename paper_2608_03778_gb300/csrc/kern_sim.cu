// Pass 2 (Sec. III-C): Markov-chain startpoint vectors, bit-packed level-by-
// level simulation with PopCount toggle counting (Eq. 4), and the hybrid
// calibration beta = clip(TR_acc / TR_model) (Sec. III-D, Eq. 5).
//
// Layout: words[n * T + t], bit b of word t = lane b (an independent chain)
// at cycle t; T words give 64 T vectors and 64 (T - 1) transitions per net.
#include "kern_common.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// floor(p * 2^16) clamped to [0, 2^16]: a 16-bit draw u is 1 iff u < thr
__device__ __forceinline__ uint32_t threshold16(double p) {
    if (!(p > 0.0)) return 0u;
    if (p >= 1.0) return 65536u;
    return (uint32_t)floor(p * 65536.0);
}

// One half-warp per startpoint k; thread q runs lanes q, q+16, q+32, q+48.
// Philox4x32-10 counter (k, t / 2, q, 0) under key (seed lo, seed hi);
// output component r drives lane 16 r + q, its low 16 bits at even cycles
// and its high 16 bits at odd cycles.  t = 0 draws the initial state with
// P(1) = SP; t >= 1 flips a 1 with p10 = TR / 2SP and a 0 with
// p01 = TR / 2(1 - SP), which keeps SP stationary and makes TR the expected
// toggle rate.  The four lanes' states live in a 4-bit mask; the 64-bit word
// of each cycle is assembled from four warp ballots.
__global__ void __launch_bounds__(256) k_sim_start(const float *__restrict__ sp_in, const float *__restrict__ tr_in,
                                                   uint64_t *words, uint32_t *toggles, uint32_t *ones, int64_t ns,
                                                   int T, uint32_t key0, uint32_t key1) {
    const int q = threadIdx.x & 15;
    const int half = (threadIdx.x >> 4) & 1;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
    const bool valid = k < ns;
    // the three thresholds of startpoint k, computed by one thread of its half-warp (the
    // divisions run on the FP64 pipe, slow on this part) and shared with the other fifteen
    uint32_t t_init = 0, t10 = 0, t01 = 0;
    if (valid && q == 0) {
        const double sp = (double)sp_in[k], tr = (double)tr_in[k];
        const double p10 = sp > 0.0 ? tr / (2.0 * sp) : 0.0;
        const double p01 = sp < 1.0 ? tr / (2.0 * (1.0 - sp)) : 0.0;
        t_init = threshold16(sp);
        t10 = threshold16(p10);
        t01 = threshold16(p01);
    }
    t_init = __shfl_sync(0xFFFFFFFFu, t_init, 0, 16);
    t10 = __shfl_sync(0xFFFFFFFFu, t10, 0, 16);
    t01 = __shfl_sync(0xFFFFFFFFu, t01, 0, 16);
    const uint32_t sel = half ? 0x7632u : 0x5410u;  // this half-warp's 16 ballot bits of two ballots
    uint32_t st = 0;                                // bit r = current value of lane 16 r + q
    uint32_t n_flip = 0, n_one = 0;
    uint64_t mine = 0;                              // word t with t % 16 == q of the current 16 cycles
    uint4 u = make_uint4(0, 0, 0, 0);
    for (int t = 0; t < T; t++) {
        if ((t & 1) == 0) u = philox4x32_10(make_uint4((uint32_t)k, (uint32_t)(t >> 1), (uint32_t)q, 0u), key0, key1);
        const int sh = (t & 1) << 4;
        const uint32_t d0 = (u.x >> sh) & 0xFFFFu, d1 = (u.y >> sh) & 0xFFFFu;
        const uint32_t d2 = (u.z >> sh) & 0xFFFFu, d3 = (u.w >> sh) & 0xFFFFu;
        if (t == 0) {
            st = (uint32_t)(d0 < t_init) | ((uint32_t)(d1 < t_init) << 1) | ((uint32_t)(d2 < t_init) << 2) |
                 ((uint32_t)(d3 < t_init) << 3);
        } else {
            const uint32_t f = (uint32_t)(d0 < ((st & 1u) ? t10 : t01)) |
                               ((uint32_t)(d1 < ((st & 2u) ? t10 : t01)) << 1) |
                               ((uint32_t)(d2 < ((st & 4u) ? t10 : t01)) << 2) |
                               ((uint32_t)(d3 < ((st & 8u) ? t10 : t01)) << 3);
            n_flip += __popc(f);
            st ^= f;
        }
        n_one += __popc(st);
        const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, st & 1u), b1 = __ballot_sync(0xFFFFFFFFu, st & 2u);
        const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, st & 4u), b3 = __ballot_sync(0xFFFFFFFFu, st & 8u);
        const uint64_t w = (uint64_t)__byte_perm(b0, b1, sel) | ((uint64_t)__byte_perm(b2, b3, sel) << 32);
        if ((t & 15) == q) mine = w;
        if ((t & 15) == 15 || t == T - 1) {
            const int t_q = (t & ~15) + q;
            if (valid && t_q < T) words[k * T + t_q] = mine;
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        n_flip += __shfl_xor_sync(0xFFFFFFFFu, n_flip, o);
        n_one += __shfl_xor_sync(0xFFFFFFFFu, n_one, o);
    }
    if (valid && q == 0) {
        toggles[k] = n_flip;
        ones[k] = n_one;
    }
}

// The same chains for T a multiple of 16, arranged for fewer instructions: one
// Philox call per two cycles with its low and high halves at fixed positions,
// sixteen cycles unrolled per block (so the word a thread keeps and the store
// are fixed at compile time), and the first cycle - the initial draw -
// peeled off.  Each flip is formed from both threshold tests and the state by
// one bitwise select.  Identical bits to k_sim_start.
struct ChainState {
    uint32_t st, n_flip, n_one;
};

// one cycle: the four lanes' 16-bit draws d[r]; FIRST draws the initial state
template <bool FIRST>
__device__ __forceinline__ uint64_t chain_cycle(ChainState &c, const uint32_t (&d)[4], uint32_t t_init, uint32_t t10,
                                                uint32_t t01, uint32_t sel) {
    if (FIRST) {
        c.st = (uint32_t)(d[0] < t_init) | ((uint32_t)(d[1] < t_init) << 1) | ((uint32_t)(d[2] < t_init) << 2) |
               ((uint32_t)(d[3] < t_init) << 3);
    } else {
        const uint32_t c10 = (uint32_t)(d[0] < t10) | ((uint32_t)(d[1] < t10) << 1) | ((uint32_t)(d[2] < t10) << 2) |
                             ((uint32_t)(d[3] < t10) << 3);
        const uint32_t c01 = (uint32_t)(d[0] < t01) | ((uint32_t)(d[1] < t01) << 1) | ((uint32_t)(d[2] < t01) << 2) |
                             ((uint32_t)(d[3] < t01) << 3);
        const uint32_t f = (c.st & c10) | (~c.st & c01 & 15u);   // a 1 flips on p10, a 0 on p01
        c.n_flip += __popc(f);
        c.st ^= f;
    }
    c.n_one += __popc(c.st);
    const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, c.st & 1u), b1 = __ballot_sync(0xFFFFFFFFu, c.st & 2u);
    const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, c.st & 4u), b3 = __ballot_sync(0xFFFFFFFFu, c.st & 8u);
    return (uint64_t)__byte_perm(b0, b1, sel) | ((uint64_t)__byte_perm(b2, b3, sel) << 32);
}

// sixteen cycles from cycle t0 (a multiple of 16): thread q returns word t0 + q
template <bool FIRST>
__device__ __forceinline__ uint64_t chain_block16(ChainState &c, uint32_t k, int t0, int q, uint32_t key0,
                                                  uint32_t key1, uint32_t t_init, uint32_t t10, uint32_t t01,
                                                  uint32_t sel) {
    uint64_t mine = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint4 u = philox4x32_10(make_uint4(k, (uint32_t)((t0 >> 1) + i), (uint32_t)q, 0u), key0, key1);
        const uint32_t lo[4] = {u.x & 0xFFFFu, u.y & 0xFFFFu, u.z & 0xFFFFu, u.w & 0xFFFFu};
        const uint32_t hi[4] = {u.x >> 16, u.y >> 16, u.z >> 16, u.w >> 16};
        const uint64_t w0 = (FIRST && i == 0) ? chain_cycle<true>(c, lo, t_init, t10, t01, sel)
                                              : chain_cycle<false>(c, lo, t_init, t10, t01, sel);
        const uint64_t w1 = chain_cycle<false>(c, hi, t_init, t10, t01, sel);
        if (q == 2 * i) mine = w0;
        if (q == 2 * i + 1) mine = w1;
    }
    return mine;
}

// Fast form of the same chains when every threshold of the warp is below 2^16
// (no probability of exactly 1): a 16-bit draw d is compared in the high half
// of a 32-bit word against thr << 16, which holds whatever the low half is, so
// the high-half draws need no extraction.  Each lane keeps only the threshold
// of its current state (t10 in state 1, t01 in state 0; a flip toggles it by
// one XOR).  The warp votes on the flips, and the cycle's word is the previous
// word XOR the flip word, so no lane state is formed.  Ones and toggles are
// counted from the finished words.
struct FastChain {
    uint32_t thr[4];
    uint64_t word;   // lane states of the previous cycle (this half-warp's startpoint)
};

// one cycle on draws d[r] (in the high half); FIRST draws the initial state
template <bool FIRST>
__device__ __forceinline__ uint64_t fast_cycle(FastChain &c, const uint32_t (&d)[4], uint32_t ti16, uint32_t t10_16,
                                               uint32_t t01_16, uint32_t sel) {
    bool b[4];   // FIRST: the initial state; else: a flip
#pragma unroll
    for (int r = 0; r < 4; r++) {
        if (FIRST) {
            b[r] = d[r] < ti16;
            c.thr[r] = b[r] ? t10_16 : t01_16;
        } else {
            b[r] = d[r] < c.thr[r];
            c.thr[r] ^= b[r] ? (t10_16 ^ t01_16) : 0u;
        }
    }
    const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, b[0]), b1 = __ballot_sync(0xFFFFFFFFu, b[1]);
    const uint32_t b2 = __ballot_sync(0xFFFFFFFFu, b[2]), b3 = __ballot_sync(0xFFFFFFFFu, b[3]);
    const uint64_t w = (uint64_t)__byte_perm(b0, b1, sel) | ((uint64_t)__byte_perm(b2, b3, sel) << 32);
    c.word = FIRST ? w : c.word ^ w;
    return c.word;
}

template <bool FIRST>
__device__ __forceinline__ uint64_t fast_block16(FastChain &c, uint32_t k, int t0, int q, uint32_t key0,
                                                 uint32_t key1, uint32_t ti16, uint32_t t10_16, uint32_t t01_16,
                                                 uint32_t sel) {
    uint64_t mine = 0;
    // unrolled by 4, not 8: fully unrolled, the compiler keeps several calls' draws live
    // (124 registers); at 4 the kernel needs 48 and more warps fit on an SM
#pragma unroll 4
    for (int i = 0; i < 8; i++) {
        const uint4 u = philox4x32_10(make_uint4(k, (uint32_t)((t0 >> 1) + i), (uint32_t)q, 0u), key0, key1);
        const uint32_t lo[4] = {u.x << 16, u.y << 16, u.z << 16, u.w << 16};
        const uint32_t hi[4] = {u.x, u.y, u.z, u.w};
        const uint64_t w0 = (FIRST && i == 0) ? fast_cycle<true>(c, lo, ti16, t10_16, t01_16, sel)
                                              : fast_cycle<false>(c, lo, ti16, t10_16, t01_16, sel);
        const uint64_t w1 = fast_cycle<false>(c, hi, ti16, t10_16, t01_16, sel);
        if (q == 2 * i) mine = w0;
        if (q == 2 * i + 1) mine = w1;
    }
    return mine;
}

__global__ void __launch_bounds__(256) k_sim_start16(const float *__restrict__ sp_in, const float *__restrict__ tr_in,
                                                     uint64_t *words, uint32_t *toggles, uint32_t *ones, int64_t ns,
                                                     int T, uint32_t key0, uint32_t key1) {
    const int q = threadIdx.x & 15;
    const int half = (threadIdx.x >> 4) & 1;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4);
    const bool valid = k < ns;
    uint32_t t_init = 0, t10 = 0, t01 = 0;
    if (valid && q == 0) {
        const double sp = (double)sp_in[k], tr = (double)tr_in[k];
        const double p10 = sp > 0.0 ? tr / (2.0 * sp) : 0.0;
        const double p01 = sp < 1.0 ? tr / (2.0 * (1.0 - sp)) : 0.0;
        t_init = threshold16(sp);
        t10 = threshold16(p10);
        t01 = threshold16(p01);
    }
    t_init = __shfl_sync(0xFFFFFFFFu, t_init, 0, 16);
    t10 = __shfl_sync(0xFFFFFFFFu, t10, 0, 16);
    t01 = __shfl_sync(0xFFFFFFFFu, t01, 0, 16);
    const uint32_t sel = half ? 0x7632u : 0x5410u;
    uint64_t *out = words + (valid ? k : 0) * T;
    if (!__any_sync(0xFFFFFFFFu, (t_init | t10 | t01) >= 65536u)) {   // warp-uniform
        FastChain c{};
        uint32_t n_one = 0, n_flip = 0;
        uint64_t carry = 0;
        for (int t0 = 0; t0 < T; t0 += 16) {
            const uint64_t w = t0 == 0 ? fast_block16<true>(c, (uint32_t)k, 0, q, key0, key1, t_init << 16,
                                                            t10 << 16, t01 << 16, sel)
                                       : fast_block16<false>(c, (uint32_t)k, t0, q, key0, key1, t_init << 16,
                                                             t10 << 16, t01 << 16, sel);
            if (valid) out[t0 + q] = w;
            const uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, w, 1, 16);
            n_one += __popcll(w);
            if (t0 + q > 0) n_flip += __popcll(w ^ (q > 0 ? prev : carry));
            carry = __shfl_sync(0xFFFFFFFFu, w, 15, 16);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            n_flip += __shfl_xor_sync(0xFFFFFFFFu, n_flip, o);
            n_one += __shfl_xor_sync(0xFFFFFFFFu, n_one, o);
        }
        if (valid && q == 0) {
            toggles[k] = n_flip;
            ones[k] = n_one;
        }
        return;
    }
    ChainState c{0u, 0u, 0u};
    uint64_t w = chain_block16<true>(c, (uint32_t)k, 0, q, key0, key1, t_init, t10, t01, sel);
    if (valid) out[q] = w;
    for (int t0 = 16; t0 < T; t0 += 16) {
        w = chain_block16<false>(c, (uint32_t)k, t0, q, key0, key1, t_init, t10, t01, sel);
        if (valid) out[t0 + q] = w;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        c.n_flip += __shfl_xor_sync(0xFFFFFFFFu, c.n_flip, o);
        c.n_one += __shfl_xor_sync(0xFFFFFFFFu, c.n_one, o);
    }
    if (valid && q == 0) {
        toggles[k] = c.n_flip;
        ones[k] = c.n_one;
    }
}

// One warp per cell of a level: lane l evaluates word t = 32 i + l of the
// cell on its fanin words (bitwise), writes it, and counts ones and toggles;
// the previous word comes from the neighbour lane (or the last lane of the
// previous chunk).
__global__ void __launch_bounds__(256) k_sim_level(const uint4 *__restrict__ fanin, uint64_t *words,
                                                   uint32_t *toggles, uint32_t *ones, int32_t c0, int32_t c1,
                                                   int64_t ns, int T, OpTable ops) {
    const int lane = threadIdx.x & 31;
    const int32_t c = c0 + (int32_t)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= c1) return;  // whole warp
    const uint4 r = fanin[c];
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    const uint32_t tt = op_tt(ops, op);
    // fanin rows (slots beyond the arity are unused and never formed)
    const uint64_t *in0 = k > 0 ? words + (size_t)(r.x & kMask24) * T : words;
    const uint64_t *in1 = k > 1 ? words + (size_t)r.y * T : words;
    const uint64_t *in2 = k > 2 ? words + (size_t)r.z * T : words;
    const uint64_t *in3 = k > 3 ? words + (size_t)r.w * T : words;
    uint64_t *out = words + (size_t)(ns + c) * T;
    uint32_t tg = 0, on = 0;
    uint64_t carry = 0;
    for (int base = 0; base < T; base += 32) {
        const int t = base + lane;
        const bool act = t < T;
        uint64_t x[4] = {0, 0, 0, 0};
        if (act) {
            if (k > 0) x[0] = in0[t];
            if (k > 1) x[1] = in1[t];
            if (k > 2) x[2] = in2[t];
            if (k > 3) x[3] = in3[t];
        }
        const uint64_t w = cell_bits(k, tt, x);
        uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, w, 1);
        if (lane == 0) prev = carry;
        if (act) {
            out[t] = w;
            on += __popcll(w);
            if (t > 0) tg += __popcll(w ^ prev);
        }
        carry = __shfl_sync(0xFFFFFFFFu, w, 31);
    }
    tg = __reduce_add_sync(0xFFFFFFFFu, tg);
    on = __reduce_add_sync(0xFFFFFFFFu, on);
    if (lane == 0) {
        toggles[ns + c] = tg;
        ones[ns + c] = on;
    }
}

// Eq. 4 and Eq. 5: TR_acc = toggles / 64(T-1); beta = clip(TR_acc / TR_model);
// TR_model = 0 gives beta = 1 without toggles, else beta_max.  The ratio is
// formed in float-float from the float-float (P, Q) pair and rounded once:
// the paper's gradient rule multiplies by beta at every net (Eq. 6), so
// beta's rounding error compounds along paths.
__global__ void k_hybrid(const uint32_t *__restrict__ toggles, const float *__restrict__ tr,
                         const float4 *__restrict__ pq, float *beta, float *trh, int64_t nn, int64_t ns, int tr_mode,
                         float nsim, float bmin, float bmax) {
    int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nn) return;
    const uint32_t tg = toggles[n];
    const float m = tr[n];
    ff model;
    if (n < ns && tr_mode == 0) {
        model = ff_make(m);
    } else {
        const float4 v = pq_decode(pq[n]);
        const ff t = ff_mul(ff{v.x, v.y}, ff{v.z, v.w});
        model = ff{2.f * t.hi, 2.f * t.lo};
    }
    float b;
    if (model.hi > 0.f) {
        const ff r = ff_div(ff_div(ff_make((float)tg), ff_make(nsim)), model);
        b = fminf(fmaxf(r.hi + r.lo, bmin), bmax);
    } else {
        b = tg == 0 ? 1.f : bmax;
    }
    beta[n] = b;
    trh[n] = b * m;
}

}  // namespace

void launch_sim_start(const DevDesign &d, int T, uint64_t seed, cudaStream_t s) {
    if (d.n_start == 0) return;
    if (T % 16 == 0) {
        k_sim_start16<<<(unsigned)cdiv(d.n_start, 16), 256, 0, s>>>(d.sp_in, d.tr_in, d.words, d.toggles, d.ones,
                                                                    d.n_start, T, (uint32_t)seed,
                                                                    (uint32_t)(seed >> 32));
        return;
    }
    k_sim_start<<<(unsigned)cdiv(d.n_start, 16), 256, 0, s>>>(d.sp_in, d.tr_in, d.words, d.toggles, d.ones,
                                                              d.n_start, T, (uint32_t)seed, (uint32_t)(seed >> 32));
}

void launch_sim_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, int T, cudaStream_t s) {
    if (c1 <= c0) return;
    k_sim_level<<<(unsigned)cdiv((int64_t)(c1 - c0) * 32, 256), 256, 0, s>>>(d.fanin, d.words, d.toggles, d.ones,
                                                                              c0, c1, d.n_start, T, ops);
}

void launch_hybrid(const DevDesign &d, int T, int tr_mode, float beta_min, float beta_max, cudaStream_t s) {
    if (d.n_nets == 0) return;
    const float nsim = 64.f * (float)(T - 1);
    k_hybrid<<<(unsigned)cdiv(d.n_nets, 256), 256, 0, s>>>(d.toggles, d.tr, d.pq, d.beta, d.trh, d.n_nets,
                                                           d.n_start, tr_mode, nsim, beta_min, beta_max);
}

}  // namespace dp
