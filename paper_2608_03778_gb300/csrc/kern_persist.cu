// Persistent schedule: one cooperative launch per pass (forward, simulation,
// backward) that walks all levels, with a grid-wide barrier between levels
// instead of one kernel launch per level.  Every wait is bounded: a block
// that waits longer than the limit records an error word and returns, the
// others see the word and return too, and the host reports DP_ETIMEOUT.
//
// Data written by other blocks during the launch is read through L2
// (ld.global.cg); the barrier's release/acquire pair orders it.  Static data
// of the next level (fanin records, fanout ranges, forward results) is loaded
// between a block's arrival at the barrier and its wait, so the wait hides its
// latency.
#include "kern_common.cuh"

namespace dp {
namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Level barrier over all blocks of the grid, in two halves.  Each barrier of a
// launch has its own arrival counter (own 128-byte line, zeroed before the
// launch).  barrier_arrive: once every thread of the block is done with the
// level, thread 0 arrives with a release reduction (no round trip).
// barrier_wait: thread 0 polls the counter with acquire loads until every
// block has arrived; returns false, identically in every thread of the block,
// when the wait gave up (limit reached, or another block reported an error).
// Between the two a block may load whatever does not depend on the other
// blocks' work of the level (the next level's static data), so those loads
// overlap the barrier's latency instead of delaying the block's arrival.
__device__ __forceinline__ void barrier_arrive(unsigned *ctr) {
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

__device__ bool barrier_wait(unsigned *ctr, int *err, unsigned nblocks, long long limit) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = clock64();
        unsigned spins = 0;
        while (ld_acquire_u32(ctr) < nblocks) {
            if ((++spins & 255u) == 0) {
                if (ld_relaxed_u32(reinterpret_cast<unsigned *>(err)) != 0) { ok = 0; break; }
                if (clock64() - t0 > limit) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ bool level_barrier(unsigned *ctr, int *err, unsigned nblocks, long long limit) {
    barrier_arrive(ctr);
    return barrier_wait(ctr, err, nblocks, limit);
}

// L2 prefetch of one line; the persistent passes fetch a level's static data two
// levels ahead, so its DRAM latency is hidden by a whole level instead of by the
// part of one barrier that follows a block's arrival
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// thread index that spreads consecutive 32-element groups over all blocks
// (and so over all SMs) before giving any block a second warp of work
__device__ __forceinline__ int64_t spread_tid() {
    return ((int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
}
__device__ __forceinline__ int64_t spread_warp() { return (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; }

// ---------------------------------------------------------------- forward
__device__ __forceinline__ void fwd_cell(const uint4 &r, int64_t c, float4 *pq, float *tr, int64_t ns,
                                         const OpTable &ops, uint32_t par) {
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    pair_ff x[4];
    gather_ff<true>(pq, r, k, x);
    const pair_ff o = cell_pair(k, op_tt(ops, op), x);
    pq[ns + c] = pair_store(o, par);
    tr[ns + c] = pair_tr(o);
}

__global__ void __launch_bounds__(kFwdThreads) k_fwd_persist(
    const uint4 *__restrict__ fanin, float4 *pq, float *tr, const float *__restrict__ sp_in,
    const float *__restrict__ tr_in, const int32_t *__restrict__ lvl, int L, int64_t ns, int tr_mode, OpTable ops,
    unsigned *bar, int *err, long long limit, const uint32_t *epoch) {
    const int64_t tid = spread_tid();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const uint32_t par = epoch[0] & 1u;
    for (int64_t k = tid; k < ns; k += T) {
        const pair_ff a = pair_of(sp_in[k]);
        pq[k] = pair_store(a, par);
        tr[k] = tr_mode ? pair_tr(a) : tr_in[k];
    }
    for (int l = 1; l <= L; l++) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        const int64_t c = c0 + tid;
        barrier_arrive(bar + 32 * (l - 1));
        uint4 r = make_uint4(0, 0, 0, 0);
        if (c < c1) r = fanin[c];   // static: loaded between arrival and wait
        if (l + 2 <= L) {
            const int64_t cp = lvl[l + 1] + tid;
            if (cp < lvl[l + 2]) prefetch_l2(fanin + cp);
        }
        if (!barrier_wait(bar + 32 * (l - 1), err, gridDim.x, limit)) return;
        if (c < c1) fwd_cell(r, c, pq, tr, ns, ops, par);
        for (int64_t cc = c + T; cc < c1; cc += T) fwd_cell(fanin[cc], cc, pq, tr, ns, ops, par);
    }
}

// --------------------------------------------------------------- backward
__device__ __forceinline__ float combine(int grad_mode, float acc, float local, float b) {
    return adj_combine(grad_mode, acc, local, b);
}

// everything the adjoint of one cell needs except its fanout contributions
struct BwdStatic {
    int32_t e0, e1;
    int4 ep;
    float local, b;
    float d[4];
    int k;
};

__device__ __forceinline__ BwdStatic bwd_static_r(const uint4 &r, const int32_t *fptr, const int4 *efpos,
                                                  const float4 *pq, const float *cload, const float *beta, int64_t c,
                                                  int64_t ns, int grad_mode, float K, const OpTable &ops) {
    BwdStatic s;
    const int64_t n = ns + c;
    s.ep = efpos[c];
    s.e0 = fptr[n];
    s.e1 = fptr[n + 1];
    // local term: d(K C 2P(1-P))/dP = 2 K C (Q - P)
    s.local = adj_local(K, cload[n], pair_qmp(pq[n]));
    s.b = grad_mode ? beta[n] : 1.f;
    const uint32_t op = r.x >> 24;
    s.k = op_arity(ops, op);
    float p[4], q[4];
    gather_pairs(pq, r, s.k, p, q);
    cell_partials(s.k, op_tt(ops, op), p, q, s.d);
    return s;
}

__device__ __forceinline__ BwdStatic bwd_static(const uint4 *fanin, const int32_t *fptr, const int4 *efpos,
                                                const float4 *pq, const float *cload, const float *beta, int64_t c,
                                                int64_t ns, int grad_mode, float K, const OpTable &ops) {
    return bwd_static_r(fanin[c], fptr, efpos, pq, cload, beta, c, ns, grad_mode, K, ops);
}

// the static data of one cell for the reverse pass, loaded a level before it is used (the
// fanin pairs as stored; an unused slot as the pair P = 0, Q = 1)
struct BwdPre {
    int4 ep;
    int32_t e0, e1;
    float cl, b;
    float4 self, in[4];
};

__device__ __forceinline__ void bwd_pre(BwdPre &w, const uint4 &r, const int32_t *fptr, const int4 *efpos,
                                        const float4 *pq, const float *cload, const float *beta, int64_t c,
                                        int64_t ns, int grad_mode, const OpTable &ops) {
    const int64_t n = ns + c;
    w.ep = efpos[c];
    w.e0 = fptr[n];
    w.e1 = fptr[n + 1];
    w.cl = cload[n];
    w.b = grad_mode ? beta[n] : 1.f;
    w.self = pq[n];
    const int k = op_arity(ops, r.x >> 24);
    const uint32_t nid[4] = {r.x & kMask24, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; j++) w.in[j] = j < k ? pq[nid[j]] : make_float4(0.f, 0.f, 1.f, 0.f);
}

// bwd_static_r from the preloaded data: the same operations on the same values
__device__ __forceinline__ BwdStatic bwd_static_pre(const BwdPre &w, const uint4 &r, float K, const OpTable &ops) {
    BwdStatic s;
    s.ep = w.ep;
    s.e0 = w.e0;
    s.e1 = w.e1;
    s.local = adj_local(K, w.cl, pair_qmp(w.self));
    s.b = w.b;
    const uint32_t op = r.x >> 24;
    s.k = op_arity(ops, op);
    float p[4], q[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        p[j] = 0.f;
        q[j] = 1.f;
        if (j < s.k) {
            const float4 v = pq_decode(w.in[j]);
            p[j] = v.x + v.y;
            q[j] = v.z + v.w;
        }
    }
    cell_partials(s.k, op_tt(ops, op), p, q, s.d);
    return s;
}

__device__ __forceinline__ void bwd_finish(const BwdStatic &s, int64_t n, float *gnet, float *gfo, int grad_mode) {
    const float acc = fanout_sum_l2(gfo, s.e0, s.e1);
    const float g = combine(grad_mode, acc, s.local, s.b);
    gnet[n] = g;
    if (s.k > 0) gfo[s.ep.x] = g * s.d[0];
    if (s.k > 1) gfo[s.ep.y] = g * s.d[1];
    if (s.k > 2) gfo[s.ep.z] = g * s.d[2];
    if (s.k > 3) gfo[s.ep.w] = g * s.d[3];
}

// PRE: the whole static part of a level's cell (fanout range, edge positions, C_load, beta,
// its own and its fanins' pairs) is loaded a level ahead and its fanin record two levels ahead,
// so the window between a block's arrival and its wait only computes (about 120 registers:
// the block holds its SM's register file).  Without PRE only the record is loaded a level
// ahead and the rest in the window (64 registers), for the step, whose gradient-output kernel
// runs beside this pass.
template <bool PRE>
__global__ void __launch_bounds__(kPersistThreads) k_bwd_persist(
    const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr, const int4 *__restrict__ efpos,
    const float4 *__restrict__ pq, const float *__restrict__ cload, const float *__restrict__ beta, float *gnet,
    float *gfo, const int32_t *__restrict__ lvl, int L, int64_t ns, int grad_mode, int tr_mode, float K,
    float *out_gsp, OpTable ops, unsigned *bar, int *err, long long limit) {
    const int64_t tid = spread_tid();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    auto rec = [&](int l) {   // the fanin record of this thread's cell on level l (if any)
        if (l < 1) return make_uint4(0, 0, 0, 0);
        const int64_t cl = lvl[l - 1] + tid;
        return cl < lvl[l] ? fanin[cl] : make_uint4(0, 0, 0, 0);
    };
    uint4 r1 = rec(L), r2 = PRE ? rec(L - 1) : make_uint4(0, 0, 0, 0);
    BwdPre w;
    if (PRE && L > 0 && lvl[L - 1] + tid < lvl[L])
        bwd_pre(w, r1, fptr, efpos, pq, cload, beta, lvl[L - 1] + tid, ns, grad_mode, ops);
    for (int l = L; l >= 1; l--) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        const int64_t c = c0 + tid;
        // the top level has no fanout inside the pass: no barrier before it.  Below it the
        // block arrives for the level above, then forms this level's static part (it does not
        // depend on the level above) and issues the next level's loads while the other blocks
        // arrive.
        if (l < L) barrier_arrive(bar + 32 * (L - 1 - l));
        BwdStatic s;
        if (PRE) {
            if (c < c1) s = bwd_static_pre(w, r1, K, ops);
            if (l > 1 && lvl[l - 2] + tid < lvl[l - 1])
                bwd_pre(w, r2, fptr, efpos, pq, cload, beta, lvl[l - 2] + tid, ns, grad_mode, ops);
            r1 = r2;
            r2 = rec(l - 2);
        } else {
            if (c < c1) s = bwd_static_r(r1, fptr, efpos, pq, cload, beta, c, ns, grad_mode, K, ops);
            r1 = rec(l - 1);
        }
        if (l >= 3) {
            const int64_t cp = lvl[l - 3] + tid;
            if (cp < lvl[l - 2]) {
                prefetch_l2(fanin + cp);
                prefetch_l2(efpos + cp);
                prefetch_l2(fptr + ns + cp);
                prefetch_l2(cload + ns + cp);
                if (grad_mode) prefetch_l2(beta + ns + cp);
            }
        }
        if (l < L && !barrier_wait(bar + 32 * (L - 1 - l), err, gridDim.x, limit)) return;
        if (c < c1) bwd_finish(s, ns + c, gnet, gfo, grad_mode);
        for (int64_t cc = c + T; cc < c1; cc += T)
            bwd_finish(bwd_static(fanin, fptr, efpos, pq, cload, beta, cc, ns, grad_mode, K, ops), ns + cc, gnet,
                       gfo, grad_mode);
    }
    if (!level_barrier(bar + 32 * (L - 1), err, gridDim.x, limit)) return;
    for (int64_t k = tid; k < ns; k += T) {
        const float acc = fanout_sum_l2(gfo, fptr[k], fptr[k + 1]);
        const float local = tr_mode ? adj_local(K, cload[k], pair_qmp(pq[k])) : 0.f;
        const float g = combine(grad_mode, acc, local, grad_mode ? beta[k] : 1.f);
        gnet[k] = g;
        if (out_gsp) out_gsp[k] = g;
    }
}

// ------------------------- forward and reverse of a small design in one block
// For a design whose levels hold at most kBlockMaxWidth cells and whose state
// fits in one SM's shared memory: the whole pass in a single block, one cell
// per thread and level.  The level barrier is a block barrier, and the data a
// level reads from the levels before it -- the (P, Q) pairs in the forward
// pass, the pairs and the edge adjoints in the reverse pass -- sit in shared
// memory, so a level costs a block barrier, shared-memory gathers and the
// cell's arithmetic instead of a grid-wide barrier through L2 and gathers from
// L2.  The fanin records of the next level are loaded while the current one
// computes.  Every value is computed by the same code in the same order as in
// the grid-wide passes, so the results are bitwise the same.
//
// The forward kernel also advances the pass counter (whose parity tags the stored pairs).  All
// static data a pass reads is prefetched into L2 at its start: the loads a level issues for the
// next one then wait for L2, not for DRAM.  (The model power stays with the grid-wide
// reduction kernels: the FP64 sum of a design's terms on one SM's narrow FP64 pipe took longer
// than those two launches.)
//
// Shared memory, forward: n_nets pairs, then the n_levels + 1 level bounds.  Reverse: n_nets
// pairs, n_edges edge adjoints, the level bounds.

__device__ __forceinline__ void load_bounds(int *slvl, const int32_t *lvl, int L) {
    for (int i = threadIdx.x; i <= L; i += blockDim.x) slvl[i] = lvl[i];
}

// every 128-byte line of bytes [p, p + n) into L2
__device__ __forceinline__ void prefetch_all_l2(const void *p, int64_t n) {
    const char *c = static_cast<const char *>(p);
    for (int64_t i = (int64_t)threadIdx.x * 128; i < n; i += (int64_t)blockDim.x * 128) prefetch_l2(c + i);
}

__global__ void __launch_bounds__(kBlockThreads) k_fwd_block(
    const uint4 *__restrict__ fanin, float4 *pq, float *tr, const float *__restrict__ sp_in,
    const float *__restrict__ tr_in, const int32_t *__restrict__ lvl, int L, int64_t ns, int64_t nn, int tr_mode, OpTable ops, uint32_t *epoch) {
    extern __shared__ float4 spq[];
    int *slvl = reinterpret_cast<int *>(spq + nn);
    const int t = threadIdx.x;
    const uint32_t pass = epoch[0] + 1u;   // this pass's number
    const uint32_t par = pass & 1u;
    prefetch_all_l2(fanin, (nn - ns) * (int64_t)sizeof(uint4));
    load_bounds(slvl, lvl, L);
    for (int64_t k = t; k < ns; k += blockDim.x) {
        const pair_ff a = pair_of(sp_in[k]);
        const float4 v = pair_store(a, par);
        pq[k] = v;
        spq[k] = v;
        tr[k] = tr_mode ? pair_tr(a) : tr_in[k];
    }
    __syncthreads();
    uint4 r = make_uint4(0, 0, 0, 0);
    if (L > 0 && slvl[0] + t < slvl[1]) r = fanin[slvl[0] + t];
    for (int l = 1; l <= L; l++) {
        const int64_t c = slvl[l - 1] + t;
        const bool on = c < slvl[l];
        uint4 rn = make_uint4(0, 0, 0, 0);
        if (l < L && slvl[l] + t < slvl[l + 1]) rn = fanin[slvl[l] + t];   // the next level's record
        if (l > 1) __syncthreads();   // the levels below are in shared memory
        if (on) {
            const uint32_t op = r.x >> 24;
            const int k = op_arity(ops, op);
            pair_ff x[4];
            gather_ff<false>(spq, r, k, x);
            const pair_ff o = cell_pair(k, op_tt(ops, op), x);
            const float4 v = pair_store(o, par);
            spq[ns + c] = v;
            pq[ns + c] = v;
            tr[ns + c] = pair_tr(o);
        }
        r = rn;
    }
    if (t == 0) epoch[0] = pass;   // every thread read the old value before the level barriers
}

// the raw static data of one cell for the reverse pass
struct BwdRaw {
    uint4 r;
    int4 ep;
    int32_t e0, e1;
    float cl, b;
};

__device__ __forceinline__ BwdRaw bwd_raw(const uint4 *fanin, const int32_t *fptr, const int4 *efpos,
                                          const float *cload, const float *beta, int64_t c, int64_t ns,
                                          int grad_mode) {
    BwdRaw w;
    const int64_t n = ns + c;
    w.r = fanin[c];
    w.ep = efpos[c];
    w.e0 = fptr[n];
    w.e1 = fptr[n + 1];
    w.cl = cload[n];
    w.b = grad_mode ? beta[n] : 1.f;
    return w;
}

__global__ void __launch_bounds__(kBlockThreads) k_bwd_block(
    const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr, const int4 *__restrict__ efpos,
    const float4 *__restrict__ pq, const float *__restrict__ cload, const float *__restrict__ beta, float *gnet,
    const int32_t *__restrict__ lvl, int L, int64_t ns, int64_t nn, int64_t ne, int grad_mode, int tr_mode,
    float K, float *out_gsp, OpTable ops) {
    extern __shared__ float4 spq[];
    float *sgfo = reinterpret_cast<float *>(spq + nn);
    int *slvl = reinterpret_cast<int *>(sgfo + ne);
    const int t = threadIdx.x;
    const int64_t nc = nn - ns;
    prefetch_all_l2(fanin, nc * (int64_t)sizeof(uint4));
    prefetch_all_l2(efpos, nc * (int64_t)sizeof(int4));
    prefetch_all_l2(fptr, (nn + 1) * (int64_t)sizeof(int32_t));
    prefetch_all_l2(cload, nn * (int64_t)sizeof(float));
    if (grad_mode) prefetch_all_l2(beta, nn * (int64_t)sizeof(float));
    load_bounds(slvl, lvl, L);
#pragma unroll 8
    for (int64_t k = t; k < nn; k += blockDim.x) spq[k] = pq[k];
    BwdRaw w{};
    if (L > 0 && lvl[L - 1] + t < lvl[L]) w = bwd_raw(fanin, fptr, efpos, cload, beta, lvl[L - 1] + t, ns, grad_mode);
    __syncthreads();
    for (int l = L; l >= 1; l--) {
        const int64_t c = slvl[l - 1] + t;
        const bool on = c < slvl[l];
        // the cell's static part (as in the grid-wide pass), from the pairs in shared memory
        float local = 0.f, d[4] = {0.f, 0.f, 0.f, 0.f};
        int k = 0;
        if (on) {
            local = adj_local(K, w.cl, pair_qmp(spq[ns + c]));
            const uint32_t op = w.r.x >> 24;
            k = op_arity(ops, op);
            float p[4], q[4];
            gather_pairs(spq, w.r, k, p, q);
            cell_partials(k, op_tt(ops, op), p, q, d);
        }
        const BwdRaw cur = w;
        if (l > 1 && slvl[l - 2] + t < slvl[l - 1])   // the next level's raw data
            w = bwd_raw(fanin, fptr, efpos, cload, beta, slvl[l - 2] + t, ns, grad_mode);
        if (l < L) __syncthreads();   // the levels above have written their edge adjoints
        if (on) {
            float acc = 0.f;
            for (int32_t e = cur.e0; e < cur.e1; e++) acc += sgfo[e];
            const float g = combine(grad_mode, acc, local, cur.b);
            gnet[ns + c] = g;
            if (k > 0) sgfo[cur.ep.x] = g * d[0];
            if (k > 1) sgfo[cur.ep.y] = g * d[1];
            if (k > 2) sgfo[cur.ep.z] = g * d[2];
            if (k > 3) sgfo[cur.ep.w] = g * d[3];
        }
    }
    __syncthreads();
    for (int64_t k = t; k < ns; k += blockDim.x) {
        float acc = 0.f;
        for (int32_t e = fptr[k]; e < fptr[k + 1]; e++) acc += sgfo[e];
        const float local = tr_mode ? adj_local(K, cload[k], pair_qmp(spq[k])) : 0.f;
        const float g = combine(grad_mode, acc, local, grad_mode ? beta[k] : 1.f);
        gnet[k] = g;
        if (out_gsp) out_gsp[k] = g;
    }
}

// ------------------------------------------------------------- simulation
// One warp per cell.  Chunks of 64 words: lane l evaluates words 2l and
// 2l + 1 (one 16-byte load per fanin when T is even, two 8-byte loads
// otherwise), counts ones, and counts toggles against the previous word
// (its own first word, or the last word of the neighbour lane / chunk).
__device__ __forceinline__ void sim_cell(const uint4 &r, int64_t c, uint64_t *words, uint32_t *toggles,
                                         uint32_t *ones, int64_t ns, int T, const OpTable &ops, int lane) {
    const uint32_t op = r.x >> 24;
    const int k = op_arity(ops, op);
    const uint32_t tt = op_tt(ops, op);
    const uint64_t *in[4] = {words, words, words, words};
    if (k > 0) in[0] = words + (size_t)(r.x & kMask24) * T;
    if (k > 1) in[1] = words + (size_t)r.y * T;
    if (k > 2) in[2] = words + (size_t)r.z * T;
    if (k > 3) in[3] = words + (size_t)r.w * T;
    uint64_t *out = words + (size_t)(ns + c) * T;
    const bool even = (T & 1) == 0;
    uint32_t tg = 0, on = 0;
    uint64_t carry = 0;
    for (int base = 0; base < T; base += 64) {
        const int t0 = base + 2 * lane, t1 = t0 + 1;
        uint64_t x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0};
        if (even && t1 < T) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (j < k) {
                    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(in[j] + t0));
                    x0[j] = v.x;
                    x1[j] = v.y;
                }
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (j < k) {
                    if (t0 < T) x0[j] = __ldcg(in[j] + t0);
                    if (t1 < T) x1[j] = __ldcg(in[j] + t1);
                }
        }
        uint64_t w0, w1;
        cell_bits2(k, tt, op_lut(ops, op), x0, x1, w0, w1);
        uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, w1, 1);
        if (lane == 0) prev = carry;
        if (even && t1 < T) {
            *reinterpret_cast<ulonglong2 *>(out + t0) = make_ulonglong2(w0, w1);
        } else {
            if (t0 < T) out[t0] = w0;
            if (t1 < T) out[t1] = w1;
        }
        if (t0 < T) {
            on += __popcll(w0);
            if (t0 > 0) tg += __popcll(w0 ^ prev);
        }
        if (t1 < T) {
            on += __popcll(w1);
            tg += __popcll(w1 ^ w0);
        }
        carry = __shfl_sync(0xFFFFFFFFu, w1, 31);
    }
    tg = __reduce_add_sync(0xFFFFFFFFu, tg);
    on = __reduce_add_sync(0xFFFFFFFFu, on);
    if (lane == 0) {
        toggles[ns + c] = tg;
        ones[ns + c] = on;
    }
}

__global__ void __launch_bounds__(kSimThreads) k_sim_persist(const uint4 *__restrict__ fanin, uint64_t *words,
                                                             uint32_t *toggles, uint32_t *ones,
                                                             const int32_t *__restrict__ lvl, int L, int64_t ns,
                                                             int T, OpTable ops, unsigned *bar, int *err,
                                                             long long limit) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = spread_warp();
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int l = 1; l <= L; l++) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        const int64_t c = c0 + gw;
        // level 1 reads only startpoint words, written by the previous launch
        if (l > 1) barrier_arrive(bar + 32 * (l - 2));
        uint4 r = make_uint4(0, 0, 0, 0);
        if (c < c1) r = fanin[c];
        if (l > 1 && !barrier_wait(bar + 32 * (l - 2), err, gridDim.x, limit)) return;
        if (c < c1) sim_cell(r, c, words, toggles, ones, ns, T, ops, lane);
        for (int64_t cc = c + W; cc < c1; cc += W) sim_cell(fanin[cc], cc, words, toggles, ones, ns, T, ops, lane);
    }
}

// ------------------------------------------------ simulation, wide lanes
// Same computation as k_sim_persist for T divisible by 4: 16 lanes per cell,
// lane h of a half-warp owns words 4h .. 4h+3 of each 64-word chunk, so a
// warp evaluates two consecutive cells (usually the same logic id, since
// cells are sorted by it inside a level).  Every lane issues its two 16-byte
// loads per fanin before using any of them, which keeps several kilobytes in
// flight per warp; toggle and ones counts are reduced over the half-warp.
// The words are scratch of the pass: once the last level that reads a net is
// complete, its words are dead, and when T is a multiple of 16 (whole 128-byte
// lines per net) they are dropped from L2 without a write-back
// (discard.global.L2).  A net dies at its death level (the highest level of
// the cells it feeds, else its own); the nets of death level d, listed in
// dead_net[dead_ptr[d] .. dead_ptr[d+1]), are discarded by the whole grid during
// level d + 2, between a block's arrival and its wait (every block passed the
// barrier that ended level d before it worked on level d + 1).  Without it the
// pass writes every cell's words back to DRAM as L2 fills with them.
__device__ __forceinline__ void discard_l2(const void *p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

__global__ void __launch_bounds__(kSimThreads, 2) k_sim_wide(const uint4 *__restrict__ fanin, uint64_t *words,
                                                            uint32_t *toggles, uint32_t *ones,
                                                            const int32_t *__restrict__ lvl, int L, int64_t ns,
                                                            int T, OpTable ops, const int32_t *__restrict__ dead_ptr,
                                                            const int32_t *__restrict__ dead_net, unsigned *bar,
                                                            int *err, long long limit) {
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t gw = spread_warp();
    const int64_t step = 2 * (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lines = (T & 15) == 0 && dead_ptr ? T / 16 : 0;   // 128-byte lines per net
    for (int l = 1; l <= L; l++) {
        const int32_t c0 = lvl[l - 1], c1 = lvl[l];
        const int64_t cfirst = c0 + 2 * gw + half;
        if (l > 1) barrier_arrive(bar + 32 * (l - 2));
        uint4 r = make_uint4(0, 0, 0, 0);
        if (cfirst < c1) r = fanin[cfirst];   // static: loaded between arrival and wait
        if (lines && l >= 2) {
            const int64_t d0 = dead_ptr[l - 2], nd = (int64_t)(dead_ptr[l - 1] - d0) * lines;
            for (int64_t i = spread_tid(); i < nd; i += (int64_t)gridDim.x * blockDim.x)
                discard_l2(words + (size_t)dead_net[d0 + i / lines] * T + (size_t)(i % lines) * 16);
        }
        if (l > 1 && !barrier_wait(bar + 32 * (l - 2), err, gridDim.x, limit)) return;
        for (int64_t c = cfirst;; c += step) {
            const bool valid = c < c1;
            if (!__any_sync(0xFFFFFFFFu, valid)) break;
            if (c != cfirst) r = valid ? fanin[c] : make_uint4(0, 0, 0, 0);
            const uint32_t op = r.x >> 24;
            const int k = valid ? op_arity(ops, op) : 0;
            const uint32_t tt = op_tt(ops, op), lut = op_lut(ops, op);
            const uint32_t nid[4] = {r.x & kMask24, r.y, r.z, r.w};
            uint64_t *out = words + (size_t)(ns + (valid ? c : 0)) * T;
            uint32_t tg = 0, on = 0;
            uint64_t carry = 0;
            for (int base = 0; base < T; base += 64) {
                const int t = base + 4 * hl;
                const bool act = valid && t < T;
                uint64_t w[4];
                if (k <= 3) {
                    uint64_t x[3][4];
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        x[j][0] = x[j][1] = x[j][2] = x[j][3] = 0;
                        if (act && j < k) {
                            const uint64_t *src = words + (size_t)nid[j] * T + t;
                            const ulonglong2 a = __ldcg(reinterpret_cast<const ulonglong2 *>(src));
                            const ulonglong2 b = __ldcg(reinterpret_cast<const ulonglong2 *>(src + 2));
                            x[j][0] = a.x;
                            x[j][1] = a.y;
                            x[j][2] = b.x;
                            x[j][3] = b.y;
                        }
                    }
                    const uint64_t a0[4] = {x[0][0], x[1][0], x[2][0], 0}, a1[4] = {x[0][1], x[1][1], x[2][1], 0};
                    const uint64_t b0[4] = {x[0][2], x[1][2], x[2][2], 0}, b1[4] = {x[0][3], x[1][3], x[2][3], 0};
                    cell_bits_lop3(lut, a0, a1, w[0], w[1]);
                    cell_bits_lop3(lut, b0, b1, w[2], w[3]);
                } else {
                    // 4-input cells: the two cofactors in x3 by LOP3 (tables tt & 0xFF and
                    // tt >> 8 over x2, x1, x0), then a select by x3.  No leaf words: the
                    // multiplexer tree's 16 leaves made the kernel spill at its 64 registers
#pragma unroll
                    for (int h2 = 0; h2 < 2; h2++) {
                        uint64_t x0[4] = {0, 0, 0, 0}, x1[4] = {0, 0, 0, 0};
                        if (act)
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                const ulonglong2 a = __ldcg(
                                    reinterpret_cast<const ulonglong2 *>(words + (size_t)nid[j] * T + t + 2 * h2));
                                x0[j] = a.x;
                                x1[j] = a.y;
                            }
                        uint64_t f00, f01, f10, f11;
                        cell_bits_lop3(tt & 0xFFu, x0, x1, f00, f01);
                        cell_bits_lop3((tt >> 8) & 0xFFu, x0, x1, f10, f11);
                        w[2 * h2] = (x0[3] & f10) | (~x0[3] & f00);
                        w[2 * h2 + 1] = (x1[3] & f11) | (~x1[3] & f01);
                    }
                }
                const uint64_t prev = __shfl_up_sync(0xFFFFFFFFu, w[3], 1, 16);
                const uint64_t last = __shfl_sync(0xFFFFFFFFu, w[3], 15, 16);
                if (act) {
                    *reinterpret_cast<ulonglong2 *>(out + t) = make_ulonglong2(w[0], w[1]);
                    *reinterpret_cast<ulonglong2 *>(out + t + 2) = make_ulonglong2(w[2], w[3]);
                    on += __popcll(w[0]) + __popcll(w[1]) + __popcll(w[2]) + __popcll(w[3]);
                    tg += __popcll(w[1] ^ w[0]) + __popcll(w[2] ^ w[1]) + __popcll(w[3] ^ w[2]);
                    if (t > 0) tg += __popcll(w[0] ^ (hl > 0 ? prev : carry));
                }
                carry = last;
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                tg += __shfl_xor_sync(0xFFFFFFFFu, tg, o);
                on += __shfl_xor_sync(0xFFFFFFFFu, on, o);
            }
            if (valid && hl == 0) {
                toggles[ns + c] = tg;
                ones[ns + c] = on;
            }
        }
    }
}

// ---------------------------------------------------------- latency probes
// The level-synchronous skeleton of the persistent passes without their
// arithmetic: `levels` levels, each ended by the same level barrier.
// gather = 0: the barriers alone.  gather = 1: after each barrier every thread
// loads, through L2, three values that threads of three other blocks stored in
// the previous level, and stores one value: the barrier plus one dependent L2
// round trip and a store per level, the least a level of the forward pass does.
__global__ void k_probe_levels(float *buf, int levels, int gather, unsigned *bar, int *err, long long limit) {
    const int64_t N = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockDim.x, g = gridDim.x;
    const int64_t s0 = (t + b * (g / 4 + 1)) % N, s1 = (t + b * (g / 2 + 1)) % N, s2 = (t + b * (3 * g / 4 + 1)) % N;
    for (int l = 0; l < levels; l++) {
        const float *prev = buf + (l & 1) * N;
        float *cur = buf + ((l + 1) & 1) * N;
        if (gather) cur[t] = (__ldcg(prev + s0) + __ldcg(prev + s1) + __ldcg(prev + s2)) * (1.f / 3.f);
        if (!level_barrier(bar + 32 * l, err, gridDim.x, limit)) return;
    }
}

// one thread follows a chain of dependent loads through L2 (ld.global.cg):
// the latency of one dependent L2 access
__global__ void k_probe_chase(const uint32_t *next, int hops, uint32_t *sink) {
    uint32_t i = 0;
    for (int h = 0; h < hops; h++) i = __ldcg(next + i);
    *sink = i;
}

// self-test of the bounded wait: the barrier expects one arrival more than
// the grid has blocks, so it can only end by giving up
__global__ void k_wait_selftest(unsigned *bar, int *err, long long limit) {
    level_barrier(bar, err, gridDim.x + 1, limit);
}

template <class... Args>
cudaError_t launch_coop(void (*kern)(Args...), int grid, int block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

size_t bar_bytes(const DevDesign &d) { return sizeof(unsigned) * 32 * ((size_t)d.n_levels + 2); }

}  // namespace

int wide_grid(int sm_count) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sim_wide, kSimThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sm_count * (per < 2 ? per : 2);
}

int persist_grid(int which, int sm_count) {
    int per = 0;
    cudaError_t e;
    if (which == 3) return wide_grid(sm_count);
    if (which == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_persist, kFwdThreads, 0);
    else if (which == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sim_persist, kSimThreads, 0);
    else {   // both forms of the reverse pass run on the same grid: the smaller occupancy
        int per2 = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bwd_persist<true>, kPersistThreads, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_bwd_persist<false>, kPersistThreads, 0);
        per = per < per2 ? per : per2;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int cap = which == 1 ? 2 : 1;   // blocks per SM used: enough warps, few barrier arrivals
    return sm_count * (per < cap ? per : cap);
}

size_t persist_bar_words(int n_levels) { return 3 * 32 * ((size_t)n_levels + 2); }

cudaError_t launch_fwd_persist(const DevDesign &d, const OpTable &ops, int tr_mode, int grid, cudaStream_t s,
                               cudaEvent_t ready) {
    unsigned *bar = d.bar;
    cudaMemsetAsync(bar, 0, bar_bytes(d), s);
    if (ready) cudaEventRecord(ready, s);   // work forked here becomes ready together with the kernel
    return launch_coop(k_fwd_persist, grid, kFwdThreads, s, d.fanin, d.pq, d.tr, (const float *)d.sp_in,
                       (const float *)d.tr_in, d.lvl, d.n_levels, d.n_start, tr_mode, ops, bar, d.err,
                       kWaitLimitCycles, (const uint32_t *)d.epoch);
}

cudaError_t launch_sim_persist(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s) {
    unsigned *bar = d.bar + 32 * ((size_t)d.n_levels + 2);
    cudaMemsetAsync(bar, 0, bar_bytes(d), s);
    return launch_coop(k_sim_persist, grid, kSimThreads, s, d.fanin, d.words, d.toggles, d.ones, d.lvl, d.n_levels,
                       d.n_start, T, ops, bar, d.err, kWaitLimitCycles);
}

bool wide_ok(int T) { return T >= 4 && (T & 3) == 0; }

cudaError_t launch_sim_wide(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s) {
    unsigned *bar = d.bar + 32 * ((size_t)d.n_levels + 2);
    cudaMemsetAsync(bar, 0, bar_bytes(d), s);
    return launch_coop(k_sim_wide, grid, kSimThreads, s, d.fanin, d.words, d.toggles, d.ones, d.lvl, d.n_levels,
                       d.n_start, T, ops, d.dead_ptr, d.dead_net, bar, d.err, kWaitLimitCycles);
}

cudaError_t launch_bwd_persist(const DevDesign &d, const OpTable &ops, int grad_mode, int tr_mode, float K,
                               float *out_gsp, int grid, bool pre, cudaStream_t s) {
    unsigned *bar = d.bar + 2 * 32 * ((size_t)d.n_levels + 2);
    cudaMemsetAsync(bar, 0, bar_bytes(d), s);
    return launch_coop(pre ? k_bwd_persist<true> : k_bwd_persist<false>, grid, kPersistThreads, s, d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos,
                       (const float4 *)d.pq, (const float *)d.cload, (const float *)d.beta, d.gnet, d.gfo, d.lvl,
                       d.n_levels, d.n_start, grad_mode, tr_mode, K, out_gsp, ops, bar, d.err, kWaitLimitCycles);
}

size_t block_smem(int which, int64_t n_nets, int64_t n_edges, int n_levels) {
    return (size_t)n_nets * sizeof(float4) + (which ? (size_t)n_edges * sizeof(float) : 0) +
           (size_t)(n_levels + 1) * sizeof(int);
}

bool block_smem_init() {
    return cudaFuncSetAttribute(k_fwd_block, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockSmemMax) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_bwd_block, cudaFuncAttributeMaxDynamicSharedMemorySize, kBlockSmemMax) ==
               cudaSuccess;
}

cudaError_t launch_fwd_block(const DevDesign &d, const OpTable &ops, int tr_mode, int threads, cudaStream_t s) {
    const size_t smem = block_smem(0, d.n_nets, 0, d.n_levels);
    k_fwd_block<<<1, threads, smem, s>>>(d.fanin, d.pq, d.tr, d.sp_in, d.tr_in, d.lvl, d.n_levels, d.n_start,
                                         d.n_nets, tr_mode, ops, d.epoch);
    return cudaGetLastError();
}

cudaError_t launch_bwd_block(const DevDesign &d, const OpTable &ops, int grad_mode, int tr_mode, float K,
                             float *out_gsp, int64_t n_edges, int threads, cudaStream_t s) {
    const size_t smem = block_smem(1, d.n_nets, n_edges, d.n_levels);
    k_bwd_block<<<1, threads, smem, s>>>(d.fanin, d.fout_ptr, (const int4 *)d.edge_fpos, (const float4 *)d.pq,
                                         d.cload, d.beta, d.gnet, d.lvl, d.n_levels, d.n_start, d.n_nets, n_edges,
                                         grad_mode, tr_mode, K, out_gsp, ops);
    return cudaGetLastError();
}

cudaError_t launch_probe_levels(float *buf, int levels, int gather, int grid, int threads, unsigned *bar, int *err,
                                cudaStream_t s) {
    return launch_coop(k_probe_levels, grid, threads, s, buf, levels, gather, bar, err, kWaitLimitCycles);
}

cudaError_t launch_probe_chase(const uint32_t *next, int hops, uint32_t *sink, cudaStream_t s) {
    k_probe_chase<<<1, 1, 0, s>>>(next, hops, sink);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(unsigned *bar, int *err, long long limit, cudaStream_t s) {
    cudaMemsetAsync(bar, 0, 128, s);
    return launch_coop(k_wait_selftest, 2, 32, s, bar, err, limit);
}

}  // namespace dp
