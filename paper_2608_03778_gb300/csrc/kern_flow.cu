// Dataflow schedule: no barriers between levels.  Cells are split into
// level-aligned chunks of 32 (one cell per lane); warp w of the cooperative
// grid takes chunks w, w + W, w + 2W, ... in increasing order, and each lane
// waits only for the fanins of its own cell, recognising a finished fanin by
// the parity tag its forward pass stored with the value (the data is its own
// ready flag).  A chunk depends only on chunks of lower levels, which come
// earlier in the order, and all warps are co-resident, so the chunk with the
// smallest index that is not finished can always proceed: no deadlock.
// Every wait is bounded by a clock limit; a lane that gives up records the
// context's error word, and the others stop at their next wait.
#include "kern_common.cuh"

namespace dp {
namespace {

constexpr int kFlowThreads = 256;

__global__ void k_bump(uint32_t *counter) { *counter += 1u; }

__device__ __forceinline__ int ld_err(const int *err) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(err) : "memory");
    return v;
}

// Reads a stored pair as two single-copy-atomic 8-byte halves, through L2.
__device__ __forceinline__ void ld_pair_halves(const float4 *src, unsigned long long &h0, unsigned long long &h1) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(h0), "=l"(h1) : "l"(src) : "memory");
}

// Waits until the pair at src carries this pass's parity in both halves;
// false when the wait gave up (clock limit, or another lane's error).
__device__ __forceinline__ bool wait_pair(const float4 *src, uint32_t par, const int *err, long long limit,
                                          unsigned sleep_max, pair_ff &out) {
    unsigned long long h0, h1;
    ld_pair_halves(src, h0, h1);
    const uint32_t want = par << 31;
    if (((uint32_t)h0 & 0x80000000u) != want || ((uint32_t)h1 & 0x80000000u) != want) {
        const long long t0 = clock64();
        unsigned ns = 16;
        for (;;) {
            if (sleep_max) {
                __nanosleep(ns);
                if (ns < sleep_max) ns <<= 1;
            }
            ld_pair_halves(src, h0, h1);
            if (((uint32_t)h0 & 0x80000000u) == want && ((uint32_t)h1 & 0x80000000u) == want) break;
            if (clock64() - t0 > limit || ld_err(err) != 0) return false;
        }
    }
    out.p = ff{__uint_as_float((uint32_t)h0 & 0x7FFFFFFFu), __uint_as_float((uint32_t)(h0 >> 32))};
    out.q = ff{__uint_as_float((uint32_t)h1 & 0x7FFFFFFFu), __uint_as_float((uint32_t)(h1 >> 32))};
    return true;
}

__global__ void __launch_bounds__(kFlowThreads) k_fwd_flow(const uint4 *__restrict__ fanin, float4 *pq, float *tr,
                                                           const float *__restrict__ sp_in,
                                                           const float *__restrict__ tr_in,
                                                           const int32_t *__restrict__ lvl,
                                                           const int32_t *__restrict__ chunk_ptr, int L, int64_t ns,
                                                           int tr_mode, OpTable ops, const uint32_t *epoch, int *err,
                                                           long long limit, unsigned sleep_max) {
    const uint32_t par = epoch[0] & 1u;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nchunks = chunk_ptr[L + 1];
    int lv = 0;
    for (int64_t j = gw; j < nchunks; j += W) {
        while (j >= chunk_ptr[lv + 1]) lv++;
        if (lv == 0) {
            const int64_t k = j * 32 + lane;
            if (k < ns) {
                const pair_ff a = pair_of(sp_in[k]);
                tr[k] = tr_mode ? pair_tr(a) : tr_in[k];
                pair_put(pq + k, a, par);
            }
            continue;
        }
        const int64_t c = lvl[lv - 1] + (j - chunk_ptr[lv]) * 32 + lane;
        if (c >= lvl[lv]) continue;
        const uint4 r = fanin[c];
        const uint32_t op = r.x >> 24;
        const int k = op_arity(ops, op);
        const uint32_t n[4] = {r.x & kMask24, r.y, r.z, r.w};
        pair_ff x[4];
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            x[q] = pair_ff{ff_make(0.f), ff_make(1.f)};
            if (q < k && ok) ok = wait_pair(pq + n[q], par, err, limit, sleep_max, x[q]);
        }
        if (!ok) {
            atomicExch(err, 1);
            return;
        }
        const pair_ff o = cell_pair(k, op_tt(ops, op), x);
        tr[ns + c] = pair_tr(o);
        pair_put(pq + ns + c, o, par);
    }
}

// ------------------------------------------------------ simulation, dataflow
// The wide simulation (16 lanes per cell, two cells of one level per warp)
// without level barriers.  Cells are grouped in level-aligned pairs; warp w
// takes pairs w, w + W, w + 2W, ... in increasing order, and lane h < k of a
// half-warp waits only for the flag of fanin h when that fanin is a cell.  A
// cell publishes its words by storing the pass number into its flag with
// release semantics after a warp barrier that orders the sixteen lanes'
// stores; the waiting lane reads the flag with acquire semantics and a warp
// barrier orders that before the other lanes' word loads.  Flags need no
// clearing: each pass has its own number.  A pair depends only on pairs of
// lower levels, which come earlier in the order, so (all warps co-resident)
// the lowest unfinished pair can always proceed.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// true once the flag holds this pass's number; false when the wait gave up
__device__ __forceinline__ bool wait_done(const unsigned *f, unsigned ep, const int *err, long long limit) {
    if (ld_acquire_u32(f) == ep) return true;
    const long long t0 = clock64();
    for (;;) {
        __nanosleep(32);
        if (ld_acquire_u32(f) == ep) return true;
        if (clock64() - t0 > limit || ld_err(err) != 0) return false;
    }
}

// cell index of pair p (from level lv on, updated) and half h; -1 past the end
__device__ __forceinline__ int64_t pair_cell(int64_t p, int &lv, int L, const int32_t *lvl, const int32_t *pair_ptr,
                                             int h) {
    while (lv <= L && p >= pair_ptr[lv]) lv++;
    if (lv > L) return -1;
    const int64_t c = lvl[lv - 1] + 2 * (p - pair_ptr[lv - 1]) + h;
    return c < lvl[lv] ? c : -1;
}

__global__ void __launch_bounds__(kSimThreads, 2) k_sim_flow(const uint4 *__restrict__ fanin, uint64_t *words,
                                                            uint32_t *toggles, uint32_t *ones, unsigned *done,
                                                            const int32_t *__restrict__ lvl,
                                                            const int32_t *__restrict__ pair_ptr, int L, int64_t ns,
                                                            int T, OpTable ops, const uint32_t *epoch, int *err,
                                                            long long limit) {
    const unsigned ep = epoch[1];
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t npairs = pair_ptr[L];
    int lv = 1, lvn = 1;
    int64_t p = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    int64_t cn = p < npairs ? pair_cell(p, lvn, L, lvl, pair_ptr, half) : -1;
    uint4 rn = cn >= 0 ? fanin[cn] : make_uint4(0, 0, 0, 0);
    for (; p < npairs; p += W) {   // warp-uniform
        const int64_t c = cn;
        const uint4 r = rn;
        lv = lvn;
        // the next pair's record, ahead of its use
        cn = p + W < npairs ? pair_cell(p + W, lvn, L, lvl, pair_ptr, half) : -1;
        rn = cn >= 0 ? fanin[cn] : make_uint4(0, 0, 0, 0);
        const bool valid = c >= 0;
        const uint32_t op = r.x >> 24;
        const int k = valid ? op_arity(ops, op) : 0;
        const uint32_t tt = op_tt(ops, op), lut = op_lut(ops, op);
        const uint32_t nid[4] = {r.x & kMask24, r.y, r.z, r.w};
        bool ok = true;
        if (hl < k) {
            const uint32_t n = hl == 0 ? nid[0] : hl == 1 ? nid[1] : hl == 2 ? nid[2] : nid[3];
            if (n >= ns) ok = wait_done(done + (n - ns), ep, err, limit);
        }
        if (!__all_sync(0xFFFFFFFFu, ok)) {
            if (!ok) atomicExch(err, 1);
            return;
        }
        __syncwarp();   // the flags' acquire before every lane's word loads
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
                    w[2 * h2] = bits_eval<4>(tt, x0);
                    w[2 * h2 + 1] = bits_eval<4>(tt, x1);
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
        __syncwarp();   // every lane's word stores before the flag's release
        if (valid && hl == 0) {
            toggles[ns + c] = tg;
            ones[ns + c] = on;
            st_release_u32(done + c, ep);
        }
    }
}

}  // namespace

void launch_bump(uint32_t *counter, cudaStream_t s) { k_bump<<<1, 1, 0, s>>>(counter); }

int flow_grid(int which, int sm_count, int blocks_per_sm) {
    int per = 0;
    const cudaError_t e = which == 1
                              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sim_flow, kSimThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_flow, kFlowThreads, 0);
    if (which == 1) blocks_per_sm = 2;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sm_count * (per < blocks_per_sm ? per : blocks_per_sm);
}

cudaError_t launch_fwd_flow(const DevDesign &d, const OpTable &ops, int tr_mode, int grid, unsigned sleep_max,
                            cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kFlowThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all warps co-resident: needed for progress
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fwd_flow, d.fanin, d.pq, d.tr, (const float *)d.sp_in, (const float *)d.tr_in,
                              d.lvl, d.chunk_ptr, d.n_levels, d.n_start, tr_mode, ops, (const uint32_t *)d.epoch,
                              d.err, kWaitLimitCycles, sleep_max);
}

cudaError_t launch_sim_flow(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s) {
    launch_bump(d.epoch + 1, s);   // a new pass number for the flags
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)kSimThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sim_flow, d.fanin, d.words, d.toggles, d.ones, d.simdone, d.lvl, d.pair_ptr,
                              d.n_levels, d.n_start, T, ops, (const uint32_t *)d.epoch, d.err, kWaitLimitCycles);
}

}  // namespace dp
