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

}  // namespace

void launch_bump(uint32_t *counter, cudaStream_t s) { k_bump<<<1, 1, 0, s>>>(counter); }

int flow_grid(int which, int sm_count, int blocks_per_sm) {
    (void)which;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fwd_flow, kFlowThreads, 0) != cudaSuccess) {
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

}  // namespace dp
