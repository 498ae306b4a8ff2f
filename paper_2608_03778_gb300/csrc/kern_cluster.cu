// Forward and reverse passes of a mid-size design in one thread-block cluster.
//
// A design too large for one block's shared memory but whose per-block share fits (up to
// about 130,000 nets on a 16-block cluster) runs each pass on one cluster of kClusterBlocks
// blocks.  Every level (the startpoints are level 0) is cut into C contiguous chunks, block b
// taking chunk b: consecutive cells of a level share their function (levels are sorted by logic
// id), so a warp's cells mostly take the same branch.  A net lives in the shared memory of the
// block that computes it, at a slot that the host assigns level by level (loc = block << 24 |
// slot): its (P, Q) pair, and in the reverse pass the edge adjoints of its fanout range.  A
// block reads its cells' fanin pairs from their owners' shared memory (distributed shared
// memory) and, in the reverse pass, writes the edge adjoints into the owners of the fanin
// nets.  The level barrier is the hardware cluster barrier (about 450 cycles on GB300, against
// 1.3 us for a grid-wide barrier through L2), split into arrive (release) and wait (acquire)
// so that the static data of later levels is loaded in between.  Every thread of every block
// runs the same arrive/wait sequence, with no early exit, and a block leaves only after the
// last wait: no block then reads or writes another's shared memory.
//
// Each value is computed by the same code in the same order as in the grid-wide passes (a
// net's fanout range keeps its order in its owner's copy), so the results are bitwise the same.
#include <cooperative_groups.h>

#include "kern_common.cuh"

namespace cg = cooperative_groups;

namespace dp {
namespace {

constexpr uint32_t kSlotMask = 0xFFFFFFu;

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// block r of C prefetches its share of the 128-byte lines of bytes [p, p + n) into L2
__device__ __forceinline__ void prefetch_share_l2(const void *p, int64_t n, int r, int C) {
    const char *c = static_cast<const char *>(p);
    for (int64_t i = ((int64_t)r * blockDim.x + threadIdx.x) * 128; i < n; i += (int64_t)C * blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + i));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// the block's tables in shared memory: level bounds (cells), chunk length per level, and the
// first slot of the block's chunk of each level
struct Tables {
    int *lvl, *chunk, *base;
};
__device__ __forceinline__ void load_tables(const Tables &s, const int32_t *lvl, const int32_t *chunk,
                                            const int32_t *base, int L, int r) {
    for (int i = threadIdx.x; i <= L; i += blockDim.x) {
        s.lvl[i] = lvl[i];
        s.chunk[i] = chunk[i];
        s.base[i] = base[(int64_t)r * (L + 1) + i];
    }
}

// a pair from its owner's shared memory
__device__ __forceinline__ float4 dsm_pair(const cg::cluster_group &cl, float4 *spq, uint32_t loc) {
    return *(cl.map_shared_rank(spq, loc >> 24) + (loc & kSlotMask));
}

// this thread's cell on level l >= 1 (if any): its internal cell index and own slot
__device__ __forceinline__ bool cell_at(const Tables &s, int l, int L, int r, int t, int64_t &c, int &slot) {
    if (l < 1 || l > L) return false;
    const int chunk = s.chunk[l];
    c = s.lvl[l - 1] + (int64_t)r * chunk + t;
    slot = s.base[l] + t;
    return t < chunk && c < s.lvl[l];
}

// Shared memory: the block's slots of (P, Q) pairs, then its tables.
__global__ void __launch_bounds__(kClusterMaxThreads) k_fwd_cluster(
    const uint4 *__restrict__ fanin, const uint4 *__restrict__ floc, float4 *pq, float *tr,
    const float *__restrict__ sp_in, const float *__restrict__ tr_in, const int32_t *__restrict__ lvl,
    const int32_t *__restrict__ chunk, const int32_t *__restrict__ base, int L, int64_t ns, int64_t nn,
    int64_t slots, int tr_mode, OpTable ops, const uint32_t *epoch) {
    extern __shared__ float4 spq[];
    const cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rk = (int)cl.block_rank();
    int *tab = reinterpret_cast<int *>(spq + slots);
    const Tables s{tab, tab + (L + 1), tab + 2 * (L + 1)};
    const int t = threadIdx.x, B = blockDim.x;
    const uint32_t par = epoch[0] & 1u;
    prefetch_share_l2(fanin, (nn - ns) * (int64_t)sizeof(uint4), rk, C);
    prefetch_share_l2(floc, (nn - ns) * (int64_t)sizeof(uint4), rk, C);
    load_tables(s, lvl, chunk, base, L, rk);
    __syncthreads();
    for (int p = t; p < s.chunk[0]; p += B) {   // the block's startpoints
        const int64_t n = (int64_t)rk * s.chunk[0] + p;
        if (n >= ns) break;
        const pair_ff a = pair_of(sp_in[n]);
        const float4 v = pair_store(a, par);
        spq[s.base[0] + p] = v;
        pq[n] = v;
        tr[n] = tr_mode ? pair_tr(a) : tr_in[n];
    }
    // this thread's cells, two levels ahead: record and fanin locations
    int64_t c = 0, c1 = 0;
    int slot = 0, slot1 = 0;
    uint4 r = make_uint4(0, 0, 0, 0), f = r, r1 = r, f1 = r;
    bool on = cell_at(s, 1, L, rk, t, c, slot), on1 = cell_at(s, 2, L, rk, t, c1, slot1);
    if (on) r = fanin[c], f = floc[c];
    if (on1) r1 = fanin[c1], f1 = floc[c1];
    cluster_arrive();
    for (int l = 1; l <= L; l++) {
        cluster_wait();   // the levels below are in every block's shared memory
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        float y = 0.f;
        if (on) {
            const uint32_t op = r.x >> 24;
            const int k = op_arity(ops, op);
            const uint32_t fl[4] = {f.x, f.y, f.z, f.w};
            pair_ff x[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                x[j] = pair_ff{ff_make(0.f), ff_make(1.f)};
                if (j < k) x[j] = pair_load(dsm_pair(cl, spq, fl[j]));
            }
            const pair_ff o = cell_pair(k, op_tt(ops, op), x);
            v = pair_store(o, par);
            y = pair_tr(o);
            spq[slot] = v;
        }
        cluster_arrive();
        if (on) {   // the global copies after the arrival: its release does not wait for them
            pq[ns + c] = v;
            tr[ns + c] = y;
        }
        c = c1, slot = slot1, r = r1, f = f1, on = on1;   // the next level's cell; the one after it now
        on1 = cell_at(s, l + 2, L, rk, t, c1, slot1);
        if (on1) r1 = fanin[c1], f1 = floc[c1];
    }
    cluster_wait();
}

// the raw static data of one cell for the reverse pass
struct ClRaw {
    uint4 r, f;   // record, fanin locations
    int4 lep;     // positions of its input edges in their owners' copies
    int32_t e0, cnt;
    float cl, b;
};
__device__ __forceinline__ void cl_raw(ClRaw &w, const uint4 *fanin, const uint4 *floc, const int32_t *fptr,
                                       const int32_t *lfptr, const int4 *lefpos, const float *cload,
                                       const float *beta, int64_t c, int64_t ns, int grad_mode) {
    const int64_t n = ns + c;
    w.r = fanin[c];
    w.f = floc[c];
    w.lep = lefpos[c];
    w.e0 = lfptr[n];
    w.cnt = fptr[n + 1] - fptr[n];
    w.cl = cload[n];
    w.b = grad_mode ? beta[n] : 1.f;
}

// Shared memory: the block's slots of (P, Q) pairs, the edge adjoints of its nets' fanout
// ranges (net n's range starts at lfptr[n] in its owner's copy), then its tables.
__global__ void __launch_bounds__(kClusterMaxThreads) k_bwd_cluster(
    const uint4 *__restrict__ fanin, const uint4 *__restrict__ floc, const int32_t *__restrict__ fptr,
    const int32_t *__restrict__ lfptr, const int4 *__restrict__ lefpos, const float4 *__restrict__ pq,
    const float *__restrict__ cload, const float *__restrict__ beta, float *gnet, const int32_t *__restrict__ lvl,
    const int32_t *__restrict__ chunk, const int32_t *__restrict__ base, int L, int64_t ns, int64_t nn,
    int64_t slots, int64_t ne_local, int grad_mode, int tr_mode, float K, float *out_gsp, OpTable ops) {
    extern __shared__ float4 spq[];
    const cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rk = (int)cl.block_rank();
    float *sgfo = reinterpret_cast<float *>(spq + slots);
    int *tab = reinterpret_cast<int *>(sgfo + ne_local);
    const Tables s{tab, tab + (L + 1), tab + 2 * (L + 1)};
    const int t = threadIdx.x, B = blockDim.x;
    const int64_t nc = nn - ns;
    prefetch_share_l2(fanin, nc * (int64_t)sizeof(uint4), rk, C);
    prefetch_share_l2(floc, nc * (int64_t)sizeof(uint4), rk, C);
    prefetch_share_l2(lefpos, nc * (int64_t)sizeof(int4), rk, C);
    prefetch_share_l2(lfptr, nn * (int64_t)sizeof(int32_t), rk, C);
    prefetch_share_l2(fptr, (nn + 1) * (int64_t)sizeof(int32_t), rk, C);
    prefetch_share_l2(cload, nn * (int64_t)sizeof(float), rk, C);
    if (grad_mode) prefetch_share_l2(beta, nn * (int64_t)sizeof(float), rk, C);
    load_tables(s, lvl, chunk, base, L, rk);
    __syncthreads();
    // the block's pairs: its chunk of every level (contiguous nets, contiguous slots)
    for (int l = 0; l <= L; l++) {
        const int64_t lo = l ? ns + s.lvl[l - 1] : 0, hi = l ? ns + s.lvl[l] : ns;
        const int64_t first = lo + (int64_t)rk * s.chunk[l];
        for (int p = t; p < s.chunk[l] && first + p < hi; p += B) cp_async16(spq + s.base[l] + p, pq + first + p);
    }
    cp_async_wait_all();
    __syncthreads();
    int64_t c = 0, c1 = 0;
    int slot = 0, slot1 = 0;
    ClRaw w{}, w1{};
    bool on = cell_at(s, L, L, rk, t, c, slot);
    if (on) cl_raw(w, fanin, floc, fptr, lfptr, lefpos, cload, beta, c, ns, grad_mode);
    cluster_arrive();
    cluster_wait();   // every block's pairs are in place
    for (int l = L; l >= 1; l--) {
        // the cell's static part (as in the grid-wide pass), before the wait
        float local = 0.f, d[4] = {0.f, 0.f, 0.f, 0.f};
        int k = 0;
        if (on) {
            local = adj_local(K, w.cl, pair_qmp(spq[slot]));
            const uint32_t op = w.r.x >> 24;
            k = op_arity(ops, op);
            const uint32_t fl[4] = {w.f.x, w.f.y, w.f.z, w.f.w};
            float p[4], q[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                p[j] = 0.f;
                q[j] = 1.f;
                if (j < k) {
                    const float4 v = pq_decode(dsm_pair(cl, spq, fl[j]));
                    p[j] = v.x + v.y;
                    q[j] = v.z + v.w;
                }
            }
            cell_partials(k, op_tt(ops, op), p, q, d);
        }
        const bool on1 = cell_at(s, l - 1, L, rk, t, c1, slot1);   // the next level's raw data
        if (on1) cl_raw(w1, fanin, floc, fptr, lfptr, lefpos, cload, beta, c1, ns, grad_mode);
        if (l < L) cluster_wait();   // the levels above have written their edge adjoints
        float g = 0.f;
        if (on) {
            float acc = 0.f;
            for (int32_t i = 0; i < w.cnt; i++) acc += sgfo[w.e0 + i];
            g = adj_combine(grad_mode, acc, local, w.b);
            const uint32_t fl[4] = {w.f.x, w.f.y, w.f.z, w.f.w};
            const int pos[4] = {w.lep.x, w.lep.y, w.lep.z, w.lep.w};
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (j < k) *(cl.map_shared_rank(sgfo, fl[j] >> 24) + pos[j]) = g * d[j];
        }
        cluster_arrive();
        if (on) gnet[ns + c] = g;   // after the arrival, as in the forward pass
        c = c1, slot = slot1, w = w1, on = on1;
    }
    cluster_wait();   // the last level's edge adjoints are in place; nothing remote after this
    for (int p = t; p < s.chunk[0]; p += B) {   // the block's startpoints
        const int64_t n = (int64_t)rk * s.chunk[0] + p;
        if (n >= ns) break;
        float acc = 0.f;
        const int32_t e0 = lfptr[n], cnt = fptr[n + 1] - fptr[n];
        for (int32_t i = 0; i < cnt; i++) acc += sgfo[e0 + i];
        const float local = tr_mode ? adj_local(K, cload[n], pair_qmp(spq[s.base[0] + p])) : 0.f;
        const float g = adj_combine(grad_mode, acc, local, grad_mode ? beta[n] : 1.f);
        gnet[n] = g;
        if (out_gsp) out_gsp[n] = g;
    }
}

template <class... KArgs, class... Args>
cudaError_t launch_cluster(void (*kern)(KArgs...), int threads, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)kClusterBlocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)kClusterBlocks;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace

size_t cluster_smem(int which, int64_t slots, int64_t n_edges_local, int n_levels) {
    return (size_t)slots * sizeof(float4) + (which ? (size_t)n_edges_local * sizeof(float) : 0) +
           3 * (size_t)(n_levels + 1) * sizeof(int);
}

bool cluster_fits(int threads, size_t smem_fwd, size_t smem_bwd) {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (cudaFuncSetAttribute(k_fwd_cluster, a, kBlockSmemMax) != cudaSuccess ||
        cudaFuncSetAttribute(k_bwd_cluster, a, kBlockSmemMax) != cudaSuccess ||
        cudaFuncSetAttribute(k_fwd_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(k_bwd_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int w = 0; w < 2; w++) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)kClusterBlocks);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = w ? smem_bwd : smem_fwd;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)kClusterBlocks;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        const cudaError_t e = w ? cudaOccupancyMaxActiveClusters(&n, k_bwd_cluster, &cfg)
                                : cudaOccupancyMaxActiveClusters(&n, k_fwd_cluster, &cfg);
        if (e != cudaSuccess || n < 1) {
            cudaGetLastError();
            return false;
        }
    }
    return true;
}

cudaError_t launch_fwd_cluster(const DevDesign &d, const OpTable &ops, const ClusterMap &m, int tr_mode,
                               cudaStream_t s) {
    return launch_cluster(k_fwd_cluster, m.threads, cluster_smem(0, m.slots, 0, d.n_levels), s, d.fanin,
                          (const uint4 *)m.floc, d.pq, d.tr, (const float *)d.sp_in, (const float *)d.tr_in, d.lvl,
                          (const int32_t *)m.chunk, (const int32_t *)m.base, d.n_levels, d.n_start, d.n_nets,
                          m.slots, tr_mode, ops, (const uint32_t *)d.epoch);
}

cudaError_t launch_bwd_cluster(const DevDesign &d, const OpTable &ops, const ClusterMap &m, int grad_mode,
                               int tr_mode, float K, float *out_gsp, cudaStream_t s) {
    return launch_cluster(k_bwd_cluster, m.threads, cluster_smem(1, m.slots, m.edges, d.n_levels), s, d.fanin,
                          (const uint4 *)m.floc, d.fout_ptr, (const int32_t *)m.lfptr, (const int4 *)m.lefpos,
                          (const float4 *)d.pq, (const float *)d.cload, (const float *)d.beta, d.gnet, d.lvl,
                          (const int32_t *)m.chunk, (const int32_t *)m.base, d.n_levels, d.n_start, d.n_nets,
                          m.slots, m.edges, grad_mode, tr_mode, K, out_gsp, ops);
}

}  // namespace dp
