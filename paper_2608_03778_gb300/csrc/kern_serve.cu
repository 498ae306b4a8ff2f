// Sizing deltas of a served batch, turned into per-scenario C_load changes on
// the device.  A delta entry (cell u, new pin cap, scenario s, position i in
// its request) changes cell u's input pin cap in scenario s; the change loads
// every input net of u (one pin cap per cell, R10).
//
// An entry's scenario is found from the requests' entry offsets (a binary
// search), its position as its index within the request.
//
//   1. win[c][s]  = the largest position i among the entries of cell c in s
//                   (a cell listed more than once counts with its last entry);
//   2. dpin[c][s] = new cap - base cap, written by that entry alone;
//   3. every input net n of a changed cell is claimed once per scenario; the
//      claimer sums dpin over n's sink cells in fanout-CSR order (so the value
//      does not depend on which entry claimed it) into dcl[n][s] and records
//      (n, s) for the clean-up;
//   4. after the batch every touched entry of win, dpin, flag and dcl returns to
//      its resting value.
// All values written are independent of thread order: the batch's results are
// reproducible bit for bit.
#include "kern_common.cuh"

namespace dp {
namespace {

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// scenario and position within its request of entry i (off: request offsets, ascending)
__device__ __forceinline__ void entry_of(const int32_t *__restrict__ off, int32_t n_req, int64_t i, int64_t &s,
                                         int32_t &pos) {
    int32_t lo = 0, hi = n_req - 1;   // the last request whose first entry is <= i
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    s = lo;
    pos = (int32_t)(i - off[lo]);
}

__global__ void k_delta_win(const int32_t *__restrict__ cell, const int32_t *__restrict__ off, int32_t n_req,
                            const int32_t *__restrict__ cell_of_user, int *win, int64_t ne, int64_t S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t sc;
    int32_t pos;
    entry_of(off, n_req, i, sc, pos);
    const int64_t c = cell_of_user[cell[i]];
    atomicMax(win + c * S + sc, pos);
}

__global__ void k_delta_pin(const int32_t *__restrict__ cell, const float *__restrict__ cap,
                            const int32_t *__restrict__ off, int32_t n_req, const int32_t *__restrict__ cell_of_user,
                            const float *__restrict__ pincap, const int *__restrict__ win, float *dpin, int64_t ne,
                            int64_t S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t sc;
    int32_t pos;
    entry_of(off, n_req, i, sc, pos);
    const int64_t c = cell_of_user[cell[i]];
    if (win[c * S + sc] == pos) dpin[c * S + sc] = __fsub_rn(cap[i], pincap[c]);
}

__global__ void k_delta_claim(const int32_t *__restrict__ cell, const int32_t *__restrict__ off, int32_t n_req,
                              const int32_t *__restrict__ cell_of_user, const int *__restrict__ win,
                              const uint4 *__restrict__ fanin, const int32_t *__restrict__ fptr,
                              const int32_t *__restrict__ fedge, const float *__restrict__ dpin, unsigned *flag,
                              float *dcl, int64_t *list, unsigned long long *count, int64_t ne, int64_t S,
                              OpTable ops) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t s;
    int32_t pos;
    entry_of(off, n_req, i, s, pos);
    const int64_t c = cell_of_user[cell[i]];
    if (win[c * S + s] != pos) return;
    const uint4 r = fanin[c];
    const int k = op_arity(ops, r.x >> 24);
    const uint32_t n4[4] = {r.x & kMask24, r.y, r.z, r.w};
    for (int j = 0; j < k; j++) {
        const int64_t n = n4[j];
        if (atomicCAS(flag + n * S + s, 0u, 1u) != 0u) continue;
        float sum = 0.f;
        for (int32_t e = fptr[n]; e < fptr[n + 1]; e++) sum += dpin[(int64_t)(fedge[e] >> 2) * S + s];
        dcl[n * S + s] = sum;
        list[atomicAdd(count, 1ull)] = n * S + s;
    }
}

__global__ void k_delta_clear_nets(const int64_t *__restrict__ list, const unsigned long long *__restrict__ count,
                                   unsigned *flag, float *dcl, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || (unsigned long long)i >= *count) return;
    const int64_t at = list[i];
    flag[at] = 0u;
    dcl[at] = 0.f;
}

__global__ void k_delta_clear_cells(const int32_t *__restrict__ cell, const int32_t *__restrict__ off,
                                    int32_t n_req, const int32_t *__restrict__ cell_of_user, int *win, float *dpin,
                                    int64_t ne, int64_t S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    int64_t sc;
    int32_t pos;
    entry_of(off, n_req, i, sc, pos);
    const int64_t at = (int64_t)cell_of_user[cell[i]] * S + sc;
    win[at] = -1;
    dpin[at] = 0.f;
}

// every scenario column of a batch gets the reference inputs' forward state:
// the float-float P of every net and the input TR of every startpoint
__global__ void k_bcast_ref(const float2 *__restrict__ ref_pq, const float *__restrict__ ref_tr, float2 *pq,
                            float *tr_in, int64_t nn, int64_t ns, int64_t S) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    for (int64_t n = blockIdx.y; n < nn; n += gridDim.y) {
        pq[n * S + s] = ref_pq[n];
        if (n < ns) tr_in[n * S + s] = ref_tr[n];
    }
}

}  // namespace

void launch_sizing_deltas(const DevDesign &d, const OpTable &ops, const SizingDeltas &z, int64_t ne, int64_t S,
                          float *dcl, cudaStream_t s) {
    if (ne <= 0) return;
    const unsigned g = (unsigned)cdiv(ne, 256);
    cudaMemsetAsync(z.count, 0, sizeof(unsigned long long), s);
    k_delta_win<<<g, 256, 0, s>>>(z.cell, z.off, z.n_req, d.cell_of_user, z.win, ne, S);
    k_delta_pin<<<g, 256, 0, s>>>(z.cell, z.cap, z.off, z.n_req, d.cell_of_user, d.pincap, z.win, z.dpin, ne, S);
    k_delta_claim<<<g, 256, 0, s>>>(z.cell, z.off, z.n_req, d.cell_of_user, z.win, d.fanin, d.fout_ptr, d.fout_edge,
                                    z.dpin, z.flag, dcl, z.list, z.count, ne, S, ops);
}

void launch_sizing_clear(const DevDesign &d, const SizingDeltas &z, int64_t ne, int64_t S, float *dcl,
                         cudaStream_t s) {
    if (ne <= 0) return;
    const int64_t cap = ne * kMaxFanin;
    k_delta_clear_nets<<<(unsigned)cdiv(cap, 256), 256, 0, s>>>(z.list, z.count, z.flag, dcl, cap);
    k_delta_clear_cells<<<(unsigned)cdiv(ne, 256), 256, 0, s>>>(z.cell, z.off, z.n_req, d.cell_of_user, z.win,
                                                                z.dpin, ne, S);
}

void launch_bcast_ref(const float2 *ref_pq, const float *ref_tr, float2 *pq, float *tr_in, int64_t nn, int64_t ns,
                      int64_t S, cudaStream_t s) {
    if (nn <= 0 || S <= 0) return;
    const unsigned bx = S >= 128 ? 128u : 32u;
    k_bcast_ref<<<dim3((unsigned)cdiv(S, bx), (unsigned)(nn < 8192 ? nn : 8192)), bx, 0, s>>>(ref_pq, ref_tr, pq,
                                                                                              tr_in, nn, ns, S);
}

}  // namespace dp
