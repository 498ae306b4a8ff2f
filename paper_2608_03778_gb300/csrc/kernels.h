// Launch wrappers for the GPU kernels (implemented in kern_*.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace dp {

// Per-design function table passed by value to kernels (lives in the
// constant bank): entry = truth table (bits 0..15) | arity << 16 |
// (for arity <= 3) the 8-bit LOP3 table of the function << 24, whose entry
// 4 x2 + 2 x1 + x0 is f(x0, x1, x2) (inputs beyond the arity ignored).
struct OpTable {
    uint32_t e[256];
};

constexpr int kPersistThreads = 512;
// the persistent forward pass runs beside the startpoint generator: a smaller block leaves
// the generator more registers on every SM (one block of 256 threads per SM still gives one
// thread per cell of a 38,912-cell level)
constexpr int kFwdThreads = 256;
constexpr int kSimThreads = 512;
// the single-block passes of small designs: at most kBlockMaxWidth cells per level
// (one per thread) and state within kBlockSmemMax bytes of shared memory
constexpr int kBlockThreads = 1024;
constexpr int kBlockMaxWidth = kBlockThreads;
constexpr int kBlockSmemMax = 224 * 1024;   // dynamic; the 227 KiB a block may hold less room for static arrays
// bounded waits give up after this many SM cycles (about 2 s at 2 GHz)
constexpr long long kWaitLimitCycles = 4000000000LL;

// Device-resident design state; every pointer is device memory.
struct DevDesign {
    int64_t n_nets, n_start, n_cells;
    int32_t n_levels;
    const uint4 *fanin;        // [n_cells]: 4 internal net ids, logic id in bits 24..31 of .x
    const int32_t *fout_ptr;   // [n_nets+1]
    const int32_t *fout_edge;  // [n_edges]: 4*cell + slot
    const int32_t *edge_fpos;  // [4*n_cells]: position of edge (cell, slot) in the fanout CSR, -1 unused
    const int32_t *lvl;        // [n_levels+1] level boundaries over internal cells
    const int32_t *net_of_user;
    const int32_t *cell_of_user;
    const float *base_cap;     // wire + DFF D pin caps
    float *pincap;             // [n_cells]
    float *cload;              // [n_nets]
    float *sp_in, *tr_in;      // [n_start] staged inputs
    float4 *pq;                // [n_nets] (P(net=1), P(net=0)) as float-float pairs (P.hi, P.lo, Q.hi, Q.lo)
    float *tr;                 // [n_nets] TR_model (startpoints: input TR in tr_mode 0)
    float *beta, *trh;         // [n_nets] beta and hybrid TR
    uint32_t *toggles, *ones;  // [n_nets]
    float *gnet;               // [n_nets] SP adjoint per net
    float *gfo;                // [n_edges] adjoint contribution of each edge, in fanout-CSR order
    uint64_t *words;           // [n_nets * T]
    double *partials;          // [2 * power_blocks]
    double *power;             // [4]: model, hybrid
    unsigned *bar;             // level-barrier arrival counters of the persistent passes (128-byte lines)
    uint32_t *epoch;           // [4] pass counters: [0] forward (its parity tags the stored pairs)
    const int32_t *chunk_ptr;  // [n_levels+2] level-aligned chunks of 32 (level 0 = startpoints)
    const int32_t *pair_ptr;   // [n_levels+1] level-aligned cell pairs: pairs of level l are [pair_ptr[l-1], pair_ptr[l])
    unsigned *simdone;         // [n_cells] pass number of the simulation pass that last wrote the cell's words
    const int32_t *dead_ptr;   // [n_levels+2] nets by death level d (the highest level reading the net, else
    const int32_t *dead_net;   // [n_nets]      its own): dead_net[dead_ptr[d] .. dead_ptr[d+1])
    int *err;                  // device error word of the context (bounded wait gave up)
};

constexpr int kPowerBlocks = 304;   // fixed grid of the power reduction -> deterministic order
constexpr int kPowerThreads = 256;

// forward (kern_fwd.cu)
void launch_init_start(const DevDesign &d, int tr_mode, cudaStream_t s);
void launch_fwd_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, cudaStream_t s);
void launch_cload(const DevDesign &d, cudaStream_t s);
void launch_set_pincap(const DevDesign &d, const int32_t *cells, const float *caps, int32_t n, cudaStream_t s);
// power: sum_n alpha_n C_n (alpha = tr, or beta*tr when hybrid), times K, into d.power[slot]
void launch_power(const DevDesign &d, bool hybrid, double K, int slot, cudaStream_t s);
// outputs in user order: grad_cload (K alpha), grad_pincap (K sum fanin alpha), grad_tr_in (K beta C or 0)
void launch_cap_grads(const DevDesign &d, const OpTable &ops, bool hybrid, int tr_mode, double K, float *grad_cload,
                      float *grad_pincap, float *grad_tr_in, cudaStream_t s);
void launch_gather_f32(const float *src, const int32_t *idx, float *dst, int64_t n, cudaStream_t s);
void launch_gather_u32(const uint32_t *src, const int32_t *idx, uint32_t *dst, int64_t n, cudaStream_t s);
void launch_trh_user(const DevDesign &d, float *dst, cudaStream_t s);
void launch_sp_user(const DevDesign &d, float *dst, cudaStream_t s);

// backward (kern_bwd.cu)
void launch_bwd_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, int grad_mode, float K,
                      cudaStream_t s);
void launch_bwd_start(const DevDesign &d, int grad_mode, int tr_mode, float K, float *grad_sp_in, cudaStream_t s);

// pass counters and the dataflow schedule (kern_flow.cu)
void launch_bump(uint32_t *counter, cudaStream_t s);
int flow_grid(int which, int sm_count, int blocks_per_sm);   // which: 0 forward, 1 simulation; 0 = unavailable
cudaError_t launch_fwd_flow(const DevDesign &d, const OpTable &ops, int tr_mode, int grid, unsigned sleep_max,
                            cudaStream_t s);
// simulation levels without barriers (T % 4 == 0), bumps epoch[1] first
cudaError_t launch_sim_flow(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s);

// persistent schedule (kern_persist.cu): one cooperative launch per pass
int persist_grid(int which, int sm_count);   // which: 0 forward, 1 simulation, 2 backward, 3 wide simulation
bool wide_ok(int T);                         // the wide simulation handles this word count
cudaError_t launch_sim_wide(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s);
size_t persist_bar_words(int n_levels);      // counters needed by the three passes
// ready (may be null) is recorded on s just before the kernel: a branch forked there becomes
// ready with it rather than ahead of it
// the forward and the reverse pass of a mid-size design in one cluster of kClusterBlocks blocks
// (kern_cluster.cu): every level cut into one contiguous chunk per block, each net kept in the
// shared memory of the block that computes it, the hardware cluster barrier between levels.
constexpr int kClusterBlocks = 16;
constexpr int kClusterMaxThreads = 512;
struct ClusterMap {
    int threads = 0;                    // threads per block (0: the design does not use the cluster)
    int64_t slots = 0;                  // the most nets one block holds
    int64_t edges = 0;                  // the most edge adjoints one block holds
    const int32_t *chunk = nullptr;     // [L+1] cells of level l per block (level 0: the startpoints)
    const int32_t *base = nullptr;      // [C][L+1] first slot of block b's chunk of level l
    const int32_t *floc = nullptr;      // [4 nc] location of each input net: owner block << 24 | slot
    const int32_t *lfptr = nullptr;     // [nn] start of net n's fanout range in its owner's copy
    const int32_t *lefpos = nullptr;    // [4 nc] position of each input edge in its owner's copy
};
// cluster_smem(0 forward, 1 reverse, ...): dynamic shared memory per block; cluster_fits:
// whether one such cluster can run on this device (also sets the kernels' shared-memory and
// cluster-size attributes)
size_t cluster_smem(int which, int64_t slots, int64_t n_edges_local, int n_levels);
bool cluster_fits(int threads, size_t smem_fwd, size_t smem_bwd);
cudaError_t launch_fwd_cluster(const DevDesign &d, const OpTable &ops, const ClusterMap &m, int tr_mode,
                               cudaStream_t s);
cudaError_t launch_bwd_cluster(const DevDesign &d, const OpTable &ops, const ClusterMap &m, int grad_mode,
                               int tr_mode, float K, float *out_gsp, cudaStream_t s);

// the forward and the reverse pass of a small design in one block (kern_persist.cu);
// block_smem(0 forward, 1 reverse, ...): the dynamic shared memory each needs;
// block_smem_init: raises the kernels' shared-memory limit to kBlockSmemMax (once)
size_t block_smem(int which, int64_t n_nets, int64_t n_edges, int n_levels);
bool block_smem_init();
// (the forward kernel also advances the pass counter)
cudaError_t launch_fwd_block(const DevDesign &d, const OpTable &ops, int tr_mode, int threads, cudaStream_t s);
cudaError_t launch_bwd_block(const DevDesign &d, const OpTable &ops, int grad_mode, int tr_mode, float K,
                             float *out_gsp, int64_t n_edges, int threads, cudaStream_t s);
cudaError_t launch_fwd_persist(const DevDesign &d, const OpTable &ops, int tr_mode, int grid, cudaStream_t s,
                               cudaEvent_t ready = nullptr);
cudaError_t launch_sim_persist(const DevDesign &d, const OpTable &ops, int T, int grid, cudaStream_t s);
// pre: the form that loads each level's static part a level ahead (about 120 registers: no
// other kernel fits beside it on an SM); otherwise the 64-register form
cudaError_t launch_bwd_persist(const DevDesign &d, const OpTable &ops, int grad_mode, int tr_mode, float K,
                               float *out_gsp, int grid, bool pre, cudaStream_t s);
cudaError_t launch_wait_selftest(unsigned *bar, int *err, long long limit, cudaStream_t s);
// latency probes (buffers owned by the caller; bar zeroed by the caller, 32 words per level)
cudaError_t launch_probe_levels(float *buf, int levels, int gather, int grid, int threads, unsigned *bar, int *err,
                                cudaStream_t s);
cudaError_t launch_probe_chase(const uint32_t *next, int hops, uint32_t *sink, cudaStream_t s);

// Batched scenarios (kern_batch.cu): S scenarios of one design, every per-net
// value stored scenario-innermost (value[n * S + s]).
struct BatchBufs {
    int64_t S;
    float *sp_in, *tr_in;   // [n_start * S] staged inputs
    float2 *pq;             // [n_nets * S] float-float P(net=1) (hi, lo); P(net=0) = 1 - P re-derived
    float *gfo;             // [n_edges * S] edge adjoints in fanout-CSR order
    float *gsp;             // [n_start * S] SP adjoint of the startpoints
    double *partials;       // [kBatchPowerChunks * S]
    double *power;          // [S] model power per scenario
    float *ks;              // [S] per-scenario seed of the backward (K * weight), binary32
    const float *dcl;       // [n_nets * S] per-scenario change of C_load (sizing deltas), or NULL
    // lag-one mode (tr_mode 2) only, else NULL:
    float *tq;              // [n_nets * S] TR of every net
    float2 *gfo2;           // [n_edges * S] edge adjoints of (P, TR)
    float *gtr;             // [n_start * S] TR adjoint of the startpoints
};
constexpr int kBatchPowerChunks = 1024;   // fixed split of the nets -> deterministic FP64 sums

struct BatchShape {
    int bx, by;   // threads over scenarios x cells per block
    int v = 1;    // scenarios per thread in the forward and reverse cell levels (1, 2 or 4; 1 unless S is a multiple)
};

void launch_fwdb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl_host, int tr_mode,
                 BatchShape sh, cudaStream_t s);
// lag-one mode (kern_lag1.cu): forward of (P, TR) and reverse pass of both adjoints
void launch_fwdl(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl_host, BatchShape sh,
                 cudaStream_t s);
void launch_bwdl(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl_host, BatchShape sh,
                 cudaStream_t s);
void launch_powerb(const DevDesign &d, const BatchBufs &b, int tr_mode, double K, cudaStream_t s);
// ks[s] = K * weights[s] (weights NULL: K)
void launch_seedb(const BatchBufs &b, double K, const double *weights, cudaStream_t s);
void launch_bwdb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, const int32_t *lvl_host, int tr_mode,
                 BatchShape sh, cudaStream_t s);
// per-scenario gradient outputs ([x][S], user order), or summed over scenarios in FP64 ([x]) when reduce
void launch_gradb(const DevDesign &d, const BatchBufs &b, const OpTable &ops, int tr_mode, bool reduce, float *gtr,
                  float *gpin, float *gcl, cudaStream_t s);
void launch_netb_user(const DevDesign &d, const BatchBufs &b, int tr_mode, float *sp, float *tr, cudaStream_t s);
// Sizing deltas of a served batch (kern_serve.cu): per-scenario changes of cell
// pin caps turned into per-scenario C_load changes, deterministically.
constexpr int kMaxFanin = 4;
struct SizingDeltas {
    const int32_t *cell;        // [ne] cell-line index of each entry
    const float *cap;           // [ne] its new input pin cap, fF
    const int32_t *off;         // [n_req + 1] entries of request (scenario) s: [off[s], off[s+1]); an entry's
    int32_t n_req;              //   position within its request (the last one counts) is its index - off[s]
    int *win;                   // [n_cells * S] -1 at rest
    float *dpin;                // [n_cells * S] 0 at rest
    unsigned *flag;             // [n_nets * S] 0 at rest
    int64_t *list;              // [kMaxFanin * ne] claimed (net, scenario) slots
    unsigned long long *count;  // entries of list
};
// fills dcl[n * S + s] for every net loaded by a changed cell
void launch_sizing_deltas(const DevDesign &d, const OpTable &ops, const SizingDeltas &z, int64_t ne, int64_t S,
                          float *dcl, cudaStream_t s);
// returns win, dpin, flag and dcl to rest after the batch
// the reference inputs' forward state (P of every net, TR of every startpoint) into every
// scenario column of a batch: a batch of requests on the reference inputs skips the forward pass
void launch_bcast_ref(const float2 *ref_pq, const float *ref_tr, float2 *pq, float *tr_in, int64_t nn, int64_t ns,
                      int64_t S, cudaStream_t s);
void launch_sizing_clear(const DevDesign &d, const SizingDeltas &z, int64_t ne, int64_t S, float *dcl,
                         cudaStream_t s);
// out[c][r] = in[r][c] (row-major R x C in, C x R out)
void launch_transpose(const float *in, float *out, int64_t R, int64_t C, cudaStream_t s);
// x <- clip(x + eta g, 0, 1) (Algorithm 4 ascent step with projection)
void launch_ascent(float *x, const float *g, int64_t n, float eta, cudaStream_t s);
// Eq. 3: threshold SP at 0.5 into v0 (v1 = not v0), two bitwise forwards, sum of C over nets whose values differ
void launch_virus(const DevDesign &d, const OpTable &ops, const int32_t *lvl_host, const float *sp, int64_t S,
                  uint64_t *words, uint8_t *v0, double *partials, double *out, cudaStream_t s);

// sizing score (kern_size.cu): Eq. 8 per cell line, and the radix select of its top k
void launch_scores(const DevDesign &d, bool hybrid, float K, int mode, float *out, cudaStream_t s);
void launch_radix_hist(const float *scores, int64_t n, uint32_t prefix, uint32_t mask, int shift, unsigned *hist,
                       cudaStream_t s);
void launch_radix_collect(const float *scores, int64_t n, uint32_t thr, int32_t *idx, unsigned *count, int64_t cap,
                          cudaStream_t s);

// simulation (kern_sim.cu)
void launch_sim_start(const DevDesign &d, int T, uint64_t seed, cudaStream_t s);
void launch_sim_level(const DevDesign &d, const OpTable &ops, int32_t c0, int32_t c1, int T, cudaStream_t s);
void launch_hybrid(const DevDesign &d, int T, int tr_mode, float beta_min, float beta_max, cudaStream_t s);

}  // namespace dp
