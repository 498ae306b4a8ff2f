/*
 * diffpower.h - C-ABI of the GB300 DiffPower hot path (libdiffpower.so).
 *
 * The library keeps a compiled netlist resident on one GPU and runs the
 * paper's analysis steps on it:
 *   load a bytecode netlist (Sec. III-A, Algorithm 1), set the startpoint SP/TR
 *   (Sec. III-A), propagate SP/TR (Sec. III-B, Algorithm 2, Eq. 2), simulate
 *   (Sec. III-C, Eq. 4), calibrate beta (Sec. III-D, Eq. 5), report switching
 *   power (Eq. 1) and back-propagate its gradient (Sec. III-E, Eq. 6, Eq. 7).
 *
 * Conventions for every entry point:
 *  - Return value: DP_OK or an error code; after an error, dp_last_error()
 *    on the context gives a one-line message. Invalid sizes, NULL required
 *    pointers and calls in the wrong order are rejected before any GPU work.
 *  - Ownership: the library owns dp_ctx, dp_design and dp_compiled objects
 *    and their device memory. Caller buffers are borrowed for the duration of
 *    the call only: inputs are copied in, outputs are written into caller
 *    memory. `on_device` = 1 means the caller's pointers are device pointers
 *    on the context's device, 0 means host pointers.
 *  - Ordering: every per-net array is in net declaration order of the
 *    netlist text, every per-startpoint array in the order in which
 *    startpoints appear (`input` and `dff` lines), every per-cell array in the
 *    order of `cell` lines. The library's internal renumbering never shows.
 *  - Streams: work is queued on the context's stream (the one given to
 *    dp_create, e.g. PyTorch's current stream, or a private one). Calls that
 *    write host memory synchronise that stream before they return; calls
 *    with device outputs return without synchronising.
 *  - Threads: one context per host thread.
 *  - Device waits: no kernel of the library waits without a bound. A wait
 *    that runs out records an error on the device; the next synchronising
 *    call returns DP_ETIMEOUT and the design stays usable.
 *
 * Text formats (whitespace separated, '#' starts a comment):
 *   library:  cell <ref> <out_pin> <pin_cap_fF> <function>
 *             seq  <ref> <d_pin> <q_pin> <d_pin_cap_fF>
 *     <function> uses identifiers (input pins), 0, 1, parentheses and
 *     ! ~ (not, prefix), ' (not, postfix), & * (and), ^ (xor), | + (or), with
 *     precedence NOT > AND > XOR > OR (Sec. III-A).
 *   netlist:  net <name> <wire_cap_fF>          (declares a net, in order)
 *             input <net>                        (primary input: startpoint)
 *             output <net>                       (primary output: no extra load)
 *             dff <inst> <seq_ref> <d>=<net> <q>=<net>
 *                 (Q is a pseudo-primary input / startpoint; D is a
 *                  pseudo-primary output and adds the D pin cap to its net)
 *             cell <inst> <ref> <pin>=<net> ... (every pin connected once)
 *   Every net needs exactly one driver; combinational cycles are rejected.
 *   Limits: at most 4 inputs per cell, fewer than 2^24 nets.
 */
#ifndef DIFFPOWER_H
#define DIFFPOWER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DP_OK = 0,
    DP_EINVAL = 1,        /* bad argument or size */
    DP_EPARSE = 2,        /* malformed library or netlist text */
    DP_ECYCLE = 3,        /* combinational cycle */
    DP_ENOMEM = 4,        /* host or device allocation failed */
    DP_ECUDA = 5,         /* a CUDA runtime call failed */
    DP_ETIMEOUT = 6,      /* a bounded device wait gave up */
    DP_ESTATE = 7,        /* call out of order (e.g. backward before propagate) */
    DP_EUNSUPPORTED = 8   /* valid input beyond this library's limits */
} dp_status;

typedef struct dp_ctx dp_ctx;
typedef struct dp_design dp_design;
typedef struct dp_compiled dp_compiled;

/* Analysis settings.  Defaults (dp_config_default): Vdd 0.8 V, f 1 GHz,
 * beta in [0.1, 10] (Sec. V-B), tr_mode 0, grad_mode 1, 64 words (4,096
 * vectors), seed 42. */
typedef struct {
    double vdd;          /* supply voltage, V (Eq. 1) */
    double fclk;         /* clock frequency, Hz (Eq. 1) */
    float beta_min;      /* Eq. 5 clip bounds */
    float beta_max;
    int32_t tr_mode;     /* 0: startpoint TR = given input TR, 2P(1-P) elsewhere;
                            1: TR = 2P(1-P) on every net (Eq. 2, Algorithm 2 kernel 3);
                            2: lag-one - every net carries (SP, TR), consecutive values follow
                               q(1,1) = P - TR/2, q(0,0) = 1 - P - TR/2, q(0,1) = q(1,0) = TR/2, and
                               a cell's TR is sum_(a,b) prod_i q_i(a_i, b_i) [f(a) != f(b)] (its
                               exact toggle rate on fanout-free circuits; Eq. 2 when every input
                               has TR = 2P(1-P)).  Batched inputs only (dp_set_inputs_batch);
                               needs TR <= 2 min(P, 1-P) at the startpoints; model gradient only. */
    int32_t grad_mode;   /* 0: gradient of the model power (Eq. 7);
                            1: hybrid, paper rule - each net's accumulated gradient
                               is multiplied by its beta (Eq. 6);
                            2: hybrid, exact gradient of sum K beta TR C with beta fixed */
    int32_t sim_words;   /* T, 64-bit words per net: 64*T vectors, 64*(T-1) transitions (Eq. 4); 2..4096 */
    int32_t schedule;    /* 0 (default): for a small design (dp_info.block_threads > 0) the
                               forward and the reverse pass each run in one thread block, with
                               block barriers between levels and the pairs and edge adjoints
                               in shared memory; for a mid-size one (dp_info.cluster_threads >
                               0) in one cluster of 16 blocks, with the cluster barrier between
                               levels and the pairs and edge adjoints spread over the blocks'
                               shared memory; otherwise, and for the simulation, as 2;
                            2: one cooperative launch per pass with grid-wide level barriers;
                            1: one launch per level;
                            3: dataflow forward pass - warps take cells in topological order and
                               wait only for their own fanins (other passes as 2).
                            Where a cooperative grid cannot be co-resident the library uses 1.
                            All give bitwise identical results. */
    uint64_t seed;       /* Philox4x32-10 key for the startpoint Markov chains (Sec. III-C) */
} dp_config;

typedef struct {
    int64_t n_nets;      /* all nets, startpoints included */
    int64_t n_start;     /* startpoints: primary inputs + DFF Q pins */
    int64_t n_cells;     /* combinational cells */
    int64_t n_edges;     /* cell input pins (fanin edges) */
    int32_t n_levels;    /* depth: cells sit on levels 1..n_levels (Sec. III-A) */
    int32_t n_ops;       /* distinct cell functions (logic ids) in use */
    size_t device_bytes; /* device memory held by the design, bytes */
    int32_t block_threads; /* > 0: the design is small enough for the single-block forward and
                              reverse passes (schedule 0), run with this many threads;
                              0: it is not (and always 0 from dp_compiled_info) */
    int32_t cluster_threads; /* > 0: the design is not, but fits the single-cluster passes
                                (schedule 0: 16 blocks of this many threads, nets spread over
                                their shared memory); 0 otherwise and from dp_compiled_info */
} dp_info;

/* Fills *cfg with the defaults above. */
void dp_config_default(dp_config *cfg);

/* One-line message of the last failing call on this context (never NULL). */
const char *dp_last_error(const dp_ctx *ctx);

/* ---------------- host-only compilation (no GPU needed) ---------------- */

/* Compiles library + netlist text on the host (Sec. III-A, Algorithm 1):
 * parses every library function into post-order stack bytecode (IN(k), NOT,
 * AND, OR, XOR, CONST_0/1), matches common gates to fixed logic ids and
 * deduplicates the rest by bytecode signature, derives each function's truth
 * table by running its bytecode, levelizes the netlist, renumbers cells level
 * by level sorted by logic id, and builds the fanin records and the
 * transposed fanout CSR.  On failure returns DP_EPARSE / DP_ECYCLE /
 * DP_EUNSUPPORTED / DP_ENOMEM and writes a message into err (errlen bytes,
 * may be NULL). *out is owned by the caller and freed with dp_compiled_free. */
dp_status dp_compile(const char *netlist, size_t netlist_len, const char *library, size_t library_len,
                     dp_compiled **out, char *err, size_t errlen);
void dp_compiled_free(dp_compiled *c);
dp_status dp_compiled_info(const dp_compiled *c, dp_info *info);

/* A compiled netlist as a self-contained byte blob (host memory, little-endian):
 * compile once, store, load later without the netlist text.  dp_compiled_save
 * writes the blob into buf when cap is large enough (buf may be NULL to ask for
 * the size) and always sets *len to the blob's size; DP_EINVAL when buf is too
 * small.  dp_compiled_load reads a blob (borrowed for the call) into a new
 * compiled netlist owned by the caller; every size and every structural
 * property the device code relies on (levels, fanin ids below the cell's own
 * level, fanout CSR and edge positions, user-order permutations, finite
 * non-negative caps, bytecode ranges) is checked, and a damaged blob returns
 * DP_EPARSE with a message in err. */
dp_status dp_compiled_save(const dp_compiled *c, void *buf, size_t cap, size_t *len);
dp_status dp_compiled_load(const void *blob, size_t len, dp_compiled **out, char *err, size_t errlen);

/* Read-only views into a compiled netlist, for inspection and tests.  All
 * pointers are host memory owned by *c and valid until dp_compiled_free.
 * Internal numbering: nets [0, n_start) are the startpoints in input order;
 * internal cell i (level-major, sorted by logic id inside a level) drives
 * internal net n_start + i. */
typedef struct {
    const int32_t *lvl_ptr;      /* [n_levels+1]: cells of level l (1-based) are [lvl_ptr[l-1], lvl_ptr[l]) */
    const uint32_t *fanin;       /* [4*n_cells]: word 4i+j = internal net of input slot j of cell i;
                                    bits 24..31 of word 4i hold the cell's logic id; unused slots 0xFFFFFF */
    const int32_t *fout_ptr;     /* [n_nets+1]: fanout edges of internal net n */
    const int32_t *fout_edge;    /* [n_edges]: edge id 4*cell+slot, ascending within a net */
    const int32_t *net_of_user;  /* [n_nets]: declaration index -> internal net */
    const int32_t *cell_of_user; /* [n_cells]: cell line index -> internal cell */
    const float *base_cap;       /* [n_nets]: wire cap + DFF D pin caps, fF, internal order */
    const float *pincap;         /* [n_cells]: input pin cap, fF, internal order */
    const uint8_t *op_arity;     /* [256]: inputs of each logic id */
    const uint16_t *op_tt;       /* [256]: truth table, bit m = f(m), bit j of m = input slot j */
    /* Algorithm 1 export: bytecode of every non-common function (logic id >= 32) */
    const uint8_t *bc_ops;       /* [n_bc]: 0 IN, 1 NOT, 2 AND, 3 OR, 4 XOR, 5 CONST_0, 6 CONST_1 */
    const int8_t *bc_args;       /* [n_bc]: IN slot, else 0 */
    const int32_t *bc_offset;    /* [256]: start of a logic id's bytecode, -1 for common gates */
    const int32_t *bc_length;    /* [256] */
    int64_t n_bc;
} dp_compiled_view;
dp_status dp_compiled_view_get(const dp_compiled *c, dp_compiled_view *view);

/* Logic id and bytecode of one function string under the library rules
 * (Algorithm 1 for a single expression).  ops/args receive up to cap
 * instructions; *len the full length; *n_inputs the input count; *tt the
 * truth table when n_inputs <= 4; *logic_id the common-gate id (< 32), or -1
 * for a function that would get a generated id. */
dp_status dp_compile_function(const char *func, uint8_t *ops, int8_t *args, int32_t cap, int32_t *len,
                              int32_t *n_inputs, uint16_t *tt, int32_t *logic_id);

/* ------------------------------ GPU side ------------------------------- */

/* Creates a context on CUDA device `device`.  `cuda_stream` is the
 * cudaStream_t to queue work on, used as given: NULL is the device's default
 * (legacy) stream, which is also PyTorch's default current stream. */
dp_status dp_create(int device, void *cuda_stream, dp_ctx **out);
void dp_destroy(dp_ctx *ctx);

/* Waits for all work queued by this context; returns DP_ETIMEOUT if a bounded
 * device wait gave up since the last synchronisation (the error word is then
 * cleared and the context stays usable). */
dp_status dp_sync(dp_ctx *ctx);

/* Self-test of the bounded device wait: runs a two-block grid barrier that
 * waits for an arrival that never comes, with a limit of `seconds`; the wait
 * gives up, and the call returns DP_ETIMEOUT with the context still usable.
 * No GPU fault is involved. */
dp_status dp_selftest_wait(dp_ctx *ctx, double seconds);

/* Test hook on the calling thread's CUDA runtime error state (the library's
 * own runtime, linked statically).  action 1 plants a launch-configuration
 * error: a kernel launch with zero threads per block, which the runtime
 * rejects on the host, so no work reaches the GPU.  action 2 takes (reads and
 * clears) the pending error; action 0 only reads it.  *pending (may be NULL)
 * receives the cudaError_t code pending after the action (before the clear,
 * for action 2).  Any other action returns DP_EINVAL. */
dp_status dp_selftest_pending_error(int action, int32_t *pending);

/* Latency probes of the level-synchronous schedule on this GPU: the cost per
 * level that bounds the persistent passes (Algorithm 2 and 3 walk the levels
 * in order, so each level waits for the one before it).  Each figure is the
 * difference of two timed launches (n and 3n units, CUDA events), divided by
 * 2n, so launch costs cancel.  out[6] (host):
 *   [0] us per level barrier on one block of 256 threads per SM (the forward
 *       pass's grid), [1] us per level of its skeleton: barrier, then three
 *       loads through L2 of values other blocks stored in the previous level
 *       and one store, [2], [3] the same on 512-thread blocks (the reverse
 *       pass's grid), [4] us per dependent L2 load (one thread chasing a
 *       pointer cycle through 8 MB resident in L2), [5] blocks of the grid.
 * levels in [16, 20000] (DP_EINVAL otherwise).  Every wait is bounded
 * (DP_ETIMEOUT).  Allocates and frees its own buffers; synchronises. */
dp_status dp_probe_latency(dp_ctx *ctx, int32_t levels, double *out);

/* Compiles (as dp_compile) and uploads a netlist; the design keeps its whole
 * graph and per-net state resident in device memory (Sec. III). */
dp_status dp_design_load(dp_ctx *ctx, const char *netlist, size_t netlist_len, const char *library,
                         size_t library_len, dp_design **out);
/* Uploads an already compiled netlist (the compiled object is not consumed). */
dp_status dp_design_upload(dp_ctx *ctx, const dp_compiled *c, dp_design **out);
/* Loads (as dp_compiled_load) and uploads a compiled-netlist blob. */
dp_status dp_design_load_blob(dp_ctx *ctx, const void *blob, size_t len, dp_design **out);
void dp_design_free(dp_design *d);
dp_status dp_design_info(const dp_design *d, dp_info *info);

/* Startpoint SP and TR (Sec. III-A), binary32.  n_scen = 1: n_start values
 * each, analysed by the single-scenario path (float-float pairs, simulation,
 * hybrid).  n_scen > 1: the same as dp_set_inputs_batch.  SP must lie in
 * [0,1] and TR in [0,1]; values are not checked on the device path. */
dp_status dp_set_inputs(dp_design *d, const float *sp, const float *tr, int32_t n_scen, int on_device);

/* Switches the stream that later calls on this context queue their work on
 * (e.g. PyTorch's current stream, or a stream being captured into a graph). */
dp_status dp_set_stream(dp_ctx *ctx, void *cuda_stream);

/* Sizing delta: sets the input pin cap (fF) of n cells given by cell-line index
 * and updates the loads C_load of the nets they read (Eq. 1). Indices must be
 * in range (checked for host input only).  cells = NULL with n = n_cells sets
 * every cell's cap, in cell-line order. */
dp_status dp_set_pincap(dp_design *d, const int32_t *cells, const float *pincap, int32_t n, int on_device);

/* Pass 1 (Sec. III-B, Algorithm 2): SP and TR_model (Eq. 2) of every net, and the
 * model power (Eq. 1).  Needs dp_set_inputs. */
dp_status dp_propagate(dp_design *d, const dp_config *cfg);

/* Pass 2 and hybrid (Sec. III-C, III-D): Markov-chain startpoint vectors
 * (Philox4x32-10), bit-packed simulation of cfg->sim_words words per net,
 * PopCount toggle and ones counts, beta (Eq. 5), hybrid TR = beta TR_model and
 * the hybrid power.  Needs dp_propagate with the same tr_mode. */
dp_status dp_simulate(dp_design *d, const dp_config *cfg);

/* Total switching power (Eq. 1) in watts into watts[0] (host):
 * hybrid = 0 model TR, 1 hybrid TR.  Synchronises.  Batched inputs: one
 * value per scenario, watts[n_scen], model TR only. */
dp_status dp_total_power(dp_design *d, int hybrid, double *watts);

/* dp_total_power into host or device memory; with on_device = 1 the copy is
 * queued on the context stream without synchronising. */
dp_status dp_get_power(dp_design *d, int hybrid, double *watts, int on_device);

/* Sec. III-E: gradient of the power with respect to the startpoint SP
 * (grad_sp_in[n_start]), startpoint TR (grad_tr_in[n_start]), the input pin
 * cap of each cell (grad_pincap[n_cells], W/fF) and each net's load
 * (grad_cload[n_nets], W/fF).  Any output may be NULL.  cfg->grad_mode picks
 * the model (needs dp_propagate) or a hybrid objective (needs dp_simulate).
 * No atomics: results are bitwise reproducible. */
dp_status dp_backward(dp_design *d, const dp_config *cfg, float *grad_sp_in, float *grad_tr_in,
                      float *grad_pincap, float *grad_cload, int on_device);

/* Per-net results: SP, TR_model, beta, hybrid TR, toggle and ones counts.
 * Any output may be NULL; beta/tr_hyb/toggles/ones need dp_simulate.
 * Batched inputs: sp and tr as [n_nets][n_scen] (scenario innermost); the
 * simulation outputs must be NULL (DP_EUNSUPPORTED). */
dp_status dp_get_nets(dp_design *d, float *sp, float *tr, float *beta, float *tr_hyb, uint32_t *toggles,
                      uint32_t *ones, int on_device);

/* The whole hot path in one call: dp_propagate, dp_simulate, dp_backward and
 * both powers (watts[0] model, watts[1] hybrid; host, may be NULL), replayed
 * as one CUDA graph per (design, config).  Gradient outputs as dp_backward. */
dp_status dp_step(dp_design *d, const dp_config *cfg, float *grad_sp_in, float *grad_tr_in, float *grad_pincap,
                  float *grad_cload, double *watts, int on_device);

/* Device time in milliseconds of the last dp_step / dp_propagate / dp_simulate /
 * dp_backward per phase (CUDA events on the context stream; synchronises):
 * ms5[0] forward + model power, ms5[1] simulation levels (the bitwise cells;
 * in dp_step the startpoint generator runs beside the forward pass),
 * ms5[2] beta + hybrid power, ms5[3] backward, ms5[4] gradient outputs. */
dp_status dp_phase_times(dp_design *d, float *ms5);

/* ------------------ batched scenarios (S scenarios per launch) ------------------
 * Every per-scenario array is [rows][n_scen]: row-major with the scenario
 * innermost, rows in the orders above.  After dp_set_inputs_batch, the calls
 * dp_propagate, dp_total_power / dp_get_power, dp_backward and dp_get_nets
 * work on the batch; dp_simulate and dp_step return DP_EUNSUPPORTED (the
 * simulation and the hybrid objective run on single-scenario inputs).
 * Each cell's (P, P(net=0)) pair is evaluated in float-float and renormalised
 * as for one scenario; P is kept in float-float (P(net=0) re-derived as 1 - P);
 * the adjoint is binary32;
 * powers and scenario sums are FP64 in a fixed order (reproducible).  Calls
 * with device outputs neither allocate nor synchronise once a call with the
 * largest n_scen has been made, so they may be captured into a CUDA graph. */

/* Stages n_scen scenarios of startpoint SP and TR, sp[n_start][n_scen] and
 * tr[n_start][n_scen].  The first call with a larger n_scen allocates the
 * batch buffers (about (8 n_nets + 4 n_edges + 12 n_start) bytes per
 * scenario) and must not be made under stream capture (DP_ESTATE); a call
 * with a new n_scen outside capture also runs the launch-shape autotuner
 * (times every candidate shape of the forward and reverse kernels on the
 * staged inputs and keeps the fastest; synchronises).  The environment
 * variable DP_BATCH_SHAPE="bx,by[,bx2,by2]" fixes the shapes instead.
 * Every shape gives bitwise identical results. */
dp_status dp_set_inputs_batch(dp_design *d, const float *sp, const float *tr, int32_t n_scen, int on_device);

/* Shapes in use (bx threads over scenarios x by cells per block x v scenarios
 * per thread, v = 1 or 2; v = 2 applies to even n_scen) for the forward
 * (shape6[0..2]) and the reverse pass (shape6[3..5]), and the tuner's best
 * times in ms (ms2, may be NULL; 0 when fixed by the environment).  Every
 * shape gives bitwise the same results. */
dp_status dp_batch_tuning(const dp_design *d, int32_t *shape6, float *ms2);

/* Reverse pass of the model power (Sec. III-E, Eq. 7) for every scenario,
 * scaled by weights[n_scen] (NULL: all 1): the gradient of
 * sum_s weights[s] * P_s, i.e. the vector-Jacobian product an autograd
 * engine asks for.  weights live where the outputs live (on_device).
 * Outputs (any may be NULL): grad_sp_in and grad_tr_in [n_start][n_scen];
 * grad_pincap [n_cells][n_scen] and grad_cload [n_nets][n_scen], or, with
 * cap_reduce = 1, summed over the scenarios in FP64 into [n_cells] and
 * [n_nets] (the gradient with respect to caps shared by all scenarios).
 * Needs dp_propagate with the same tr_mode and cfg->grad_mode = 0
 * (DP_EUNSUPPORTED otherwise).  Single-scenario inputs: weights must be NULL
 * and the call is dp_backward. */
dp_status dp_backward_weighted(dp_design *d, const dp_config *cfg, const double *weights, int32_t cap_reduce,
                               float *grad_sp_in, float *grad_tr_in, float *grad_pincap, float *grad_cload,
                               int on_device);

/* One projected gradient-ascent step of Algorithm 4 on device arrays:
 * x[i] <- clip(x[i] + eta * g[i], 0, 1), in binary32 with the product and the
 * sum each rounded once.  Queued on the context stream; no synchronisation. */
dp_status dp_ascent_step(dp_ctx *ctx, float *x, const float *g, int64_t n, float eta);

/* P_virus of Eq. 3 for n_scen candidate inputs sp[n_start][n_scen]
 * (Algorithm 4, last steps): v0 = [sp >= 0.5] (compared in binary32),
 * v1 = not v0, two bitwise forward passes, and per scenario the sum of
 * C_load (fF, FP64, fixed order) over the nets whose values differ between
 * v0 and v1.  p_virus[n_scen]; v0[n_start][n_scen] as 0/1 bytes (may be NULL).
 * Works on any design state.  The first call with a larger n_scen allocates. */
dp_status dp_virus_eval(dp_design *d, const float *sp, int32_t n_scen, uint8_t *v0, double *p_virus, int on_device);

/* Gradient-weighted sizing score (Eq. 8) of every cell line, S = |dP/dP_sw| * P_sw,
 * with P_sw = K * alpha * C_load of the cell's output net (alpha = TR_model, or
 * the hybrid TR when cfg->grad_mode != 0), from the adjoint of the last
 * dp_backward / dp_step with the same config (DP_ESTATE otherwise).
 *   mode 0: dP/dP_sw read as the SP adjoint of the output net (global sensitivity);
 *   mode 1: the chain rule through Eq. 2, SP adjoint / (2 - 4 SP), |2 - 4 SP| >= 1e-6.
 * scores[n_cells] (may be NULL).  k > 0: the k highest-scoring cell lines, best
 * first, ties by cell index, into top_cells[k] and top_scores[k] (may be NULL);
 * found by a radix select on the device, the candidates ordered on the host
 * (synchronises).  Single-scenario inputs only. */
dp_status dp_sizing_scores(dp_design *d, const dp_config *cfg, int32_t mode, float *scores, int32_t k,
                           int32_t *top_cells, float *top_scores, int on_device);

/* Number of kernels the last dp_step launched: the kernel nodes of its CUDA
 * graph plus the output kernels queued after it (0 before the first dp_step). */
dp_status dp_step_kernels(const dp_design *d, int64_t *kernels);

/* Total switching power K * sum_n alpha_n * C_n with K = 1/2 Vdd^2 f 1e-15 and
 * alpha_n = tr[n] * (beta ? beta[n] : 1), from caller-owned device arrays
 * (tr, beta, cload: n binary32 values each; C in fF), written as one double
 * into the device pointer `watts`, asynchronously on `cuda_stream` (NULL:
 * the device's default stream).  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory - code running
 * inside a host framework that owns every device byte through its own pool,
 * or a service that plans its memory ahead and must not let a cudaMalloc
 * implicitly synchronise the device and stall the other streams.  It calls no
 * cudaMalloc, cudaFree or allocating routine: its scratch (one FP64 partial
 * per 8,192 nets) is a fixed 32 KB array in the library's device memory,
 * held by every GPU that loads the library until the process exits.
 * Limits and behaviour:
 *  - n <= 33,554,432 (4,096 partials); larger n returns DP_EUNSUPPORTED
 *    before any GPU work.  NULL tr/cload with n > 0, NULL watts, n < 0, a
 *    bad device or non-positive vdd/fclk return DP_EINVAL.
 *  - The first call on a device looks up the scratch array's device address
 *    (with that device made current) and caches it; make that first call
 *    before any stream capture.  The cached address belongs to the device's
 *    primary context: do not call this after cudaDeviceReset() of that device
 *    in the same process.
 *  - Every call shares the scratch and overwrites the partials it reads
 *    (nothing needs clearing); calls that overlap on the GPU (other streams,
 *    other threads) race on it and must be serialised by the caller.
 *  - The summation order is fixed, so results are reproducible.
 *  - DP_ECUDA comes only from this call's own runtime calls and launches: a
 *    launch error the caller left pending on the calling thread is neither
 *    reported as this call's result nor cleared.
 *  - There is no context, so dp_last_error() has no message for this call. */
dp_status dp_power_noalloc(int device, const float *tr, const float *beta, const float *cload, int64_t n,
                           double vdd, double fclk, double *watts, void *cuda_stream);

/* ------------------------------ request server ------------------------------
 * Several designs resident on one GPU; power and gradient requests of any of
 * them are served by continuous batching: a worker thread takes the requests
 * waiting for a design that has a free batch slot (up to max_batch, in arrival
 * order) and runs them as the scenarios of one batched pass on that slot's
 * own stream, so batches of different designs, and of the slots of one
 * design, overlap on the device, and requests that arrive while every slot of
 * their design is busy join its next batch.  A batch whose
 * requests all use the reference inputs (sizing deltas) skips the forward
 * pass: caps do not enter SP or TR, so it starts from the reference inputs'
 * forward state, computed once by dp_server_add_design.  A request's
 * results do not depend on the requests it shares a batch with: they are
 * bitwise the same alone and in any mix.  Model power and model gradient
 * (Eq. 1, Eq. 2, Eq. 7); no simulation.
 *
 * Each slot holds one CUDA stream.  The device has a fixed number of hardware
 * work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless the process sets it
 * before its first CUDA call, at most 32); streams beyond that share queues,
 * and a batch on a stream that shares a queue with a busy one waits behind
 * its work.  A process that holds many other streams, or creates servers one
 * after another, should set it to 32. */
typedef struct dp_server dp_server;

typedef struct {
    int32_t device;       /* CUDA device */
    int32_t max_batch;    /* requests per batch per design, 1..4096 (default 64) */
    size_t hbm_budget;    /* device bytes the server may hold for designs and their batch buffers;
                             0: 80 % of the free memory at creation */
    int32_t plain;        /* 1: no worker and no batching - dp_server_submit runs the request on the
                             calling thread and returns when it is done (the one-at-a-time loop) */
    dp_config analysis;   /* vdd, fclk, tr_mode; grad_mode must be 0 */
    int32_t slots_per_design;   /* batch slots per design, 1..8 (default 1; 0 also means 1; plain: 1).
                                   Each slot holds its own copy of the design's device state and batch
                                   buffers and its own stream, so batches of one design overlap (one
                                   batch's copies beside the next one's kernels); the HBM budget is
                                   charged for every slot */
} dp_server_config;

/* One request.  Every pointer is host memory borrowed until dp_server_wait
 * returns for it; page-locked buffers make the copies asynchronous. */
typedef struct {
    int32_t design;        /* id from dp_server_add_design */
    const float *sp;       /* n_start startpoint SP, or NULL for the design's reference inputs */
    const float *tr;       /* n_start startpoint TR (NULL exactly when sp is) */
    const int32_t *cells;  /* sizing delta: cell-line indices (may repeat: the last entry counts) */
    const float *pincap;   /* their new input pin caps (absolute values, fF) */
    int32_t n_delta;       /* entries in cells / pincap (0: the design's own caps) */
    int32_t want_grad;     /* 1: also the gradients below */
    double *power;         /* out: model power, W */
    float *grad_sp;        /* out (want_grad, may be NULL): dP/dSP_in [n_start] */
    float *grad_tr;        /* out (want_grad, may be NULL): dP/dTR_in [n_start] */
    float *grad_pincap;    /* out (want_grad, may be NULL): dP/dpincap [n_cells], W/fF */
} dp_request;

typedef struct {
    int64_t batches;          /* batches run */
    int64_t requests;         /* requests finished */
    int64_t max_batch_seen;   /* largest batch */
    size_t device_bytes;      /* device bytes charged against the budget */
    int32_t designs;          /* resident designs */
    double host_launch_s;     /* host seconds spent queuing batches (copies, graph launches) */
} dp_server_stats;

void dp_server_config_default(dp_server_config *cfg);
/* Creates a server (and its worker thread unless cfg->plain).  DP_EINVAL for a
 * bad max_batch, grad_mode != 0, or a tr_mode other than 0 and 1 (the lag-one
 * mode runs through dp_set_inputs_batch only). */
dp_status dp_server_create(const dp_server_config *cfg, dp_server **out);
/* Stops the worker after the batches in flight, frees every design. */
void dp_server_destroy(dp_server *srv);
const char *dp_server_last_error(const dp_server *srv);
/* Compiles and uploads a design, reserves its batch buffers for max_batch
 * requests, tunes its launch shapes once (on max_batch copies of the reference
 * inputs) and keeps them, and computes the reference inputs' forward state.  ref_sp / ref_tr (n_start each, may be NULL: 0.5 and
 * 0.25) are the inputs of requests that give none.  Admission: DP_ENOMEM when
 * the design would exceed the HBM budget. */
dp_status dp_server_add_design(dp_server *srv, const char *netlist, size_t netlist_len, const char *library,
                               size_t library_len, const float *ref_sp, const float *ref_tr, int32_t *id);
/* Sizes of a resident design; device_bytes = what it is charged. */
dp_status dp_server_design_info(dp_server *srv, int32_t id, dp_info *info);
/* Queues a request (validated first: DP_EINVAL) and returns its ticket without
 * waiting; thread-safe. */
dp_status dp_server_submit(dp_server *srv, const dp_request *req, uint64_t *ticket);
/* Queues n requests at once (reqs[n], their tickets into tickets[n]): all are validated
 * first, and if one is invalid nothing is queued and its status (DP_EINVAL) is returned
 * with its index in the message; otherwise they enter their designs' queues in order,
 * under one lock, before the worker is woken, so a burst forms full batches.  A plain
 * server runs them one after another.  Thread-safe. */
dp_status dp_server_submit_many(dp_server *srv, const dp_request *reqs, int32_t n, uint64_t *tickets);
/* Waits until the request is done (timeout_s > 0: at most that long, then
 * DP_ETIMEOUT and the ticket stays valid), reports its latency from submission
 * to completion in ms and releases the ticket. */
dp_status dp_server_wait(dp_server *srv, uint64_t ticket, double timeout_s, double *latency_ms);
dp_status dp_server_get_stats(dp_server *srv, dp_server_stats *stats);

#ifdef __cplusplus
}
#endif
#endif /* DIFFPOWER_H */
