// Internal state of the C-ABI objects, shared by the translation units that
// implement the entry points (capi.cu: single scenario; capi_batch.cu:
// batched scenarios, power-virus evaluation).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "diffpower.h"
#include "kernels.h"

struct dp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int clock_khz = 0;
    int *d_err = nullptr;   // device error word: a bounded wait gave up
    std::string err;
};

// Buffers of the batched path (S scenarios, scenario innermost).  They are
// sized for `cap` scenarios and reallocated only when a larger S arrives.
struct dp_batch {
    int64_t S = 0;                 // scenarios of the staged inputs
    int64_t cap = 0;               // scenarios the buffers hold
    dp::BatchBufs b{};
    double *weights = nullptr;     // [cap] staging of host weights
    float *stage = nullptr;        // [max(n_nets, n_cells) * cap] staging of host outputs (lazy)
    std::vector<void *> allocs;    // freed together on reallocation
    size_t bytes = 0;
    bool fwd_valid = false;
    int fwd_tr_mode = -1;
    dp::BatchShape fwd_shape{128, 1}, bwd_shape{128, 1};
    int64_t tuned_S = 0;           // S the shapes were tuned for (0: not tuned)
    bool shapes_locked = false;    // keep the shapes whatever S comes (a server fixes them once)
    float tune_ms[2] = {0.f, 0.f}; // best forward / backward time seen by the tuner
    // power-virus evaluation (Eq. 3): words [n_nets * 2 ceil(S/64)], partials, sums, staging
    int64_t vcap = 0;
    uint64_t *vwords = nullptr;
    double *vpart = nullptr, *vout = nullptr;
    float *vsp = nullptr;
    uint8_t *vv0 = nullptr;
    std::vector<void *> vallocs;
    size_t vbytes = 0;
};

struct dp_design {
    dp_ctx *ctx = nullptr;
    dp::DevDesign d{};
    dp::OpTable ops{};
    std::vector<int32_t> lvl_ptr;
    int64_t n_edges = 0;
    int32_t n_ops = 0;
    std::vector<void *> allocs;
    size_t bytes = 0;
    int words_T = 0;
    // output staging for host outputs
    float *st_gsp = nullptr, *st_gtr = nullptr, *st_gpin = nullptr, *st_gcl = nullptr;
    // state
    bool inputs_set = false;
    bool batched = false;          // the staged inputs are a batch (dp_set_inputs_batch)
    bool fwd_valid = false;
    int fwd_tr_mode = -1;
    bool sim_valid = false;
    bool bwd_valid = false;        // gnet holds the adjoint of the current state
    int bwd_grad_mode = -1;
    // staging of host sizing deltas (dp_set_pincap): grown on demand, never shrunk; pc_done is
    // recorded after the kernels that read it, so a later call waits for them on any stream
    int32_t *pc_cells = nullptr;
    float *pc_caps = nullptr;
    int64_t pc_cap = 0;
    cudaEvent_t pc_done = nullptr;
    // sizing-score scratch (lazy): scores [n_cells], candidates [n_cells], histogram [256] + count
    float *sc_scores = nullptr;
    int32_t *sc_idx = nullptr;
    unsigned *sc_hist = nullptr;
    dp_batch batch;
    // graph of the whole step for one config
    cudaGraphExec_t graph = nullptr;
    dp_config graph_cfg{};
    cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // the step's output copies: a side stream that starts them when the gradient branch of
    // the step graph is done (ev_grads, recorded by the graph), and their completion
    cudaStream_t out_stream = nullptr;
    cudaEvent_t ev_grads = nullptr, ev_copies = nullptr;
    int grid[4] = {0, 0, 0, 0};   // persistent grids: forward, simulation, backward, wide simulation
    int flow_grid[2] = {0, 0};     // dataflow grids: forward, simulation
    int block_threads = 0;         // > 0: the design fits the single-block passes, with this many threads
    dp::ClusterMap cl;             // the single-cluster passes (cl.threads > 0: the design uses them)
    // launch-shape tuning (defaults, overridable by DP_FLOW_BLOCKS / DP_FLOW_SLEEP for sweeps)
    int flow_blocks_per_sm = 2;
    unsigned flow_sleep = 0;
    int64_t graph_kernels = 0;
    int64_t step_kernels = 0;
    // phase boundaries: start, forward, simulation levels, hybrid + power, backward, outputs
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool ev_valid[6] = {false, false, false, false, false, false};
};

namespace dpi {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

dp_status set_err(dp_ctx *c, dp_status s, const std::string &m);
dp_status cuda_err(dp_ctx *c, cudaError_t e, const char *where);
dp_status launch_check(dp_ctx *c, const char *where);
// Reads and clears the device error word (synchronises the stream).
dp_status check_device_error(dp_ctx *c);
// cudaMalloc of `bytes` with the DP_FAULT=alloc:N injection; the pointer is
// appended to *list and its size added to *total.
dp_status alloc_into(dp_ctx *c, void **p, size_t bytes, std::vector<void *> *list, size_t *total);
double power_K(const dp_config &c);
dp_status check_cfg(dp_ctx *ctx, const dp_config *c);
// true when the stream is being captured into a CUDA graph
bool capturing(cudaStream_t s);
// frees the batched buffers (the caller has synchronised)
void free_batch(dp_design *D);
// batched halves of dp_propagate, dp_get_power and dp_get_nets (capi_batch.cu)
dp_status batch_propagate(dp_design *D, const dp_config &c);
dp_status batch_get_power(dp_design *D, int hybrid, double *watts, int on_device);
dp_status batch_get_nets(dp_design *D, float *sp, float *tr, int on_device);
// batch buffers for S scenarios plus the host-output staging (synchronises; not under capture)
dp_status batch_reserve(dp_design *D, int64_t S);
// runs the launch-shape tuner on the staged batch of B.S scenarios, then locks the shapes
dp_status batch_tune_and_lock(dp_design *D);

template <class T>
dp_status dalloc(dp_design *D, T **p, size_t count) {
    void *v = nullptr;
    dp_status s = alloc_into(D->ctx, &v, sizeof(T) * (count ? count : 1), &D->allocs, &D->bytes);
    *p = static_cast<T *>(v);
    return s;
}

}  // namespace dpi
