// C-ABI of libdiffpower.so: contexts, resident designs, and the call sequence
// of the hot path (load, set inputs, propagate, simulate, power, backward).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "compiled.h"

namespace dpi {

// Host-side fault injection for tests: DP_FAULT=alloc:N fails the N-th
// device allocation of the process with DP_ENOMEM (no GPU fault involved).
static long g_alloc_count = 0;
static long fault_alloc_at() {
    static long at = -2;
    if (at == -2) {
        at = -1;
        const char *f = std::getenv("DP_FAULT");
        if (f && std::strncmp(f, "alloc:", 6) == 0) at = std::atol(f + 6);
    }
    return at;
}

dp_status set_err(dp_ctx *c, dp_status s, const std::string &m) {
    if (c) c->err = m;
    return s;
}

dp_status cuda_err(dp_ctx *c, cudaError_t e, const char *where) {
    if (e == cudaSuccess) return DP_OK;
    dp_status s = e == cudaErrorMemoryAllocation ? DP_ENOMEM : DP_ECUDA;
    return set_err(c, s, std::string(where) + ": " + cudaGetErrorString(e));
}

dp_status launch_check(dp_ctx *c, const char *where) { return cuda_err(c, cudaGetLastError(), where); }

dp_status check_device_error(dp_ctx *c) {
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "device error word");
    if (v != 0) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        cudaStreamSynchronize(c->stream);
        return set_err(c, DP_ETIMEOUT, "a bounded device wait gave up (grid barrier timeout)");
    }
    return DP_OK;
}

dp_status alloc_into(dp_ctx *c, void **p, size_t bytes, std::vector<void *> *list, size_t *total) {
    *p = nullptr;
    long n = ++g_alloc_count;
    if (fault_alloc_at() == n) return set_err(c, DP_ENOMEM, "injected allocation failure (DP_FAULT)");
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, bytes ? bytes : 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_err(c, e, "cudaMalloc");
    }
    list->push_back(v);
    *total += bytes;
    *p = v;
    return DP_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

double power_K(const dp_config &c) { return 0.5 * c.vdd * c.vdd * c.fclk * 1e-15; }

dp_status check_cfg(dp_ctx *ctx, const dp_config *c) {
    if (!c) return set_err(ctx, DP_EINVAL, "NULL config");
    if (!(c->vdd > 0) || !(c->fclk > 0) || !std::isfinite(c->vdd) || !std::isfinite(c->fclk))
        return set_err(ctx, DP_EINVAL, "vdd and fclk must be positive");
    if (!(c->beta_min > 0) || !(c->beta_max >= c->beta_min) || !std::isfinite(c->beta_max))
        return set_err(ctx, DP_EINVAL, "need 0 < beta_min <= beta_max");
    if (c->tr_mode < 0 || c->tr_mode > 2) return set_err(ctx, DP_EINVAL, "tr_mode must be 0, 1 or 2");
    if (c->grad_mode < 0 || c->grad_mode > 2) return set_err(ctx, DP_EINVAL, "grad_mode must be 0, 1 or 2");
    if (c->sim_words < 2 || c->sim_words > 4096) return set_err(ctx, DP_EINVAL, "sim_words must be in [2, 4096]");
    if (c->schedule < 0 || c->schedule > 3) return set_err(ctx, DP_EINVAL, "schedule must be 0, 1, 2 or 3");
    return DP_OK;
}

}  // namespace dpi

using namespace dpi;

namespace {

void free_design(dp_design *D) {
    if (!D) return;
    DeviceGuard g(D->ctx ? D->ctx->device : 0);
    if (D->ctx) cudaStreamSynchronize(D->ctx->stream);
    if (D->graph) cudaGraphExecDestroy(D->graph);
    if (D->cap_stream) cudaStreamDestroy(D->cap_stream);
    if (D->cap_stream2) cudaStreamDestroy(D->cap_stream2);
    if (D->fork) cudaEventDestroy(D->fork);
    if (D->join) cudaEventDestroy(D->join);
    if (D->out_stream) cudaStreamDestroy(D->out_stream);
    if (D->ev_grads) cudaEventDestroy(D->ev_grads);
    if (D->ev_copies) cudaEventDestroy(D->ev_copies);
    for (auto &e : D->ev)
        if (e) cudaEventDestroy(e);
    free_batch(D);
    if (D->pc_done) cudaEventDestroy(D->pc_done);
    if (D->pc_cells) cudaFree(D->pc_cells);
    if (D->pc_caps) cudaFree(D->pc_caps);
    for (void *p : D->allocs) cudaFree(p);
    delete D;
}

// Staging for n host sizing-delta entries: grows (with headroom) only when n exceeds what is
// held; the old buffers are freed after the stream that last read them is done.
dp_status reserve_pincap_staging(dp_design *D, int64_t n) {
    dp_ctx *c = D->ctx;
    if (!D->pc_done) {
        cudaError_t e = cudaEventCreateWithFlags(&D->pc_done, cudaEventDisableTiming);
        if (e != cudaSuccess) { D->pc_done = nullptr; return cuda_err(c, e, "dp_set_pincap"); }
    }
    if (n <= D->pc_cap) return DP_OK;
    int64_t want = std::max<int64_t>(n, std::max<int64_t>(1024, 2 * D->pc_cap));
    want = std::min<int64_t>(want, std::max<int64_t>(n, D->d.n_cells));
    if (D->pc_cells || D->pc_caps) {
        cudaEventSynchronize(D->pc_done);
        cudaFree(D->pc_cells);
        cudaFree(D->pc_caps);
        D->bytes -= (sizeof(int32_t) + sizeof(float)) * (size_t)D->pc_cap;
        D->pc_cells = nullptr;
        D->pc_caps = nullptr;
        D->pc_cap = 0;
    }
    std::vector<void *> got;
    size_t bytes = 0;
    void *a = nullptr, *b = nullptr;
    dp_status s = alloc_into(c, &a, sizeof(int32_t) * (size_t)want, &got, &bytes);
    if (s == DP_OK) s = alloc_into(c, &b, sizeof(float) * (size_t)want, &got, &bytes);
    if (s != DP_OK) {
        for (void *p : got) cudaFree(p);
        return s;
    }
    D->pc_cells = static_cast<int32_t *>(a);
    D->pc_caps = static_cast<float *>(b);
    D->pc_cap = want;
    D->bytes += bytes;
    return DP_OK;
}

dp_status ensure_words(dp_design *D, int T) {
    if (D->words_T >= T && D->d.words) return DP_OK;
    if (D->d.words) {
        cudaStreamSynchronize(D->ctx->stream);
        for (auto it = D->allocs.begin(); it != D->allocs.end(); ++it)
            if (*it == D->d.words) {
                cudaFree(*it);
                D->allocs.erase(it);
                D->bytes -= sizeof(uint64_t) * (size_t)D->d.n_nets * (size_t)D->words_T;
                break;
            }
        D->d.words = nullptr;
        D->words_T = 0;
        if (D->graph) { cudaGraphExecDestroy(D->graph); D->graph = nullptr; }
    }
    dp_status s = dalloc(D, &D->d.words, (size_t)D->d.n_nets * (size_t)T);
    if (s == DP_OK) D->words_T = T;
    if (s == DP_OK && !D->d.simdone) {   // flags of the dataflow simulation: pass number 0 = none
        s = dalloc(D, &D->d.simdone, (size_t)D->d.n_cells);
        if (s == DP_OK) {
            const cudaError_t e = cudaMemsetAsync(D->d.simdone, 0, sizeof(unsigned) * (size_t)D->d.n_cells,
                                                  D->ctx->stream);
            if (e != cudaSuccess) s = cuda_err(D->ctx, e, "cudaMemsetAsync");
        }
    }
    return s;
}

// The step graph's capture and branch streams and the side stream of its output copies,
// created by the first dp_step.  A design that never steps (a server slot, a batched or
// per-pass caller) holds no stream of its own: streams beyond the device's hardware work
// queues share queues, and a stream sharing a queue with a busy one waits behind its work.
dp_status ensure_step_streams(dp_design *D) {
    cudaError_t e = cudaSuccess;
    for (cudaStream_t *p : {&D->cap_stream, &D->cap_stream2, &D->out_stream})
        if (!*p && e == cudaSuccess) e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
    return e == cudaSuccess ? DP_OK : cuda_err(D->ctx, e, "step streams");
}

dp_status ensure_stage(dp_design *D) {
    if (D->st_gsp) return DP_OK;
    dp_status s;
    if ((s = dalloc(D, &D->st_gsp, (size_t)D->d.n_start)) != DP_OK) return s;
    if ((s = dalloc(D, &D->st_gtr, (size_t)D->d.n_start)) != DP_OK) return s;
    if ((s = dalloc(D, &D->st_gpin, (size_t)D->d.n_cells)) != DP_OK) return s;
    return dalloc(D, &D->st_gcl, (size_t)D->d.n_nets);
}

void rec(dp_design *D, int i, cudaStream_t s) {
    cudaEventRecord(D->ev[i], s);
    D->ev_valid[i] = true;
}

// ---- the phases, queued on stream s (also used under graph capture) ----
bool persistent(const dp_design *D, const dp_config &c, int which) {
    return c.schedule != 1 && D->grid[which] > 0 && D->d.n_levels > 0;
}
// the forward and reverse passes of a small design in one block (schedule 0)
bool small_pass(const dp_design *D, const dp_config &c) { return c.schedule == 0 && D->block_threads > 0; }
// ... and of a mid-size design in one thread-block cluster (schedule 0)
bool cluster_pass(const dp_design *D, const dp_config &c) { return c.schedule == 0 && D->cl.threads > 0; }
bool dataflow(const dp_design *D, const dp_config &c, int which) {
    return c.schedule == 3 && D->flow_grid[which] > 0 && D->d.n_levels > 0;
}

// each q_* returns the first launch error (a cooperative launch reports it directly)
// The forward pass and the model power.  ready (may be null) is recorded on s just before
// the first forward kernel: a branch forked there becomes ready with that kernel.
cudaError_t q_forward(dp_design *D, const dp_config &c, cudaStream_t s, cudaEvent_t ready = nullptr) {
    if (small_pass(D, c)) {   // the kernel advances the pass counter itself
        if (ready) cudaEventRecord(ready, s);
        cudaError_t e = dp::launch_fwd_block(D->d, D->ops, c.tr_mode, D->block_threads, s);
        if (e != cudaSuccess) return e;
        dp::launch_power(D->d, false, power_K(c), 0, s);
        return cudaGetLastError();
    }
    dp::launch_bump(D->d.epoch, s);   // new parity for the stored (P, Q) pairs
    if (cluster_pass(D, c)) {
        if (ready) cudaEventRecord(ready, s);
        cudaError_t e = dp::launch_fwd_cluster(D->d, D->ops, D->cl, c.tr_mode, s);
        if (e != cudaSuccess) return e;
    } else if (dataflow(D, c, 0)) {
        if (ready) cudaEventRecord(ready, s);
        cudaError_t e = dp::launch_fwd_flow(D->d, D->ops, c.tr_mode, D->flow_grid[0], D->flow_sleep, s);
        if (e != cudaSuccess) return e;
    } else if (persistent(D, c, 0)) {
        cudaError_t e = dp::launch_fwd_persist(D->d, D->ops, c.tr_mode, D->grid[0], s, ready);
        if (e != cudaSuccess) return e;
    } else {
        if (ready) cudaEventRecord(ready, s);
        dp::launch_init_start(D->d, c.tr_mode, s);
        for (int l = 1; l <= D->d.n_levels; l++)
            dp::launch_fwd_level(D->d, D->ops, D->lvl_ptr[l - 1], D->lvl_ptr[l], s);
    }
    dp::launch_power(D->d, false, power_K(c), 0, s);
    return cudaGetLastError();
}

// the startpoint generator alone (needs only the inputs, not the forward pass)
void q_sim_start(dp_design *D, const dp_config &c, cudaStream_t s) {
    dp::launch_sim_start(D->d, c.sim_words, c.seed, s);
}

// the simulation levels, beta and the hybrid power (after the generator and the forward pass)
cudaError_t q_sim_levels(dp_design *D, const dp_config &c, cudaStream_t s) {
    if (dataflow(D, c, 1) && dp::wide_ok(c.sim_words) && D->d.simdone) {
        cudaError_t e = dp::launch_sim_flow(D->d, D->ops, c.sim_words, D->flow_grid[1], s);
        if (e != cudaSuccess) return e;
    } else if (persistent(D, c, 3) && dp::wide_ok(c.sim_words)) {
        cudaError_t e = dp::launch_sim_wide(D->d, D->ops, c.sim_words, D->grid[3], s);
        if (e != cudaSuccess) return e;
    } else if (persistent(D, c, 1)) {
        cudaError_t e = dp::launch_sim_persist(D->d, D->ops, c.sim_words, D->grid[1], s);
        if (e != cudaSuccess) return e;
    } else {
        for (int l = 1; l <= D->d.n_levels; l++)
            dp::launch_sim_level(D->d, D->ops, D->lvl_ptr[l - 1], D->lvl_ptr[l], c.sim_words, s);
    }
    return cudaGetLastError();
}

// beta, hybrid TR and the hybrid power (after the simulation levels)
cudaError_t q_hybrid(dp_design *D, const dp_config &c, cudaStream_t s) {
    dp::launch_hybrid(D->d, c.sim_words, c.tr_mode, c.beta_min, c.beta_max, s);
    dp::launch_power(D->d, true, power_K(c), 1, s);
    return cudaGetLastError();
}

// beside: other kernels run beside this pass (the step's gradient outputs), so its grid-wide
// form leaves them room on the SMs
cudaError_t q_backward(dp_design *D, const dp_config &c, float *gsp, cudaStream_t s, bool beside = false) {
    const float K = (float)power_K(c);
    if (small_pass(D, c))
        return dp::launch_bwd_block(D->d, D->ops, c.grad_mode, c.tr_mode, K, gsp, D->n_edges, D->block_threads, s);
    if (cluster_pass(D, c))
        return dp::launch_bwd_cluster(D->d, D->ops, D->cl, c.grad_mode, c.tr_mode, K, gsp, s);
    if (persistent(D, c, 2))
        return dp::launch_bwd_persist(D->d, D->ops, c.grad_mode, c.tr_mode, K, gsp, D->grid[2], !beside, s);
    for (int l = D->d.n_levels; l >= 1; l--)
        dp::launch_bwd_level(D->d, D->ops, D->lvl_ptr[l - 1], D->lvl_ptr[l], c.grad_mode, K, s);
    dp::launch_bwd_start(D->d, c.grad_mode, c.tr_mode, K, gsp, s);
    return cudaGetLastError();
}

// gradient outputs (user order) into device pointers, staged when the caller's buffers are host memory
dp_status q_outputs(dp_design *D, const dp_config &c, float *gsp, float *gtr, float *gpin, float *gcl, int on_device,
                    bool gsp_done) {
    cudaStream_t s = D->ctx->stream;
    const bool hyb = c.grad_mode != 0;
    if (on_device) {
        if (gsp && !gsp_done && D->d.n_start)
            cudaMemcpyAsync(gsp, D->d.gnet, sizeof(float) * (size_t)D->d.n_start, cudaMemcpyDeviceToDevice, s);
        dp::launch_cap_grads(D->d, D->ops, hyb, c.tr_mode, power_K(c), gcl, gpin, gtr, s);
        return launch_check(D->ctx, "gradient outputs");
    }
    dp_status st = ensure_stage(D);
    if (st != DP_OK) return st;
    dp::launch_cap_grads(D->d, D->ops, hyb, c.tr_mode, power_K(c), gcl ? D->st_gcl : nullptr,
                         gpin ? D->st_gpin : nullptr, gtr ? D->st_gtr : nullptr, s);
    if ((st = launch_check(D->ctx, "gradient outputs")) != DP_OK) return st;
    cudaError_t e = cudaSuccess;
    if (gsp && D->d.n_start)
        e = cudaMemcpyAsync(gsp, D->d.gnet, sizeof(float) * (size_t)D->d.n_start, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && gtr && D->d.n_start)
        e = cudaMemcpyAsync(gtr, D->st_gtr, sizeof(float) * (size_t)D->d.n_start, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && gpin && D->d.n_cells)
        e = cudaMemcpyAsync(gpin, D->st_gpin, sizeof(float) * (size_t)D->d.n_cells, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && gcl && D->d.n_nets)
        e = cudaMemcpyAsync(gcl, D->st_gcl, sizeof(float) * (size_t)D->d.n_nets, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "gradient copy");
    return check_device_error(D->ctx);
}

// the step's outputs from its staging buffers (and the startpoint adjoints) into the
// caller's buffers, and both powers into watts (host); host buffers are complete on
// return, after one synchronisation
dp_status q_step_copies(dp_design *D, float *gsp, float *gtr, float *gpin, float *gcl, double *watts,
                        int on_device) {
    cudaStream_t s = D->ctx->stream, o = D->out_stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    // the staged gradients go out on the side stream while the backward pass still runs
    // (the graph records ev_grads when its gradient branch is done); the stream joins
    // back before anything else is queued on s, so the next step cannot overwrite the
    // staging buffers under these copies
    const bool side = (gtr && D->d.n_start) || (gpin && D->d.n_cells) || (gcl && D->d.n_nets);
    if (side) e = cudaStreamWaitEvent(o, D->ev_grads, 0);
    if (e == cudaSuccess && gtr && D->d.n_start)
        e = cudaMemcpyAsync(gtr, D->st_gtr, sizeof(float) * (size_t)D->d.n_start, kind, o);
    if (e == cudaSuccess && gpin && D->d.n_cells)
        e = cudaMemcpyAsync(gpin, D->st_gpin, sizeof(float) * (size_t)D->d.n_cells, kind, o);
    if (e == cudaSuccess && gcl && D->d.n_nets)
        e = cudaMemcpyAsync(gcl, D->st_gcl, sizeof(float) * (size_t)D->d.n_nets, kind, o);
    if (e == cudaSuccess && side) e = cudaEventRecord(D->ev_copies, o);
    if (e == cudaSuccess && gsp && D->d.n_start)
        e = cudaMemcpyAsync(gsp, D->d.gnet, sizeof(float) * (size_t)D->d.n_start, kind, s);
    if (e == cudaSuccess && side) e = cudaStreamWaitEvent(s, D->ev_copies, 0);
    if (e == cudaSuccess && watts) e = cudaMemcpyAsync(watts, D->d.power, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    rec(D, 5, s);   // the outputs phase: these copies (the gradient kernels ran beside the backward pass)
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "dp_step outputs");
    if (on_device && !watts) return DP_OK;
    return check_device_error(D->ctx);   // synchronises the stream
}

}  // namespace

extern "C" {

void dp_config_default(dp_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->vdd = 0.8;
    c->fclk = 1e9;
    c->beta_min = 0.1f;
    c->beta_max = 10.f;
    c->tr_mode = 0;
    c->grad_mode = 1;
    c->sim_words = 64;
    c->schedule = 0;
    c->seed = 42;
}

const char *dp_last_error(const dp_ctx *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

dp_status dp_create(int device, void *cuda_stream, dp_ctx **out) {
    if (!out) return DP_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return DP_ECUDA;
    }
    if (device < 0 || device >= n) return DP_EINVAL;
    dp_ctx *c = new (std::nothrow) dp_ctx();
    if (!c) return DP_ENOMEM;
    c->device = device;
    DeviceGuard g(device);
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->own_stream = false;
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->clock_khz, cudaDevAttrClockRate, device) != cudaSuccess ||
        cudaMalloc((void **)&c->d_err, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        delete c;
        return DP_ECUDA;
    }
    *out = c;
    return DP_OK;
}

void dp_destroy(dp_ctx *c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->d_err) cudaFree(c->d_err);
    delete c;
}

dp_status dp_sync(dp_ctx *c) {
    if (!c) return DP_EINVAL;
    DeviceGuard g(c->device);
    dp_status s = cuda_err(c, cudaStreamSynchronize(c->stream), "dp_sync");
    return s == DP_OK ? check_device_error(c) : s;
}

dp_status dp_set_stream(dp_ctx *c, void *cuda_stream) {
    if (!c) return DP_EINVAL;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return DP_OK;
}

dp_status dp_selftest_wait(dp_ctx *c, double seconds) {
    if (!c || !(seconds > 0) || seconds > 60) return set_err(c, DP_EINVAL, "seconds must be in (0, 60]");
    DeviceGuard g(c->device);
    unsigned *gs = nullptr;
    cudaError_t e = cudaMalloc((void **)&gs, 128);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_selftest_wait");
    const long long limit = (long long)(seconds * (double)c->clock_khz * 1e3);
    e = dp::launch_wait_selftest(gs, c->d_err, limit, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(gs);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_selftest_wait");
    return check_device_error(c);
}

namespace {
__global__ void k_zero_threads() {}

struct ProbeBufs {
    float *buf = nullptr;
    unsigned *bar = nullptr;
    uint32_t *next = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~ProbeBufs() {
        cudaFree(buf);
        cudaFree(bar);
        cudaFree(next);
        cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};
}  // namespace

dp_status dp_probe_latency(dp_ctx *c, int32_t levels, double *out) {
    if (!c || !out || levels < 16 || levels > 20000)
        return set_err(c, DP_EINVAL, "dp_probe_latency: levels must be in [16, 20000]");
    DeviceGuard g(c->device);
    const int grid = c->sm_count, max_threads = dp::kPersistThreads;
    const int M = 65536, stride = 32;   // chain entries, one per 128-byte line: 8 MB, resident in L2
    ProbeBufs p;
    cudaError_t e = cudaMalloc((void **)&p.buf, sizeof(float) * 2 * (size_t)grid * max_threads);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p.bar, sizeof(unsigned) * 32 * 3 * (size_t)levels);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p.next, sizeof(uint32_t) * (size_t)M * stride);
    if (e == cudaSuccess) e = cudaMalloc((void **)&p.sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&p.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&p.e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.buf, 0, sizeof(float) * 2 * (size_t)grid * max_threads, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_probe_latency");
    {
        // one cycle through all M entries (Sattolo's shuffle, SplitMix64 draws)
        std::vector<uint32_t> perm(M), host((size_t)M * stride, 0u);
        for (int i = 0; i < M; i++) perm[i] = (uint32_t)i;
        uint64_t x = 0x5EEDu;
        for (int i = M - 1; i > 0; i--) {
            uint64_t z = (x += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            std::swap(perm[i], perm[(size_t)(z % (uint64_t)i)]);
        }
        for (int i = 0; i < M; i++) host[(size_t)perm[i] * stride] = perm[(i + 1) % M] * (uint32_t)stride;
        e = cudaMemcpy(p.next, host.data(), sizeof(uint32_t) * host.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err(c, e, "dp_probe_latency");
    }
    float ms = 0.f;
    // milliseconds of one probe launch, its barrier counters zeroed outside the timed region
    auto timed = [&](int kind, int n, int threads) -> dp_status {
        cudaError_t le = cudaSuccess;
        if (kind != 2) le = cudaMemsetAsync(p.bar, 0, sizeof(unsigned) * 32 * (size_t)n, c->stream);   // n <= 3 levels
        if (le == cudaSuccess) le = cudaEventRecord(p.e0, c->stream);
        if (le == cudaSuccess)
            le = kind == 2 ? dp::launch_probe_chase(p.next, n, p.sink, c->stream)
                           : dp::launch_probe_levels(p.buf, n, kind, grid, threads, p.bar, c->d_err, c->stream);
        if (le == cudaSuccess) le = cudaEventRecord(p.e1, c->stream);
        if (le == cudaSuccess) le = cudaEventSynchronize(p.e1);
        if (le == cudaSuccess) le = cudaEventElapsedTime(&ms, p.e0, p.e1);
        if (le != cudaSuccess) return cuda_err(c, le, "dp_probe_latency");
        return check_device_error(c);
    };
    // microseconds per unit from launches of n and 3n units (launch costs cancel)
    auto per_unit = [&](int kind, int n, int threads, double *r) -> dp_status {
        dp_status s = timed(kind, n, threads);   // warm-up
        if (s != DP_OK) return s;
        if ((s = timed(kind, n, threads)) != DP_OK) return s;
        const double t1 = ms;
        if ((s = timed(kind, 3 * n, threads)) != DP_OK) return s;
        *r = 1e3 * ((double)ms - t1) / (2.0 * n);
        return DP_OK;
    };
    dp_status s = DP_OK;
    if (s == DP_OK) s = per_unit(0, levels, dp::kFwdThreads, &out[0]);
    if (s == DP_OK) s = per_unit(1, levels, dp::kFwdThreads, &out[1]);
    if (s == DP_OK) s = per_unit(0, levels, dp::kPersistThreads, &out[2]);
    if (s == DP_OK) s = per_unit(1, levels, dp::kPersistThreads, &out[3]);
    if (s == DP_OK) s = timed(2, M, 1);   // the first pass brings the chain into L2
    if (s == DP_OK) s = per_unit(2, 8 * levels, 1, &out[4]);
    out[5] = (double)grid;
    return s;
}

dp_status dp_selftest_pending_error(int action, int32_t *pending) {
    if (action < 0 || action > 2) return DP_EINVAL;
    if (action == 1) k_zero_threads<<<1, 0>>>();   // invalid configuration, rejected on the host
    const cudaError_t e = action == 2 ? cudaGetLastError() : cudaPeekAtLastError();
    if (pending) *pending = (int32_t)e;
    return DP_OK;
}

dp_status dp_design_upload(dp_ctx *ctx, const dp_compiled *cp, dp_design **out) {
    if (!ctx || !cp || !out) return set_err(ctx, DP_EINVAL, "NULL argument");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    dp_design *D = new (std::nothrow) dp_design();
    if (!D) return set_err(ctx, DP_ENOMEM, "out of memory");
    D->ctx = ctx;
    auto &d = D->d;
    d.n_nets = cp->n_nets;
    d.n_start = cp->n_start;
    d.n_cells = cp->n_cells;
    d.n_levels = cp->n_levels;
    D->n_edges = cp->n_edges;
    D->n_ops = cp->n_ops;
    D->lvl_ptr = cp->lvl_ptr;
    for (int i = 0; i < 256; i++) {
        const uint32_t k = cp->op_arity[i], tt = cp->op_tt[i];
        uint32_t lut = 0;
        if (k <= 3)
            for (uint32_t m = 0; m < 8; m++) lut |= ((tt >> (m & ((1u << k) - 1u))) & 1u) << m;
        D->ops.e[i] = tt | (k << 16) | (lut << 24);
    }
    const size_t nn = (size_t)d.n_nets, nc = (size_t)d.n_cells, ns = (size_t)d.n_start;
    dp_status s = DP_OK;
    uint4 *fanin = nullptr;
    int32_t *fptr = nullptr, *fedge = nullptr, *nou = nullptr, *cou = nullptr, *efpos = nullptr, *lvl = nullptr;
    int32_t *chunks = nullptr;
    // level-aligned chunks of 32: level 0 = startpoints, then each level of cells
    std::vector<int32_t> chunk_ptr((size_t)cp->n_levels + 2, 0);
    chunk_ptr[1] = (int32_t)((cp->n_start + 31) / 32);
    for (int l = 1; l <= cp->n_levels; l++)
        chunk_ptr[l + 1] = chunk_ptr[l] + (cp->lvl_ptr[l] - cp->lvl_ptr[l - 1] + 31) / 32;
    // nets by death level: the highest level of a cell reading the net, else the net's own level
    std::vector<int32_t> dead_ptr((size_t)cp->n_levels + 2, 0), dead_net((size_t)cp->n_nets);
    {
        std::vector<int32_t> death((size_t)cp->n_nets, 0);
        for (int l = 1; l <= cp->n_levels; l++)
            for (int32_t c = cp->lvl_ptr[l - 1]; c < cp->lvl_ptr[l]; c++) {
                death[(size_t)(cp->n_start + c)] = l;
                const uint32_t *r = &cp->fanin[4 * (size_t)c];
                const int k = cp->op_arity[r[0] >> 24];
                for (int j = 0; j < k; j++) {
                    const uint32_t n = j == 0 ? (r[0] & dp::kNetMask) : r[j];
                    death[n] = std::max(death[n], l);
                }
            }
        for (int32_t d : death) dead_ptr[(size_t)d + 1]++;
        for (size_t l = 1; l < dead_ptr.size(); l++) dead_ptr[l] += dead_ptr[l - 1];
        std::vector<int32_t> at(dead_ptr.begin(), dead_ptr.end() - 1);
        for (size_t n = 0; n < death.size(); n++) dead_net[(size_t)at[(size_t)death[n]]++] = (int32_t)n;
    }
    int32_t *dptr = nullptr, *dnet = nullptr;
    // level-aligned cell pairs (the dataflow simulation's unit of work)
    std::vector<int32_t> pair_ptr((size_t)cp->n_levels + 1, 0);
    for (int l = 1; l <= cp->n_levels; l++)
        pair_ptr[l] = pair_ptr[l - 1] + (cp->lvl_ptr[l] - cp->lvl_ptr[l - 1] + 1) / 2;
    int32_t *pairs = nullptr;
    float *base = nullptr;
#define TRY(x) do { if ((s = (x)) != DP_OK) { free_design(D); return s; } } while (0)
    TRY(dalloc(D, &fanin, nc));
    TRY(dalloc(D, &fptr, nn + 1));
    TRY(dalloc(D, &fedge, (size_t)cp->n_edges));
    TRY(dalloc(D, &nou, nn));
    TRY(dalloc(D, &cou, nc));
    TRY(dalloc(D, &base, nn));
    TRY(dalloc(D, &d.pincap, nc));
    TRY(dalloc(D, &d.cload, nn));
    TRY(dalloc(D, &d.sp_in, ns));
    TRY(dalloc(D, &d.tr_in, ns));
    TRY(dalloc(D, &d.pq, nn));
    TRY(dalloc(D, &d.tr, nn));
    TRY(dalloc(D, &d.beta, nn));
    TRY(dalloc(D, &d.trh, nn));
    TRY(dalloc(D, &d.toggles, nn));
    TRY(dalloc(D, &d.ones, nn));
    TRY(dalloc(D, &d.gnet, nn));
    TRY(dalloc(D, &d.gfo, (size_t)cp->n_edges));
    TRY(dalloc(D, &efpos, 4 * nc));
    TRY(dalloc(D, &lvl, (size_t)cp->n_levels + 1));
    TRY(dalloc(D, &d.bar, dp::persist_bar_words(cp->n_levels)));
    TRY(dalloc(D, &d.epoch, 4));
    TRY(dalloc(D, &chunks, chunk_ptr.size()));
    TRY(dalloc(D, &pairs, pair_ptr.size()));
    TRY(dalloc(D, &dptr, dead_ptr.size()));
    TRY(dalloc(D, &dnet, dead_net.size()));
    TRY(dalloc(D, &d.partials, (size_t)dp::kPowerBlocks));
    TRY(dalloc(D, &d.power, 4));
    d.fanin = fanin;
    d.fout_ptr = fptr;
    d.fout_edge = fedge;
    d.edge_fpos = efpos;
    d.lvl = lvl;
    d.chunk_ptr = chunks;
    d.pair_ptr = pairs;
    d.dead_ptr = dptr;
    d.dead_net = dnet;
    d.err = ctx->d_err;
    d.net_of_user = nou;
    d.cell_of_user = cou;
    d.base_cap = base;
    cudaStream_t st = ctx->stream;
    cudaError_t e = cudaSuccess;
    auto up = [&](void *dst, const void *src, size_t b) {
        if (e == cudaSuccess && b) e = cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, st);
    };
    up(fanin, cp->fanin.data(), sizeof(uint32_t) * cp->fanin.size());
    up(fptr, cp->fout_ptr.data(), sizeof(int32_t) * cp->fout_ptr.size());
    up(fedge, cp->fout_edge.data(), sizeof(int32_t) * cp->fout_edge.size());
    up(efpos, cp->edge_fpos.data(), sizeof(int32_t) * cp->edge_fpos.size());
    up(lvl, cp->lvl_ptr.data(), sizeof(int32_t) * cp->lvl_ptr.size());
    up(chunks, chunk_ptr.data(), sizeof(int32_t) * chunk_ptr.size());
    up(pairs, pair_ptr.data(), sizeof(int32_t) * pair_ptr.size());
    up(dptr, dead_ptr.data(), sizeof(int32_t) * dead_ptr.size());
    up(dnet, dead_net.data(), sizeof(int32_t) * dead_net.size());
    up(nou, cp->net_of_user.data(), sizeof(int32_t) * nn);
    up(cou, cp->cell_of_user.data(), sizeof(int32_t) * nc);
    up(base, cp->base_cap.data(), sizeof(float) * nn);
    up(d.pincap, cp->pincap.data(), sizeof(float) * nc);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.power, 0, 4 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.epoch, 0, 4 * sizeof(uint32_t), st);
    // tag 0 everywhere: the first forward pass writes tag 1
    if (e == cudaSuccess) e = cudaMemsetAsync(d.pq, 0, sizeof(float4) * nn, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.bar, 0, sizeof(unsigned) * dp::persist_bar_words(cp->n_levels), st);
    for (int w = 0; w < 4; w++) D->grid[w] = dp::persist_grid(w, ctx->sm_count);
    {
        int32_t width = 0;
        for (int l = 1; l <= cp->n_levels; l++) width = std::max(width, cp->lvl_ptr[l] - cp->lvl_ptr[l - 1]);
        const size_t smem = dp::block_smem(1, cp->n_nets, cp->n_edges, cp->n_levels);   // the larger of the two
        if (cp->n_levels > 0 && width <= dp::kBlockMaxWidth && smem <= (size_t)dp::kBlockSmemMax &&
            dp::block_smem_init())
            D->block_threads = std::min(dp::kBlockThreads, std::max(256, (width + 31) / 32 * 32));
    }
    if (D->block_threads == 0 && cp->n_levels > 0 && e == cudaSuccess) {
        // the single-cluster passes: level l (level 0: the startpoints) cut into C contiguous
        // chunks, block b computing chunk b and holding its nets at consecutive slots
        const int C = dp::kClusterBlocks, L = cp->n_levels;
        auto lo_of = [&](int l) { return l ? ns + cp->lvl_ptr[(size_t)l - 1] : (int64_t)0; };
        auto hi_of = [&](int l) { return l ? ns + cp->lvl_ptr[(size_t)l] : ns; };
        std::vector<int32_t> chunk((size_t)L + 1);
        int most = 0;
        for (int l = 0; l <= L; l++) {
            chunk[(size_t)l] = (int32_t)((hi_of(l) - lo_of(l) + C - 1) / C);
            if (l) most = std::max(most, chunk[(size_t)l]);
        }
        const int threads = std::max(64, (most + 31) / 32 * 32);
        std::vector<int32_t> base((size_t)C * (L + 1));
        std::vector<int64_t> held((size_t)C, 0);
        for (int l = 0; l <= L; l++)
            for (int b = 0; b < C; b++) {
                base[(size_t)b * (L + 1) + l] = (int32_t)held[(size_t)b];
                held[(size_t)b] += std::min<int64_t>(chunk[(size_t)l],
                                                     std::max<int64_t>(0, hi_of(l) - lo_of(l) - (int64_t)b * chunk[(size_t)l]));
            }
        const int64_t slots = *std::max_element(held.begin(), held.end());
        if (threads <= dp::kClusterMaxThreads && dp::cluster_smem(0, slots, 0, L) <= (size_t)dp::kBlockSmemMax) {
            std::vector<int32_t> loc((size_t)nn), lfptr((size_t)nn);
            for (int l = 0; l <= L; l++)
                for (int64_t i = 0; i < hi_of(l) - lo_of(l); i++) {
                    const int64_t b = i / chunk[(size_t)l];
                    loc[(size_t)(lo_of(l) + i)] =
                        (int32_t)((b << 24) | (base[(size_t)b * (L + 1) + l] + i % chunk[(size_t)l]));
                }
            std::vector<int64_t> fill((size_t)C, 0);
            for (int64_t n = 0; n < nn; n++) {
                const size_t b = (size_t)((uint32_t)loc[(size_t)n] >> 24);
                lfptr[(size_t)n] = (int32_t)fill[b];
                fill[b] += cp->fout_ptr[(size_t)n + 1] - cp->fout_ptr[(size_t)n];
            }
            const int64_t edges = *std::max_element(fill.begin(), fill.end());
            const size_t sf = dp::cluster_smem(0, slots, 0, L), sb = dp::cluster_smem(1, slots, edges, L);
            if (sb <= (size_t)dp::kBlockSmemMax && dp::cluster_fits(threads, sf, sb)) {
                std::vector<int32_t> floc(4 * (size_t)nc, 0), lefpos(4 * (size_t)nc, -1);
                for (int64_t c = 0; c < nc; c++) {
                    const uint32_t *r = &cp->fanin[4 * (size_t)c];
                    const int k = cp->op_arity[r[0] >> 24];
                    for (int j = 0; j < k; j++) {
                        const uint32_t m = j == 0 ? (r[0] & dp::kNetMask) : r[j];
                        floc[4 * (size_t)c + j] = loc[m];
                        lefpos[4 * (size_t)c + j] = lfptr[m] + (cp->edge_fpos[4 * (size_t)c + j] - cp->fout_ptr[m]);
                    }
                }
                int32_t *dchunk = nullptr, *dbase = nullptr, *dfloc = nullptr, *dlfptr = nullptr, *dlefpos = nullptr;
                TRY(dalloc(D, &dchunk, chunk.size()));
                TRY(dalloc(D, &dbase, base.size()));
                TRY(dalloc(D, &dfloc, floc.size()));
                TRY(dalloc(D, &dlfptr, lfptr.size()));
                TRY(dalloc(D, &dlefpos, lefpos.size()));
                up(dchunk, chunk.data(), sizeof(int32_t) * chunk.size());
                up(dbase, base.data(), sizeof(int32_t) * base.size());
                up(dfloc, floc.data(), sizeof(int32_t) * floc.size());
                up(dlfptr, lfptr.data(), sizeof(int32_t) * lfptr.size());
                up(dlefpos, lefpos.data(), sizeof(int32_t) * lefpos.size());
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // before the host vectors go
                D->cl = dp::ClusterMap{threads, slots, edges, dchunk, dbase, dfloc, dlfptr, dlefpos};
            }
        }
    }
    if (const char *v = std::getenv("DP_FLOW_BLOCKS")) D->flow_blocks_per_sm = std::atoi(v);
    if (const char *v = std::getenv("DP_FLOW_SLEEP")) D->flow_sleep = (unsigned)std::atoi(v);
    D->flow_grid[0] = dp::flow_grid(0, ctx->sm_count, D->flow_blocks_per_sm);
    D->flow_grid[1] = dp::flow_grid(1, ctx->sm_count, 2);
    if (e != cudaSuccess) { s = cuda_err(ctx, e, "upload"); free_design(D); return s; }
    dp::launch_cload(d, st);
    for (auto &ev : D->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&D->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&D->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&D->ev_grads, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&D->ev_copies, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { s = cuda_err(ctx, e, "upload"); free_design(D); return s; }
#undef TRY
    *out = D;
    return DP_OK;
}

dp_status dp_design_load(dp_ctx *ctx, const char *netlist, size_t netlist_len, const char *library,
                         size_t library_len, dp_design **out) {
    if (!ctx || !out) return set_err(ctx, DP_EINVAL, "NULL argument");
    dp_compiled *cp = nullptr;
    char msg[512] = {0};
    dp_status s = dp_compile(netlist, netlist_len, library, library_len, &cp, msg, sizeof msg);
    if (s != DP_OK) return set_err(ctx, s, std::string("compile: ") + msg);
    s = dp_design_upload(ctx, cp, out);
    dp_compiled_free(cp);
    return s;
}

dp_status dp_design_load_blob(dp_ctx *ctx, const void *blob, size_t len, dp_design **out) {
    if (!ctx || !out) return set_err(ctx, DP_EINVAL, "NULL argument");
    dp_compiled *cp = nullptr;
    char msg[256] = {0};
    dp_status s = dp_compiled_load(blob, len, &cp, msg, sizeof msg);
    if (s != DP_OK) return set_err(ctx, s, msg);
    s = dp_design_upload(ctx, cp, out);
    dp_compiled_free(cp);
    return s;
}

void dp_design_free(dp_design *D) { free_design(D); }

dp_status dp_design_info(const dp_design *D, dp_info *info) {
    if (!D || !info) return DP_EINVAL;
    info->n_nets = D->d.n_nets;
    info->n_start = D->d.n_start;
    info->n_cells = D->d.n_cells;
    info->n_edges = D->n_edges;
    info->n_levels = D->d.n_levels;
    info->n_ops = D->n_ops;
    info->device_bytes = D->bytes + D->batch.bytes + D->batch.vbytes;
    info->block_threads = D->block_threads;
    info->cluster_threads = D->cl.threads;
    return DP_OK;
}

dp_status dp_set_inputs(dp_design *D, const float *sp, const float *tr, int32_t n_scen, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    if (n_scen < 1) return set_err(c, DP_EINVAL, "n_scen must be at least 1");
    if (n_scen > 1) return dp_set_inputs_batch(D, sp, tr, n_scen, on_device);
    const int64_t ns = D->d.n_start;
    if (ns && (!sp || !tr)) return set_err(c, DP_EINVAL, "NULL input");
    if (!on_device) {
        // a branch-free pass (vectorisable) first; the offending index only on failure
        int bad = 0;
        for (int64_t k = 0; k < ns; k++)
            bad |= !(sp[k] >= 0.f) | !(sp[k] <= 1.f) | !(tr[k] >= 0.f) | !(tr[k] <= 1.f);
        if (bad)
            for (int64_t k = 0; k < ns; k++)
                if (!(sp[k] >= 0.f && sp[k] <= 1.f && tr[k] >= 0.f && tr[k] <= 1.f))
                    return set_err(c, DP_EINVAL,
                                   "input SP and TR must lie in [0,1] (startpoint " + std::to_string(k) + ")");
    }
    DeviceGuard g(c->device);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    if (ns) e = cudaMemcpyAsync(D->d.sp_in, sp, sizeof(float) * (size_t)ns, kind, c->stream);
    if (ns && e == cudaSuccess) e = cudaMemcpyAsync(D->d.tr_in, tr, sizeof(float) * (size_t)ns, kind, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_set_inputs");
    D->inputs_set = true;
    D->batched = false;
    D->fwd_valid = false;
    D->sim_valid = false;
    D->bwd_valid = false;
    D->batch.fwd_valid = false;
    return DP_OK;
}

dp_status dp_set_pincap(dp_design *D, const int32_t *cells, const float *caps, int32_t n, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    if (n < 0 || (n > 0 && !caps)) return set_err(c, DP_EINVAL, "bad sizing delta");
    if (!cells && n != D->d.n_cells) return set_err(c, DP_EINVAL, "a NULL cell list needs one cap per cell");
    if (n == 0) return DP_OK;
    DeviceGuard g(c->device);
    int32_t *dc = nullptr;
    float *dv = nullptr;
    cudaError_t e = cudaSuccess;
    if (!on_device) {
        for (int32_t i = 0; i < n; i++)
            if ((cells && (cells[i] < 0 || cells[i] >= D->d.n_cells)) || !(caps[i] >= 0.f) || !std::isfinite(caps[i]))
                return set_err(c, DP_EINVAL, "cell index or pin cap out of range");
        // the design's own staging, grown on demand: a sizing loop allocates nothing per call
        dp_status rs = reserve_pincap_staging(D, n);
        if (rs != DP_OK) return rs;
        e = cudaStreamWaitEvent(c->stream, D->pc_done, 0);   // the previous delta's kernels are done
        if (e == cudaSuccess && cells)
            e = cudaMemcpyAsync(D->pc_cells, cells, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(D->pc_caps, caps, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_err(c, e, "dp_set_pincap");
        dc = cells ? D->pc_cells : nullptr;
        dv = D->pc_caps;
    } else {
        dc = const_cast<int32_t *>(cells);
        dv = const_cast<float *>(caps);
    }
    dp::launch_set_pincap(D->d, dc, dv, n, c->stream);
    dp::launch_cload(D->d, c->stream);
    D->bwd_valid = false;   // the local gradient terms depend on the loads
    dp_status s = launch_check(c, "dp_set_pincap");
    if (!on_device && s == DP_OK) {
        e = cudaEventRecord(D->pc_done, c->stream);
        if (e != cudaSuccess) s = cuda_err(c, e, "dp_set_pincap");
    }
    // loads changed: the powers and gradients must be recomputed (SP and TR stay valid)
    return s;
}

dp_status dp_propagate(dp_design *D, const dp_config *cfg) {
    if (!D) return DP_EINVAL;
    dp_status s = check_cfg(D->ctx, cfg);
    if (s != DP_OK) return s;
    if (!D->inputs_set) return set_err(D->ctx, DP_ESTATE, "dp_propagate before dp_set_inputs");
    if (D->batched) return batch_propagate(D, *cfg);
    if (cfg->tr_mode == 2) return set_err(D->ctx, DP_EUNSUPPORTED, "the lag-one mode runs on batched inputs");
    DeviceGuard g(D->ctx->device);
    cudaStream_t st = D->ctx->stream;
    rec(D, 0, st);
    cudaError_t le = q_forward(D, *cfg, st);
    rec(D, 1, st);
    if ((s = cuda_err(D->ctx, le, "dp_propagate")) != DP_OK) return s;
    D->fwd_valid = true;
    D->fwd_tr_mode = cfg->tr_mode;
    D->sim_valid = false;
    D->bwd_valid = false;
    return DP_OK;
}

dp_status dp_simulate(dp_design *D, const dp_config *cfg) {
    if (!D) return DP_EINVAL;
    dp_status s = check_cfg(D->ctx, cfg);
    if (s != DP_OK) return s;
    if (D->batched) return set_err(D->ctx, DP_EUNSUPPORTED, "the simulation runs on single-scenario inputs");
    if (cfg->tr_mode == 2) return set_err(D->ctx, DP_EUNSUPPORTED, "the lag-one mode runs on batched inputs");
    if (!D->fwd_valid || D->fwd_tr_mode != cfg->tr_mode)
        return set_err(D->ctx, DP_ESTATE, "dp_simulate needs dp_propagate with the same tr_mode");
    DeviceGuard g(D->ctx->device);
    if ((s = ensure_words(D, cfg->sim_words)) != DP_OK) return s;
    cudaStream_t st = D->ctx->stream;
    rec(D, 1, st);
    q_sim_start(D, *cfg, st);
    cudaError_t le = q_sim_levels(D, *cfg, st);
    rec(D, 2, st);
    if (le == cudaSuccess) le = q_hybrid(D, *cfg, st);
    rec(D, 3, st);
    if ((s = cuda_err(D->ctx, le, "dp_simulate")) != DP_OK) return s;
    D->sim_valid = true;
    return DP_OK;
}

dp_status dp_total_power(dp_design *D, int hybrid, double *watts) { return dp_get_power(D, hybrid, watts, 0); }

dp_status dp_get_power(dp_design *D, int hybrid, double *watts, int on_device) {
    if (!D || !watts) return DP_EINVAL;
    if (D->batched) return batch_get_power(D, hybrid, watts, on_device);
    if (!D->fwd_valid || (hybrid && !D->sim_valid))
        return set_err(D->ctx, DP_ESTATE, hybrid ? "hybrid power needs dp_simulate" : "power needs dp_propagate");
    DeviceGuard g(D->ctx->device);
    cudaError_t e = cudaMemcpyAsync(watts, D->d.power + (hybrid ? 1 : 0), sizeof(double),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, D->ctx->stream);
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "dp_get_power");
    if (on_device) return DP_OK;
    e = cudaStreamSynchronize(D->ctx->stream);
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "dp_get_power");
    return check_device_error(D->ctx);
}

dp_status dp_backward(dp_design *D, const dp_config *cfg, float *gsp, float *gtr, float *gpin, float *gcl,
                      int on_device) {
    if (!D) return DP_EINVAL;
    if (D->batched) return dp_backward_weighted(D, cfg, nullptr, 0, gsp, gtr, gpin, gcl, on_device);
    dp_status s = check_cfg(D->ctx, cfg);
    if (s != DP_OK) return s;
    if (!D->fwd_valid || D->fwd_tr_mode != cfg->tr_mode)
        return set_err(D->ctx, DP_ESTATE, "dp_backward needs dp_propagate with the same tr_mode");
    if (cfg->grad_mode != 0 && !D->sim_valid)
        return set_err(D->ctx, DP_ESTATE, "hybrid gradients need dp_simulate");
    DeviceGuard g(D->ctx->device);
    cudaStream_t st = D->ctx->stream;
    rec(D, 3, st);
    cudaError_t le = q_backward(D, *cfg, on_device ? gsp : nullptr, st);
    rec(D, 4, st);
    if ((s = cuda_err(D->ctx, le, "dp_backward")) != DP_OK) return s;
    D->bwd_valid = true;
    D->bwd_grad_mode = cfg->grad_mode;
    s = q_outputs(D, *cfg, gsp, gtr, gpin, gcl, on_device, on_device != 0);
    rec(D, 5, st);
    return s;
}

dp_status dp_get_nets(dp_design *D, float *sp, float *tr, float *beta, float *trh, uint32_t *tg, uint32_t *on,
                      int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    if (D->batched) {
        if (beta || trh || tg || on)
            return set_err(c, DP_EUNSUPPORTED, "simulation outputs exist for single-scenario inputs only");
        return batch_get_nets(D, sp, tr, on_device);
    }
    if ((sp || tr) && !D->fwd_valid) return set_err(c, DP_ESTATE, "SP/TR need dp_propagate");
    if ((beta || trh || tg || on) && !D->sim_valid) return set_err(c, DP_ESTATE, "simulation outputs need dp_simulate");
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    const int64_t nn = D->d.n_nets;
    if (nn == 0) return DP_OK;
    dp_status s = DP_OK;
    float *stage = nullptr;
    if (!on_device) {
        if ((s = ensure_stage(D)) != DP_OK) return s;
        stage = D->st_gcl;  // n_nets floats
    }
    struct Out { void *dst; int kind; };
    Out outs[6] = {{sp, 0}, {tr, 1}, {beta, 2}, {trh, 3}, {tg, 4}, {on, 5}};
    for (auto &o : outs) {
        if (!o.dst) continue;
        void *dst = on_device ? o.dst : (void *)stage;
        switch (o.kind) {
            case 0: dp::launch_sp_user(D->d, (float *)dst, st); break;
            case 1: dp::launch_gather_f32(D->d.tr, D->d.net_of_user, (float *)dst, nn, st); break;
            case 2: dp::launch_gather_f32(D->d.beta, D->d.net_of_user, (float *)dst, nn, st); break;
            case 3: dp::launch_trh_user(D->d, (float *)dst, st); break;
            case 4: dp::launch_gather_u32(D->d.toggles, D->d.net_of_user, (uint32_t *)dst, nn, st); break;
            case 5: dp::launch_gather_u32(D->d.ones, D->d.net_of_user, (uint32_t *)dst, nn, st); break;
        }
        if ((s = launch_check(c, "dp_get_nets")) != DP_OK) return s;
        if (!on_device) {
            cudaError_t e = cudaMemcpyAsync(o.dst, stage, 4 * (size_t)nn, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_err(c, e, "dp_get_nets");
        }
    }
    return on_device ? DP_OK : check_device_error(c);
}

dp_status dp_step(dp_design *D, const dp_config *cfg, float *gsp, float *gtr, float *gpin, float *gcl, double *watts,
                  int on_device) {
    if (!D) return DP_EINVAL;
    dp_status s = check_cfg(D->ctx, cfg);
    if (s != DP_OK) return s;
    if (!D->inputs_set) return set_err(D->ctx, DP_ESTATE, "dp_step before dp_set_inputs");
    if (D->batched) return set_err(D->ctx, DP_EUNSUPPORTED, "dp_step runs on single-scenario inputs");
    if (cfg->tr_mode == 2) return set_err(D->ctx, DP_EUNSUPPORTED, "the lag-one mode runs on batched inputs");
    DeviceGuard g(D->ctx->device);
    if ((s = ensure_words(D, cfg->sim_words)) != DP_OK) return s;
    if ((s = ensure_stage(D)) != DP_OK) return s;
    if ((s = ensure_step_streams(D)) != DP_OK) return s;
    cudaStream_t st = D->ctx->stream;
    if (!D->graph || std::memcmp(&D->graph_cfg, cfg, sizeof *cfg) != 0) {
        if (D->graph) { cudaGraphExecDestroy(D->graph); D->graph = nullptr; }
        cudaStream_t cs = D->cap_stream;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(D->ctx, e, "graph capture");
        // external event records become timing nodes of the graph (a plain record
        // inside a capture only expresses a dependency).  The startpoint generator
        // (ALU-bound) runs on a second branch, concurrently with the forward pass
        // (latency-bound); the simulation levels wait for both.  The branch forks right
        // before the forward kernel, so that the two become ready together: forked
        // earlier, the generator's blocks fill the SMs first when the GPU is idle at the
        // launch, and the cooperative forward kernel waits for room.
        cudaEventRecordWithFlags(D->ev[0], cs, cudaEventRecordExternal);
        cudaError_t le = q_forward(D, *cfg, cs, D->fork);
        cudaEventRecordWithFlags(D->ev[1], cs, cudaEventRecordExternal);
        cudaStreamWaitEvent(D->cap_stream2, D->fork, 0);
        q_sim_start(D, *cfg, D->cap_stream2);
        cudaEventRecord(D->join, D->cap_stream2);
        cudaStreamWaitEvent(cs, D->join, 0);
        if (le == cudaSuccess) le = q_sim_levels(D, *cfg, cs);
        cudaEventRecordWithFlags(D->ev[2], cs, cudaEventRecordExternal);
        if (le == cudaSuccess) le = q_hybrid(D, *cfg, cs);
        cudaEventRecordWithFlags(D->ev[3], cs, cudaEventRecordExternal);
        // the cap and TR gradients need only the hybrid activities: a second branch
        // writes them to the staging buffers beside the (latency-bound) backward pass
        cudaEventRecord(D->fork, cs);
        cudaStreamWaitEvent(D->cap_stream2, D->fork, 0);
        dp::launch_cap_grads(D->d, D->ops, cfg->grad_mode != 0, cfg->tr_mode, power_K(*cfg), D->st_gcl, D->st_gpin,
                             D->st_gtr, D->cap_stream2);
        cudaEventRecordWithFlags(D->ev_grads, D->cap_stream2, cudaEventRecordExternal);
        cudaEventRecord(D->join, D->cap_stream2);
        if (le == cudaSuccess) le = q_backward(D, *cfg, nullptr, cs, true);
        cudaStreamWaitEvent(cs, D->join, 0);
        cudaEventRecordWithFlags(D->ev[4], cs, cudaEventRecordExternal);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
        D->graph_kernels = 0;
        if (e == cudaSuccess) {
            size_t nn = 0;
            e = cudaGraphGetNodes(graph, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
            for (size_t i = 0; e == cudaSuccess && i < nn; i++) {
                cudaGraphNodeType t;
                if ((e = cudaGraphNodeGetType(nodes[i], &t)) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                    D->graph_kernels++;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&D->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) { D->graph = nullptr; return cuda_err(D->ctx, e, "graph instantiate"); }
        D->graph_cfg = *cfg;
    }
    cudaError_t e = cudaGraphLaunch(D->graph, st);
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "graph launch");
    for (int i = 0; i < 5; i++) D->ev_valid[i] = true;
    D->fwd_valid = true;
    D->fwd_tr_mode = cfg->tr_mode;
    D->sim_valid = true;
    D->bwd_valid = true;
    D->bwd_grad_mode = cfg->grad_mode;
    D->step_kernels = D->graph_kernels;
    return q_step_copies(D, gsp, gtr, gpin, gcl, watts, on_device);
}

dp_status dp_sizing_scores(dp_design *D, const dp_config *cfg, int32_t mode, float *scores, int32_t k,
                           int32_t *top_cells, float *top_scores, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    dp_status s = check_cfg(c, cfg);
    if (s != DP_OK) return s;
    if (mode < 0 || mode > 1) return set_err(c, DP_EINVAL, "mode must be 0 or 1");
    const int64_t nc = D->d.n_cells;
    if (k < 0 || (k > 0 && !top_cells)) return set_err(c, DP_EINVAL, "bad k or NULL top_cells");
    if (D->batched) return set_err(c, DP_EUNSUPPORTED, "sizing scores are computed for single-scenario inputs");
    if (!D->bwd_valid || D->bwd_grad_mode != cfg->grad_mode || D->fwd_tr_mode != cfg->tr_mode)
        return set_err(c, DP_ESTATE, "sizing scores need dp_backward (or dp_step) with the same config");
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    if (!D->sc_scores) {
        if ((s = dalloc(D, &D->sc_scores, (size_t)nc)) != DP_OK) return s;
        if ((s = dalloc(D, &D->sc_idx, (size_t)nc)) != DP_OK) return s;
        if ((s = dalloc(D, &D->sc_hist, 257)) != DP_OK) return s;
    }
    dp::launch_scores(D->d, cfg->grad_mode != 0, (float)power_K(*cfg), mode, D->sc_scores, st);
    if ((s = launch_check(c, "dp_sizing_scores")) != DP_OK) return s;
    cudaError_t e = cudaSuccess;
    if (scores && nc)
        e = cudaMemcpyAsync(scores, D->sc_scores, sizeof(float) * (size_t)nc,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores");
    if (k == 0 || nc == 0) {
        if (!on_device && (e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores");
        return on_device ? DP_OK : check_device_error(c);
    }
    const int64_t kk = k < nc ? k : nc;
    // radix select of the kk-th largest score: 8-bit digits, most significant first
    uint32_t prefix = 0, mask = 0;
    int64_t remaining = kk;
    unsigned hist[256];
    for (int shift = 24; shift >= 0; shift -= 8) {
        e = cudaMemsetAsync(D->sc_hist, 0, 256 * sizeof(unsigned), st);
        if (e == cudaSuccess) dp::launch_radix_hist(D->sc_scores, nc, prefix, mask, shift, D->sc_hist, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hist, D->sc_hist, sizeof hist, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores (select)");
        int64_t above = 0;
        int b = 255;
        for (; b > 0; b--) {
            if (above + (int64_t)hist[b] >= remaining) break;
            above += hist[b];
        }
        remaining -= above;
        prefix |= (uint32_t)b << shift;
        mask |= 0xFFu << shift;
    }
    // every cell at or above the threshold (the kk-th score), then exact ordering on the host
    unsigned cnt = 0;
    e = cudaMemsetAsync(D->sc_hist + 256, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) dp::launch_radix_collect(D->sc_scores, nc, prefix, D->sc_idx, D->sc_hist + 256, nc, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, D->sc_hist + 256, sizeof cnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores (collect)");
    std::vector<int32_t> idx(cnt);
    std::vector<float> all((size_t)nc);
    if (cnt) e = cudaMemcpy(idx.data(), D->sc_idx, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(all.data(), D->sc_scores, sizeof(float) * (size_t)nc, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores (collect)");
    std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        return all[(size_t)a] != all[(size_t)b] ? all[(size_t)a] > all[(size_t)b] : a < b;
    });
    if ((int64_t)idx.size() < kk) return set_err(c, DP_ECUDA, "top-k selection lost candidates");
    std::vector<float> ts((size_t)kk);
    for (int64_t i = 0; i < kk; i++) ts[(size_t)i] = all[(size_t)idx[(size_t)i]];
    const cudaMemcpyKind kind = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    e = cudaMemcpy(top_cells, idx.data(), sizeof(int32_t) * (size_t)kk, kind);
    if (e == cudaSuccess && top_scores) e = cudaMemcpy(top_scores, ts.data(), sizeof(float) * (size_t)kk, kind);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_sizing_scores (top)");
    return check_device_error(c);
}

dp_status dp_step_kernels(const dp_design *D, int64_t *k) {
    if (!D || !k) return DP_EINVAL;
    *k = D->step_kernels;
    return DP_OK;
}

dp_status dp_phase_times(dp_design *D, float *ms) {
    if (!D || !ms) return DP_EINVAL;
    DeviceGuard g(D->ctx->device);
    cudaError_t e = cudaStreamSynchronize(D->ctx->stream);
    if (e != cudaSuccess) return cuda_err(D->ctx, e, "dp_phase_times");
    for (int i = 0; i < 5; i++) {
        ms[i] = 0.f;
        if (D->ev_valid[i] && D->ev_valid[i + 1]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, D->ev[i], D->ev[i + 1]) == cudaSuccess) ms[i] = t;
            else cudaGetLastError();
        }
    }
    return DP_OK;
}

}  // extern "C"
