// C-ABI of the batched path: S input-activity scenarios of one resident
// design per launch (scenario-innermost SoA), the per-scenario weighted
// backward used by autograd callers, the projected ascent step and the
// power-virus evaluation of Algorithm 4 (Eq. 3).  Calls with device outputs
// neither synchronise nor allocate once the buffers for the largest S have
// been made, so a caller can capture them in a CUDA graph.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "capi_internal.h"

using namespace dpi;

namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// launch shapes the tuner tries: bx threads over scenarios x by cells per block, v scenarios
// per thread (2 or 4 only where S is a multiple of it)
const dp::BatchShape kShapes[] = {{32, 4, 1}, {32, 8, 1},  {64, 2, 1},  {64, 4, 1},  {128, 1, 1}, {128, 2, 1},
                                  {256, 1, 1}, {512, 1, 1}, {32, 8, 2},  {64, 2, 2},  {64, 4, 2},  {128, 1, 2},
                                  {128, 2, 2}, {256, 1, 2}, {32, 4, 4},  {64, 2, 4},  {128, 1, 4}};

template <class T>
dp_status balloc(dp_design *D, T **p, size_t count) {
    void *v = nullptr;
    dp_status s = alloc_into(D->ctx, &v, sizeof(T) * (count ? count : 1), &D->batch.allocs, &D->batch.bytes);
    *p = static_cast<T *>(v);
    return s;
}

template <class T>
dp_status valloc(dp_design *D, T **p, size_t count) {
    void *v = nullptr;
    dp_status s = alloc_into(D->ctx, &v, sizeof(T) * (count ? count : 1), &D->batch.vallocs, &D->batch.vbytes);
    *p = static_cast<T *>(v);
    return s;
}

void free_list(std::vector<void *> &l, size_t &bytes) {
    for (void *p : l) cudaFree(p);
    l.clear();
    bytes = 0;
}

// Buffers for S scenarios (reallocated only for a larger S).
dp_status ensure_batch(dp_design *D, int64_t S) {
    dp_batch &B = D->batch;
    if (B.cap >= S) return DP_OK;
    dp_ctx *c = D->ctx;
    if (capturing(c->stream))
        return set_err(c, DP_ESTATE, "the first call with a larger n_scen allocates: make it before stream capture");
    cudaStreamSynchronize(c->stream);
    free_list(B.allocs, B.bytes);
    B.b = dp::BatchBufs{};
    B.stage = nullptr;
    B.cap = 0;
    B.tuned_S = 0;
    B.shapes_locked = false;
    const size_t ns = (size_t)D->d.n_start, nn = (size_t)D->d.n_nets, ne = (size_t)D->n_edges, s = (size_t)S;
    dp_status st = DP_OK;
#define TRYB(x) do { if ((st = (x)) != DP_OK) { free_list(B.allocs, B.bytes); B.b = dp::BatchBufs{}; return st; } } while (0)
    TRYB(balloc(D, &B.b.sp_in, ns * s));
    TRYB(balloc(D, &B.b.tr_in, ns * s));
    TRYB(balloc(D, &B.b.pq, nn * s));
    TRYB(balloc(D, &B.b.gfo, ne * s));
    TRYB(balloc(D, &B.b.gsp, ns * s));
    TRYB(balloc(D, &B.b.partials, (size_t)dp::kBatchPowerChunks * s));
    TRYB(balloc(D, &B.b.power, s));
    TRYB(balloc(D, &B.b.ks, s));
    TRYB(balloc(D, &B.weights, s));
#undef TRYB
    B.cap = S;
    return DP_OK;
}

dp_status ensure_stage_batch(dp_design *D) {
    dp_batch &B = D->batch;
    if (B.stage) return DP_OK;
    int64_t rows = D->d.n_nets;
    if (D->d.n_cells > rows) rows = D->d.n_cells;
    return balloc(D, &B.stage, (size_t)rows * (size_t)B.cap);
}

// DP_BATCH_SHAPE = "bx,by" | "bx,by,v" (both passes) | "bx,by,bx,by" | "bx,by,v,bx,by,v" (forward, reverse)
bool parse_shape_env(dp::BatchShape *f, dp::BatchShape *b) {
    const char *v = std::getenv("DP_BATCH_SHAPE");
    if (!v) return false;
    int a[6] = {0, 0, 0, 0, 0, 0};
    const int n = std::sscanf(v, "%d,%d,%d,%d,%d,%d", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5]);
    int s[2][3];
    if (n == 2 || n == 3) {
        for (int i = 0; i < 2; i++) {
            s[i][0] = a[0];
            s[i][1] = a[1];
            s[i][2] = n == 3 ? a[2] : 1;
        }
    } else if (n == 4) {
        s[0][0] = a[0]; s[0][1] = a[1]; s[0][2] = 1;
        s[1][0] = a[2]; s[1][1] = a[3]; s[1][2] = 1;
    } else if (n == 6) {
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 3; j++) s[i][j] = a[3 * i + j];
    } else {
        return false;
    }
    for (int i = 0; i < 2; i++)
        if (s[i][0] < 32 || s[i][0] > 1024 || (s[i][0] & 31) || s[i][1] < 1 || s[i][0] * s[i][1] > 1024 ||
            (s[i][2] != 1 && s[i][2] != 2 && s[i][2] != 4))
            return false;
    *f = dp::BatchShape{s[0][0], s[0][1], s[0][2]};
    *b = dp::BatchShape{s[1][0], s[1][1], s[1][2]};
    return true;
}

// Autotuner: times the forward and the reverse pass of this design at this S
// for every candidate shape (CUDA events, best of two after a warm-up) and
// keeps the fastest of each.  Runs on the staged inputs; the results it
// leaves are overwritten by the next dp_propagate.
dp_status tune(dp_design *D) {
    dp_batch &B = D->batch;
    dp_ctx *c = D->ctx;
    if (parse_shape_env(&B.fwd_shape, &B.bwd_shape)) {
        B.tuned_S = B.S;
        return DP_OK;
    }
    const int64_t S = B.S;
    const int64_t limit = S <= 32 ? 32 : ((S + 31) / 32) * 32;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    dp_config cfg;
    dp_config_default(&cfg);
    const double K = power_K(cfg);
    cudaStream_t st = c->stream;
    dp::launch_seedb(B.b, K, nullptr, st);
    float best[2] = {1e30f, 1e30f};
    dp::BatchShape pick[2] = {B.fwd_shape, B.bwd_shape};
    for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
        if (pass == 1) dp::launch_fwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), 0, pick[0], st);
        for (const dp::BatchShape &sh : kShapes) {
            if (sh.bx > limit) continue;
            float t = 1e30f;
            for (int r = 0; r < 3 && e == cudaSuccess; r++) {
                cudaEventRecord(e0, st);
                if (pass == 0) dp::launch_fwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), 0, sh, st);
                else dp::launch_bwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), 0, sh, st);
                cudaEventRecord(e1, st);
                e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0 && ms < t) t = ms;   // first run warms up
            }
            if (e == cudaSuccess && t < best[pass]) {
                best[pass] = t;
                pick[pass] = sh;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(c, e, "batch autotuner");
    B.fwd_shape = pick[0];
    B.bwd_shape = pick[1];
    B.tune_ms[0] = best[0];
    B.tune_ms[1] = best[1];
    B.tuned_S = S;
    return check_device_error(c);
}

}  // namespace

namespace dpi {

void free_batch(dp_design *D) {
    free_list(D->batch.allocs, D->batch.bytes);
    free_list(D->batch.vallocs, D->batch.vbytes);
    D->batch = dp_batch{};
}

dp_status batch_reserve(dp_design *D, int64_t S) {
    dp_status s = ensure_batch(D, S);
    return s == DP_OK ? ensure_stage_batch(D) : s;
}

dp_status batch_tune_and_lock(dp_design *D) {
    dp_status s = tune(D);
    if (s == DP_OK) D->batch.shapes_locked = true;
    return s;
}

// the lag-one state (every net's TR, two adjoints per edge, the startpoints' TR adjoint),
// allocated on first use for the current capacity
dp_status ensure_lag1(dp_design *D) {
    dp_batch &B = D->batch;
    if (B.b.tq) return DP_OK;
    if (capturing(D->ctx->stream))
        return set_err(D->ctx, DP_ESTATE, "the first lag-one pass allocates: make it before stream capture");
    const size_t cap = (size_t)B.cap;
    dp_status s = balloc(D, &B.b.tq, (size_t)D->d.n_nets * cap);
    if (s == DP_OK) s = balloc(D, &B.b.gfo2, (size_t)D->n_edges * cap);
    if (s == DP_OK) s = balloc(D, &B.b.gtr, (size_t)D->d.n_start * cap);
    return s;
}

dp_status batch_propagate(dp_design *D, const dp_config &c) {
    dp_batch &B = D->batch;
    DeviceGuard g(D->ctx->device);
    if (c.tr_mode == 2) {
        dp_status s = ensure_lag1(D);
        if (s != DP_OK) return s;
    }
    cudaStream_t st = D->ctx->stream;
    dp::launch_fwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), c.tr_mode, B.fwd_shape, st);
    dp::launch_powerb(D->d, B.b, c.tr_mode, power_K(c), st);
    dp_status s = launch_check(D->ctx, "dp_propagate (batched)");
    if (s != DP_OK) return s;
    B.fwd_valid = true;
    B.fwd_tr_mode = c.tr_mode;
    return DP_OK;
}

dp_status batch_get_power(dp_design *D, int hybrid, double *watts, int on_device) {
    dp_batch &B = D->batch;
    dp_ctx *c = D->ctx;
    if (hybrid) return set_err(c, DP_EUNSUPPORTED, "hybrid power exists for single-scenario inputs only");
    if (!B.fwd_valid) return set_err(c, DP_ESTATE, "power needs dp_propagate");
    DeviceGuard g(c->device);
    cudaError_t e = cudaMemcpyAsync(watts, B.b.power, sizeof(double) * (size_t)B.S,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_get_power");
    if (on_device) return DP_OK;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_err(c, e, "dp_get_power");
    return check_device_error(c);
}

dp_status batch_get_nets(dp_design *D, float *sp, float *tr, int on_device) {
    dp_batch &B = D->batch;
    dp_ctx *c = D->ctx;
    if ((sp || tr) && !B.fwd_valid) return set_err(c, DP_ESTATE, "SP/TR need dp_propagate");
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    if (on_device) {
        dp::launch_netb_user(D->d, B.b, B.fwd_tr_mode, sp, tr, st);
        return launch_check(c, "dp_get_nets (batched)");
    }
    dp_status s = ensure_stage_batch(D);
    if (s != DP_OK) return s;
    float *outs[2] = {sp, tr};
    for (int i = 0; i < 2; i++) {
        if (!outs[i] || D->d.n_nets == 0) continue;
        dp::launch_netb_user(D->d, B.b, B.fwd_tr_mode, i == 0 ? B.stage : nullptr, i == 1 ? B.stage : nullptr, st);
        if ((s = launch_check(c, "dp_get_nets (batched)")) != DP_OK) return s;
        cudaError_t e = cudaMemcpyAsync(outs[i], B.stage, sizeof(float) * (size_t)D->d.n_nets * (size_t)B.S,
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_err(c, e, "dp_get_nets (batched)");
    }
    return check_device_error(c);
}

}  // namespace dpi

extern "C" {

dp_status dp_set_inputs_batch(dp_design *D, const float *sp, const float *tr, int32_t n_scen, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    if (n_scen < 1) return set_err(c, DP_EINVAL, "n_scen must be at least 1");
    const int64_t ns = D->d.n_start, S = n_scen, n = ns * S;
    if (ns && (!sp || !tr)) return set_err(c, DP_EINVAL, "NULL input");
    if (!on_device)
        for (int64_t i = 0; i < n; i++)
            if (!(sp[i] >= 0.f && sp[i] <= 1.f && tr[i] >= 0.f && tr[i] <= 1.f))
                return set_err(c, DP_EINVAL, "input SP and TR must lie in [0,1] (startpoint " + std::to_string(i / S) +
                                                 ", scenario " + std::to_string(i % S) + ")");
    DeviceGuard g(c->device);
    dp_status s = ensure_batch(D, S);
    if (s != DP_OK) return s;
    dp_batch &B = D->batch;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaSuccess;
    if (n) e = cudaMemcpyAsync(B.b.sp_in, sp, sizeof(float) * (size_t)n, kind, c->stream);
    if (n && e == cudaSuccess) e = cudaMemcpyAsync(B.b.tr_in, tr, sizeof(float) * (size_t)n, kind, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_set_inputs_batch");
    B.S = S;
    B.b.S = S;
    B.fwd_valid = false;
    D->inputs_set = true;
    D->batched = true;
    D->fwd_valid = false;
    D->sim_valid = false;
    if (B.tuned_S != S && !B.shapes_locked && !capturing(c->stream)) return tune(D);
    return DP_OK;
}

dp_status dp_batch_tuning(const dp_design *D, int32_t *shape6, float *ms2) {
    if (!D || !shape6) return DP_EINVAL;
    const dp_batch &B = D->batch;
    shape6[0] = B.fwd_shape.bx;
    shape6[1] = B.fwd_shape.by;
    shape6[2] = B.fwd_shape.v;
    shape6[3] = B.bwd_shape.bx;
    shape6[4] = B.bwd_shape.by;
    shape6[5] = B.bwd_shape.v;
    if (ms2) {
        ms2[0] = B.tune_ms[0];
        ms2[1] = B.tune_ms[1];
    }
    return DP_OK;
}

dp_status dp_backward_weighted(dp_design *D, const dp_config *cfg, const double *weights, int32_t cap_reduce,
                               float *gsp, float *gtr, float *gpin, float *gcl, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    dp_status s = check_cfg(c, cfg);
    if (s != DP_OK) return s;
    if (!D->batched) {
        if (weights) return set_err(c, DP_EUNSUPPORTED, "weights need batched inputs (dp_set_inputs_batch)");
        return dp_backward(D, cfg, gsp, gtr, gpin, gcl, on_device);
    }
    dp_batch &B = D->batch;
    if (cfg->grad_mode != 0)
        return set_err(c, DP_EUNSUPPORTED, "batched scenarios give the model gradient (grad_mode 0) only");
    if (!B.fwd_valid || B.fwd_tr_mode != cfg->tr_mode)
        return set_err(c, DP_ESTATE, "dp_backward needs dp_propagate with the same tr_mode");
    const int64_t S = B.S;
    if (weights && !on_device)
        for (int64_t i = 0; i < S; i++)
            if (!std::isfinite(weights[i])) return set_err(c, DP_EINVAL, "weights must be finite");
    DeviceGuard g(c->device);
    cudaStream_t st = c->stream;
    const double *wd = weights;
    cudaError_t e = cudaSuccess;
    if (weights && !on_device) {
        e = cudaMemcpyAsync(B.weights, weights, sizeof(double) * (size_t)S, cudaMemcpyHostToDevice, st);
        wd = B.weights;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "dp_backward_weighted");
    dp::launch_seedb(B.b, power_K(*cfg), wd, st);
    dp::launch_bwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), cfg->tr_mode, B.bwd_shape, st);
    if ((s = launch_check(c, "dp_backward (batched)")) != DP_OK) return s;
    const bool reduce = cap_reduce != 0;
    const size_t nsS = (size_t)D->d.n_start * (size_t)S;
    if (on_device) {
        if (gsp && nsS) e = cudaMemcpyAsync(gsp, B.b.gsp, sizeof(float) * nsS, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_err(c, e, "dp_backward_weighted");
        dp::launch_gradb(D->d, B.b, D->ops, cfg->tr_mode, reduce, gtr, gpin, gcl, st);
        return launch_check(c, "gradient outputs (batched)");
    }
    if ((s = ensure_stage_batch(D)) != DP_OK) return s;
    if (gsp && nsS) e = cudaMemcpyAsync(gsp, B.b.gsp, sizeof(float) * nsS, cudaMemcpyDeviceToHost, st);
    struct Out { float *dst; int which; int64_t rows; };
    const Out outs[3] = {{gtr, 0, D->d.n_start}, {gpin, 1, D->d.n_cells}, {gcl, 2, D->d.n_nets}};
    for (const Out &o : outs) {
        if (!o.dst || o.rows == 0 || e != cudaSuccess) continue;
        dp::launch_gradb(D->d, B.b, D->ops, cfg->tr_mode, reduce, o.which == 0 ? B.stage : nullptr,
                         o.which == 1 ? B.stage : nullptr, o.which == 2 ? B.stage : nullptr, st);
        if ((s = launch_check(c, "gradient outputs (batched)")) != DP_OK) return s;
        const size_t cnt = (size_t)o.rows * ((reduce && o.which != 0) ? 1 : (size_t)S);
        e = cudaMemcpyAsync(o.dst, B.stage, sizeof(float) * cnt, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the staging buffer is reused
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_backward_weighted");
    return check_device_error(c);
}

dp_status dp_ascent_step(dp_ctx *c, float *x, const float *g, int64_t n, float eta) {
    if (!c) return DP_EINVAL;
    if (n < 0 || (n > 0 && (!x || !g))) return set_err(c, DP_EINVAL, "bad ascent arrays");
    if (!std::isfinite(eta)) return set_err(c, DP_EINVAL, "eta must be finite");
    DeviceGuard gd(c->device);
    dp::launch_ascent(x, g, n, eta, c->stream);
    return launch_check(c, "dp_ascent_step");
}

dp_status dp_virus_eval(dp_design *D, const float *sp, int32_t n_scen, uint8_t *v0, double *p_virus, int on_device) {
    if (!D) return DP_EINVAL;
    dp_ctx *c = D->ctx;
    if (n_scen < 1 || !p_virus || (D->d.n_start && !sp)) return set_err(c, DP_EINVAL, "bad virus arguments");
    DeviceGuard g(c->device);
    dp_batch &B = D->batch;
    const int64_t S = n_scen, ns = D->d.n_start, nn = D->d.n_nets;
    cudaStream_t st = c->stream;
    if (B.vcap < S) {
        if (capturing(st)) return set_err(c, DP_ESTATE, "the first dp_virus_eval with a larger n_scen allocates");
        cudaStreamSynchronize(st);
        free_list(B.vallocs, B.vbytes);
        B.vcap = 0;
        dp_status s = DP_OK;
        const size_t W2 = 2 * (size_t)cdiv(S, 64);
        if ((s = valloc(D, &B.vwords, (size_t)nn * W2)) != DP_OK ||
            (s = valloc(D, &B.vpart, (size_t)dp::kBatchPowerChunks * (size_t)S)) != DP_OK ||
            (s = valloc(D, &B.vout, (size_t)S)) != DP_OK || (s = valloc(D, &B.vsp, (size_t)ns * (size_t)S)) != DP_OK ||
            (s = valloc(D, &B.vv0, (size_t)ns * (size_t)S)) != DP_OK) {
            free_list(B.vallocs, B.vbytes);
            return s;
        }
        B.vcap = S;
    }
    cudaError_t e = cudaSuccess;
    const float *spd = sp;
    if (!on_device) {
        if (ns) e = cudaMemcpyAsync(B.vsp, sp, sizeof(float) * (size_t)(ns * S), cudaMemcpyHostToDevice, st);
        spd = B.vsp;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "dp_virus_eval");
    uint8_t *v0d = on_device ? v0 : (v0 ? B.vv0 : nullptr);
    dp::launch_virus(D->d, D->ops, D->lvl_ptr.data(), spd, S, B.vwords, v0d, B.vpart, B.vout, st);
    dp_status s = launch_check(c, "dp_virus_eval");
    if (s != DP_OK) return s;
    if (on_device) {
        e = cudaMemcpyAsync(p_virus, B.vout, sizeof(double) * (size_t)S, cudaMemcpyDeviceToDevice, st);
        return cuda_err(c, e, "dp_virus_eval");
    }
    e = cudaMemcpyAsync(p_virus, B.vout, sizeof(double) * (size_t)S, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && v0 && ns) e = cudaMemcpyAsync(v0, B.vv0, (size_t)(ns * S), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_err(c, e, "dp_virus_eval");
    return check_device_error(c);
}

}  // extern "C"
