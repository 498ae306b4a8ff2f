// Request server: several designs resident on one GPU, analysis and gradient
// requests of any of them served by continuous batching.
//
// Each design has one request queue and one or more batch slots (one by
// default), each slot with its own copy of the design's device state, batch buffers and
// CUDA stream.  A worker thread takes the requests waiting for a design that
// has a free slot - up to max_batch of them, in arrival order - and runs them
// as the scenarios of one batched pass (forward, power, and the reverse pass
// when any of them wants gradients); batches of different designs, and the
// slots of one design, overlap on the device, so one batch's copies run beside
// the next batch's kernels.  Requests that arrive while every slot of their
// design is busy join the next batch.
// Admission: a design is accepted only while the device bytes it needs (the
// resident netlist plus its batch buffers for max_batch scenarios) fit in the
// server's HBM budget (for every slot of the design).
//
// A request carries either new startpoint SP/TR or the design's reference
// inputs, and optionally a sizing delta (new input pin caps of some cells,
// relative to the design's own caps).  Caps do not enter SP or TR, so a batch
// whose requests all use the reference inputs (sizing deltas) skips the forward
// pass: the forward state of the reference inputs, computed once when the
// design is added, is copied into every scenario column, and only the power and
// the reverse pass run (the columns are the ones the forward pass would write,
// bit for bit).  The delta enters the batch as a
// per-scenario change of C_load on the nets those cells load, so requests with
// different deltas share a batch.  Every (cell, scenario) is computed alone,
// by the same arithmetic in any launch shape, and the power sums of a scenario
// run in a fixed order, so a request's results do not depend on the requests
// it is batched with, nor on the batch size.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "capi_internal.h"
#include "compiled.h"

using namespace dpi;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    dp_request r{};
    uint64_t ticket = 0;
    double t_submit = 0, t_done = 0;
    int state = 0;                 // 0 queued, 1 in flight, 2 done
    dp_status status = DP_OK;
};

struct Design;

// One executor of a design: its device state, batch buffers, stream and graphs.
struct Slot {
    Design *des = nullptr;
    dp_ctx *ctx = nullptr;                  // owns this design's stream
    cudaStream_t stream = nullptr;
    dp_design *D = nullptr;
    int64_t ns = 0, nc = 0, nn = 0;
    float *d_ref_sp = nullptr, *d_ref_tr = nullptr;   // [ns]
    float2 *d_ref_pq = nullptr;                        // [nn] float-float P of the reference inputs
    float *d_in_sp = nullptr, *d_in_tr = nullptr;     // [max_batch][ns] request-major inputs
    float *d_dcl = nullptr;                            // [nn * max_batch], zero between batches
    // sizing-delta entries of a batch (capacity delta_cap, reserved at admission and grown in
    // stream order only when a batch brings more) and the device work arrays
    int64_t delta_cap = 0;
    int32_t *d_cell = nullptr;
    float *d_cap = nullptr;
    int64_t *d_list = nullptr;
    int32_t *h_off = nullptr, *d_off = nullptr;        // [max_batch + 1] entry offsets of the requests
    int *d_win = nullptr;                              // [nc * max_batch]
    float *d_dpin = nullptr;                           // [nc * max_batch]
    unsigned *d_flag = nullptr;                        // [nn * max_batch]
    unsigned long long *d_count = nullptr;
    double *h_power = nullptr;                         // [max_batch], pinned
    float *d_out_sp = nullptr, *d_out_tr = nullptr, *d_out_pin = nullptr;   // [max_batch][rows]
    cudaEvent_t done = nullptr;
    std::vector<std::array<cudaGraphExec_t, 4>> graphs;   // [log2 batch size][reverse pass + 2 reference inputs]
    std::vector<void *> dev, pinned;
    size_t bytes = 0;
    std::vector<Req *> inflight;
    bool busy = false;
    bool batch_ref = false;   // every request of the batch in flight is on the reference inputs
};

// A resident design: its request queue and the slots that serve it.
struct Design {
    int id = 0;
    int64_t ns = 0, nc = 0, nn = 0;
    size_t bytes = 0;            // device bytes of all its slots
    std::deque<Req *> queue;     // waiting requests, arrival order
    std::vector<Slot *> slots;
};

}  // namespace

struct dp_server {
    dp_server_config cfg{};
    dp_ctx *ctx = nullptr;                  // for allocation bookkeeping and messages
    std::vector<Design *> designs;
    std::vector<Slot *> slots;          // every slot of every design
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    std::thread worker;
    std::atomic<int64_t> queued{0};   // requests in the design queues (read by the worker without the lock)
    bool stop = false;
    size_t bytes_used = 0;
    dp_server_stats stats{};
    std::mutex emu;               // guards err (written by any submitting thread)
    std::string err;
};

namespace {

dp_status srv_err(dp_server *s, dp_status st, const std::string &m) {
    if (s) {
        std::lock_guard<std::mutex> lk(s->emu);
        s->err = m;
    }
    return st;
}

template <class T>
cudaError_t dmalloc(Slot *sl, T **p, size_t n) {
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess) {
        sl->dev.push_back(v);
        sl->bytes += sizeof(T) * (n ? n : 1);
    }
    *p = static_cast<T *>(v);
    return e;
}

template <class T>
cudaError_t hmalloc(Slot *sl, T **p, size_t n) {
    void *v = nullptr;
    cudaError_t e = cudaMallocHost(&v, sizeof(T) * (n ? n : 1));
    if (e == cudaSuccess) sl->pinned.push_back(v);
    *p = static_cast<T *>(v);
    return e;
}

void free_delta_arrays(Slot *sl, bool stream_ordered);

void free_slot(Slot *sl) {
    if (!sl) return;
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    free_delta_arrays(sl, false);
    for (void *p : sl->dev) cudaFree(p);
    for (void *p : sl->pinned) cudaFreeHost(p);
    if (sl->done) cudaEventDestroy(sl->done);
    for (auto &g : sl->graphs)
        for (cudaGraphExec_t x : g)
            if (x) cudaGraphExecDestroy(x);
    if (sl->D) dp_design_free(sl->D);
    if (sl->ctx) dp_destroy(sl->ctx);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    delete sl;
}

// bytes of device work arrays per sizing-delta entry: cell, cap, kMaxFanin claimed slots
constexpr int64_t kDeltaEntryBytes = 4 + 4 + 8 * dp::kMaxFanin;

// entries reserved at admission: max_batch requests that each resize 2 % of the cells
int64_t initial_delta_cap(int64_t max_batch, int64_t nc) {
    return std::max<int64_t>(4096, max_batch * std::max<int64_t>(1, nc / 50));
}

void free_delta_arrays(Slot *sl, bool stream_ordered) {
    for (void *p : {(void *)sl->d_cell, (void *)sl->d_cap, (void *)sl->d_list})
        if (p) {
            if (stream_ordered) cudaFreeAsync(p, sl->stream);
            else cudaFree(p);
        }
    sl->bytes -= (size_t)(kDeltaEntryBytes * sl->delta_cap);
    sl->d_cell = nullptr;
    sl->d_cap = nullptr;
    sl->d_list = nullptr;
    sl->delta_cap = 0;
}

// Room for the sizing-delta entries of one batch.  The arrays are reserved at admission;
// a batch that brings more entries grows them in stream order (cudaMallocAsync /
// cudaFreeAsync on the slot's stream), so the serving path never allocates pinned host
// memory, never waits for the device and never synchronises other streams.
cudaError_t ensure_delta_cap(Slot *sl, int64_t n, bool stream_ordered) {
    if (n <= sl->delta_cap) return cudaSuccess;
    int64_t cap = sl->delta_cap ? sl->delta_cap : 4096;
    while (cap < n) cap *= 2;
    if (sl->delta_cap) free_delta_arrays(sl, stream_ordered);
    cudaError_t e = cudaSuccess;
    void *a = nullptr, *b = nullptr, *c = nullptr;
    if (stream_ordered) {
        e = cudaMallocAsync(&a, sizeof(int32_t) * (size_t)cap, sl->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&b, sizeof(float) * (size_t)cap, sl->stream);
        if (e == cudaSuccess) e = cudaMallocAsync(&c, sizeof(int64_t) * (size_t)cap * dp::kMaxFanin, sl->stream);
    } else {
        e = cudaMalloc(&a, sizeof(int32_t) * (size_t)cap);
        if (e == cudaSuccess) e = cudaMalloc(&b, sizeof(float) * (size_t)cap);
        if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(int64_t) * (size_t)cap * dp::kMaxFanin);
    }
    sl->d_cell = static_cast<int32_t *>(a);
    sl->d_cap = static_cast<float *>(b);
    sl->d_list = static_cast<int64_t *>(c);
    sl->delta_cap = cap;
    sl->bytes += (size_t)(kDeltaEntryBytes * cap);
    if (e != cudaSuccess) free_delta_arrays(sl, stream_ordered);
    return e;
}

dp::SizingDeltas deltas_view(const Slot *sl, int32_t n_req) {
    return dp::SizingDeltas{sl->d_cell, sl->d_cap, sl->d_off, n_req, sl->d_win, sl->d_dpin,
                            sl->d_flag, sl->d_list, sl->d_count};
}

// Batch sizes run as graphs of a few fixed sizes: powers of two up to
// max_batch, and max_batch itself.
int64_t bucket_of(int64_t S, int64_t max_batch) {
    int64_t b = 1;
    while (b < S) b <<= 1;
    return b < max_batch ? b : max_batch;
}

int bucket_index(int64_t Sg) {
    int i = 0;
    while ((int64_t)1 << i < Sg) i++;
    return i;
}

// Captures the fixed part of a batch of Sg scenarios: inputs to scenario-innermost
// and the forward pass (or, on the reference inputs, their forward state copied into
// every column), power (copied to the pinned power buffer) and, with grad, the reverse
// pass and the outputs back to request-major.  The per-scenario C_load delta is
// always bound: where no request changed a cap it is zero, and C + 0 = C exactly.
cudaError_t capture_batch_graph(dp_server *srv, Slot *sl, int64_t Sg, bool grad, bool ref, cudaGraphExec_t *out) {
    dp_design *D = sl->D;
    dp_batch &B = D->batch;
    const dp_config &c = srv->cfg.analysis;
    const cudaStream_t st = sl->stream;
    const int64_t ns = sl->ns, nc = sl->nc;
    B.S = Sg;
    B.b.S = Sg;
    B.b.dcl = sl->d_dcl;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    if (ref) {
        dp::launch_bcast_ref(sl->d_ref_pq, sl->d_ref_tr, B.b.pq, B.b.tr_in, sl->nn, ns, Sg, st);
    } else {
        dp::launch_transpose(sl->d_in_sp, B.b.sp_in, Sg, ns, st);
        dp::launch_transpose(sl->d_in_tr, B.b.tr_in, Sg, ns, st);
        dp::launch_fwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), c.tr_mode, B.fwd_shape, st);
    }
    dp::launch_powerb(D->d, B.b, c.tr_mode, power_K(c), st);
    if (grad) {
        dp::launch_seedb(B.b, power_K(c), nullptr, st);
        dp::launch_bwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), c.tr_mode, B.bwd_shape, st);
        dp::launch_transpose(B.b.gsp, sl->d_out_sp, ns, Sg, st);
        dp::launch_gradb(D->d, B.b, D->ops, c.tr_mode, false, B.stage, nullptr, nullptr, st);
        dp::launch_transpose(B.stage, sl->d_out_tr, ns, Sg, st);
        dp::launch_gradb(D->d, B.b, D->ops, c.tr_mode, false, nullptr, B.stage, nullptr, st);
        dp::launch_transpose(B.stage, sl->d_out_pin, nc, Sg, st);
    }
    cudaMemcpyAsync(sl->h_power, B.b.power, sizeof(double) * (size_t)Sg, cudaMemcpyDeviceToHost, st);
    e = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    // upload now: the first launch of an executable graph otherwise uploads it, and the
    // worker would pay that (milliseconds for a large design's level chain) inside a batch
    if (e == cudaSuccess) e = cudaGraphUpload(*out, st);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Captures every batch graph of a design (four per batch size: with and without the
// reverse pass, on new or on the reference inputs).
cudaError_t capture_all(dp_server *srv, Slot *sl) {
    const int64_t m = srv->cfg.max_batch;
    for (int64_t Sg = 1;; Sg = Sg * 2 < m ? Sg * 2 : m) {
        const int i = bucket_index(Sg);
        for (int v = 0; v < 4; v++) {
            cudaError_t e = capture_batch_graph(srv, sl, Sg, (v & 1) != 0, (v & 2) != 0, &sl->graphs[(size_t)i][(size_t)v]);
            if (e != cudaSuccess) return e;
        }
        if (Sg == m) break;
    }
    return cudaSuccess;
}

// Queues one batch on the slot's stream: the requests' inputs and sizing deltas, the
// captured graph of the batch size, the gradients back into the requests' buffers.  Rows
// of a padded batch beyond the requests keep earlier (valid) inputs; their results are
// dropped.  Any CUDA error is returned; the requests are then failed by the caller.
cudaError_t launch_batch(dp_server *srv, Slot *sl) {
    const int64_t S = (int64_t)sl->inflight.size(), ns = sl->ns, nc = sl->nc;
    const int64_t Sg = bucket_of(S, srv->cfg.max_batch);
    const cudaStream_t st = sl->stream;
    cudaError_t e = cudaSuccess;
    bool grad = false;
    int64_t nd = 0;
    for (Req *q : sl->inflight) {
        grad = grad || q->r.want_grad;
        nd += q->r.n_delta;
    }
    for (int64_t s = 0; s < S && e == cudaSuccess && !sl->batch_ref; s++) {   // the batch runs the forward pass
        const Req *q = sl->inflight[(size_t)s];
        const bool own = q->r.sp != nullptr;
        if (ns) {
            e = cudaMemcpyAsync(sl->d_in_sp + s * ns, own ? (const void *)q->r.sp : (const void *)sl->d_ref_sp,
                                sizeof(float) * (size_t)ns, own ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sl->d_in_tr + s * ns, own ? (const void *)q->r.tr : (const void *)sl->d_ref_tr,
                                    sizeof(float) * (size_t)ns,
                                    own ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
        }
    }
    if (e != cudaSuccess) return e;
    if (nd) {   // the entries go to the device as given; the device resolves them (kern_serve.cu)
        if ((e = ensure_delta_cap(sl, nd, true)) != cudaSuccess) return e;
        int64_t off = 0;
        for (int64_t s = 0; s < S && e == cudaSuccess; s++) {
            const dp_request &r = sl->inflight[(size_t)s]->r;
            sl->h_off[s] = (int32_t)off;
            if (r.n_delta <= 0) continue;
            e = cudaMemcpyAsync(sl->d_cell + off, r.cells, sizeof(int32_t) * (size_t)r.n_delta,
                                cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sl->d_cap + off, r.pincap, sizeof(float) * (size_t)r.n_delta,
                                    cudaMemcpyHostToDevice, st);
            off += r.n_delta;
        }
        sl->h_off[S] = (int32_t)off;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl->d_off, sl->h_off, sizeof(int32_t) * (size_t)(S + 1), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        dp::launch_sizing_deltas(sl->D->d, sl->D->ops, deltas_view(sl, (int32_t)S), nd, Sg, sl->d_dcl, st);
    }
    e = cudaGraphLaunch(sl->graphs[(size_t)bucket_index(Sg)][(grad ? 1 : 0) + (sl->batch_ref ? 2 : 0)], st);
    if (e != cudaSuccess) return e;
    if (grad)
        for (int64_t s = 0; s < S && e == cudaSuccess; s++) {
            const dp_request &r = sl->inflight[(size_t)s]->r;
            if (!r.want_grad) continue;
            if (r.grad_sp && ns)
                e = cudaMemcpyAsync(r.grad_sp, sl->d_out_sp + s * ns, sizeof(float) * (size_t)ns,
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && r.grad_tr && ns)
                e = cudaMemcpyAsync(r.grad_tr, sl->d_out_tr + s * ns, sizeof(float) * (size_t)ns,
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && r.grad_pincap && nc)
                e = cudaMemcpyAsync(r.grad_pincap, sl->d_out_pin + s * nc, sizeof(float) * (size_t)nc,
                                    cudaMemcpyDeviceToHost, st);
        }
    if (e != cudaSuccess) return e;
    if (nd) dp::launch_sizing_clear(sl->D->d, deltas_view(sl, (int32_t)S), nd, Sg, sl->d_dcl, st);   // back to rest
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaEventRecord(sl->done, st);
}

// The batch finished (or failed): outputs into the requests, requests done.
void complete_batch(dp_server *srv, Slot *sl, dp_status status) {
    const double t = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    for (size_t s = 0; s < sl->inflight.size(); s++) {
        Req *q = sl->inflight[s];
        if (status == DP_OK && q->r.power) *q->r.power = sl->h_power[s];
        q->status = status;
        q->t_done = t;
        q->state = 2;
    }
    srv->stats.batches += 1;
    srv->stats.requests += (int64_t)sl->inflight.size();
    if ((int64_t)sl->inflight.size() > srv->stats.max_batch_seen) srv->stats.max_batch_seen = (int64_t)sl->inflight.size();
    sl->inflight.clear();
    sl->busy = false;
    srv->cv_done.notify_all();
}

// Takes the next batch of a free slot (lock held): up to max_batch requests waiting for
// its design, in arrival order.
bool take_batch(dp_server *srv, Slot *sl) {
    std::deque<Req *> &queue = sl->des->queue;
    if (sl->busy || queue.empty()) return false;
    const size_t m = (size_t)srv->cfg.max_batch;
    bool ref = true;
    while (!queue.empty() && sl->inflight.size() < m) {
        Req *q = queue.front();
        queue.pop_front();
        q->state = 1;
        ref = ref && q->r.sp == nullptr;
        sl->inflight.push_back(q);
    }
    sl->batch_ref = ref;
    sl->busy = true;
    return true;
}

// a failed batch may have left sizing deltas behind: clear them all
void reset_after_failure(Slot *sl) {
    cudaGetLastError();
    cudaStreamSynchronize(sl->stream);
    const size_t S = (size_t)sl->D->batch.cap;
    cudaMemsetAsync(sl->d_dcl, 0, sizeof(float) * (size_t)sl->nn * S, sl->stream);
    cudaMemsetAsync(sl->d_flag, 0, sizeof(unsigned) * (size_t)sl->nn * S, sl->stream);
    cudaMemsetAsync(sl->d_dpin, 0, sizeof(float) * (size_t)sl->nc * S, sl->stream);
    cudaMemsetAsync(sl->d_win, 0xFF, sizeof(int) * (size_t)sl->nc * S, sl->stream);
    cudaStreamSynchronize(sl->stream);
    cudaGetLastError();
    sl->D->batch.b.dcl = nullptr;
}

void run_and_complete(dp_server *srv, Slot *sl) {
    DeviceGuard g(srv->cfg.device);
    const double t0 = now_s();
    cudaError_t e = launch_batch(srv, sl);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stats.host_launch_s += now_s() - t0;
    }
    if (e != cudaSuccess) {
        reset_after_failure(sl);
        complete_batch(srv, sl, DP_ECUDA);
    }
}

// The worker owns the batches in flight (busy, inflight, the events): it polls
// them without the lock, and takes the lock only to move queued requests into
// new batches or to mark a finished batch's requests done.
void worker_main(dp_server *srv) {
    DeviceGuard g(srv->cfg.device);
    std::vector<Slot *> launch, slots;
    for (;;) {
        launch.clear();
        bool inflight = false;
        for (Slot *sl : slots) inflight = inflight || sl->busy;
        if (srv->queued.load(std::memory_order_acquire) > 0 || !inflight) {
            std::unique_lock<std::mutex> lk(srv->mu);
            slots = srv->slots;   // designs may be added meanwhile
            for (Slot *sl : slots)
                if (take_batch(srv, sl)) {
                    srv->queued.fetch_sub((int64_t)sl->inflight.size(), std::memory_order_acq_rel);
                    launch.push_back(sl);
                }
            inflight = false;
            for (Slot *sl : slots) inflight = inflight || sl->busy;
            if (launch.empty() && !inflight) {
                if (srv->stop) return;
                srv->cv_work.wait(lk);
                continue;
            }
        }
        for (Slot *sl : launch) run_and_complete(srv, sl);
        bool any_done = false;
        for (Slot *sl : slots) {
            if (!sl->busy || sl->inflight.empty()) continue;
            const cudaError_t q = cudaEventQuery(sl->done);
            if (q == cudaSuccess) {
                complete_batch(srv, sl, DP_OK);
                any_done = true;
            } else if (q != cudaErrorNotReady) {
                reset_after_failure(sl);
                complete_batch(srv, sl, DP_ECUDA);
                any_done = true;
            }
        }
        if (launch.empty() && !any_done) std::this_thread::yield();
    }
}

// validates a request against its design's sizes (design found under the lock; the
// checks themselves run outside it, since resident designs are never removed)
dp_status check_request(dp_server *srv, const dp_request *r, Design **out) {
    if (!r) return srv_err(srv, DP_EINVAL, "NULL request");
    Design *sl = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (r->design < 0 || (size_t)r->design >= srv->designs.size())
            return srv_err(srv, DP_EINVAL, "unknown design id " + std::to_string(r->design));
        sl = srv->designs[(size_t)r->design];
    }
    if ((r->sp == nullptr) != (r->tr == nullptr)) return srv_err(srv, DP_EINVAL, "give both sp and tr, or neither");
    if (r->sp) {   // branch-free scans (NaN fails every comparison)
        int bad = 0;
        for (int64_t k = 0; k < sl->ns; k++)
            bad |= !(r->sp[k] >= 0.f) | !(r->sp[k] <= 1.f) | !(r->tr[k] >= 0.f) | !(r->tr[k] <= 1.f);
        if (bad) return srv_err(srv, DP_EINVAL, "input SP and TR must lie in [0,1]");
    }
    if (r->n_delta < 0 || (r->n_delta > 0 && (!r->cells || !r->pincap)))
        return srv_err(srv, DP_EINVAL, "bad sizing delta");
    int bad = 0;
    const int32_t nc = (int32_t)sl->nc;
    for (int32_t i = 0; i < r->n_delta; i++)
        bad |= (r->cells[i] < 0) | (r->cells[i] >= nc) | !(r->pincap[i] >= 0.f) | !(r->pincap[i] < 1e30f);
    if (bad) return srv_err(srv, DP_EINVAL, "sizing delta: cell index or pin cap out of range");
    if (!r->power) return srv_err(srv, DP_EINVAL, "NULL power output");
    *out = sl;
    return DP_OK;
}

}  // namespace

extern "C" {

void dp_server_config_default(dp_server_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->device = 0;
    c->max_batch = 64;
    c->hbm_budget = 0;
    c->plain = 0;
    dp_config_default(&c->analysis);
    c->analysis.grad_mode = 0;
    c->slots_per_design = 1;
}

const char *dp_server_last_error(const dp_server *s) { return s ? s->err.c_str() : "NULL server"; }

dp_status dp_server_create(const dp_server_config *cfg, dp_server **out) {
    if (!cfg || !out) return DP_EINVAL;
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > 4096) return DP_EINVAL;
    if (cfg->slots_per_design < 0 || cfg->slots_per_design > 8) return DP_EINVAL;
    if (cfg->analysis.grad_mode != 0 || cfg->analysis.tr_mode < 0 || cfg->analysis.tr_mode > 1) return DP_EINVAL;
    dp_server *s = new (std::nothrow) dp_server();
    if (!s) return DP_ENOMEM;
    s->cfg = *cfg;
    if (s->cfg.slots_per_design == 0) s->cfg.slots_per_design = 1;
    if (s->cfg.plain) {
        s->cfg.max_batch = 1;
        s->cfg.slots_per_design = 1;
    }
    dp_status st = dp_create(cfg->device, nullptr, &s->ctx);
    if (st != DP_OK) {
        delete s;
        return st;
    }
    if (dp_status e = check_cfg(s->ctx, &s->cfg.analysis); e != DP_OK) {
        dp_destroy(s->ctx);
        delete s;
        return e;
    }
    if (s->cfg.hbm_budget == 0) {
        DeviceGuard g(cfg->device);
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) s->cfg.hbm_budget = fr / 10 * 8;
        else cudaGetLastError();
    }
    if (!s->cfg.plain) s->worker = std::thread(worker_main, s);
    *out = s;
    return DP_OK;
}

void dp_server_destroy(dp_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Slot *sl : s->slots) free_slot(sl);
    for (Design *d : s->designs) delete d;
    for (auto &kv : s->reqs) delete kv.second;
    if (s->ctx) dp_destroy(s->ctx);
    delete s;
}

}  // extern "C"

namespace {

// Builds one slot of a design from its compiled netlist (which stays the caller's):
// device state, batch buffers, tuned shapes, the reference inputs' forward state and
// the batch graphs.  On failure the slot is freed and the error recorded.
dp_status make_slot(dp_server *srv, const dp_compiled *cp, const float *ref_sp, const float *ref_tr, Slot **out) {
    *out = nullptr;
    const int64_t ns = cp->n_start, nc = cp->n_cells, nn = cp->n_nets;
    const int64_t S = srv->cfg.max_batch;
    dp_status st = DP_OK;
    Slot *sl = new (std::nothrow) Slot();
    if (!sl) return srv_err(srv, DP_ENOMEM, "out of host memory");
    sl->ns = ns;
    sl->nc = nc;
    sl->nn = nn;
    // stream priority by size: a small design's short batches are scheduled ahead of a large
    // design's long ones when both wait for SMs (arithmetic and results are unaffected)
    int lo_prio = 0, hi_prio = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) {
        cudaGetLastError();
        lo_prio = hi_prio = 0;
    }
    const int span = lo_prio - hi_prio;   // greatest priority is the most negative number
    const int rank = nc < 100000 ? 0 : (nc < 1000000 ? 1 : 2);
    const int prio = span > 0 ? hi_prio + (rank * span) / 2 : 0;
    cudaError_t e = cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_slot(sl);
        return srv_err(srv, DP_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    st = dp_create(srv->cfg.device, sl->stream, &sl->ctx);
    if (st == DP_OK) st = dp_design_upload(sl->ctx, cp, &sl->D);
    if (st != DP_OK) {
        srv_err(srv, st, sl->ctx ? dp_last_error(sl->ctx) : "context");
        free_slot(sl);
        return st;
    }
    dp_design *D = sl->D;
    if ((st = batch_reserve(D, S)) != DP_OK) {
        srv_err(srv, st, dp_last_error(sl->ctx));
        free_slot(sl);
        return st;
    }
    e = dmalloc(sl, &sl->d_ref_sp, (size_t)ns);
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_ref_tr, (size_t)ns);
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_in_sp, (size_t)(ns * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_in_tr, (size_t)(ns * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_dcl, (size_t)(nn * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_out_sp, (size_t)(ns * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_out_tr, (size_t)(ns * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_out_pin, (size_t)(nc * S));
    if (e == cudaSuccess) e = hmalloc(sl, &sl->h_power, (size_t)S);
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_win, (size_t)(nc * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_dpin, (size_t)(nc * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_flag, (size_t)(nn * S));
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_count, 1);
    if (e == cudaSuccess) e = dmalloc(sl, &sl->d_off, (size_t)(S + 1));
    if (e == cudaSuccess) e = hmalloc(sl, &sl->h_off, (size_t)(S + 1));
    if (e == cudaSuccess) e = ensure_delta_cap(sl, initial_delta_cap(S, nc), false);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl->d_dcl, 0, sizeof(float) * (size_t)(nn * S), sl->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl->d_win, 0xFF, sizeof(int) * (size_t)(nc * S), sl->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl->d_dpin, 0, sizeof(float) * (size_t)(nc * S), sl->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl->d_flag, 0, sizeof(unsigned) * (size_t)(nn * S), sl->stream);
    if (e == cudaSuccess && ns) {
        std::vector<float> sp(ref_sp ? ref_sp : nullptr, ref_sp ? ref_sp + ns : nullptr);
        std::vector<float> tr(ref_tr ? ref_tr : nullptr, ref_tr ? ref_tr + ns : nullptr);
        if (!ref_sp) sp.assign((size_t)ns, 0.5f);
        if (!ref_tr) tr.assign((size_t)ns, 0.25f);
        for (int64_t k = 0; k < ns; k++)
            if (!(sp[(size_t)k] >= 0.f && sp[(size_t)k] <= 1.f && tr[(size_t)k] >= 0.f && tr[(size_t)k] <= 1.f)) {
                free_slot(sl);
                return srv_err(srv, DP_EINVAL, "reference SP and TR must lie in [0,1]");
            }
        e = cudaMemcpy(sl->d_ref_sp, sp.data(), sizeof(float) * (size_t)ns, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(sl->d_ref_tr, tr.data(), sizeof(float) * (size_t)ns, cudaMemcpyHostToDevice);
        // the tuner times full batches of the reference inputs, then the shapes stay fixed
        for (int64_t s = 0; s < S && e == cudaSuccess; s++) {
            e = cudaMemcpyAsync(sl->d_in_sp + s * ns, sl->d_ref_sp, sizeof(float) * (size_t)ns,
                                cudaMemcpyDeviceToDevice, sl->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sl->d_in_tr + s * ns, sl->d_ref_tr, sizeof(float) * (size_t)ns,
                                    cudaMemcpyDeviceToDevice, sl->stream);
        }
    }
    if (e == cudaSuccess) {
        dp_batch &B = D->batch;
        B.S = S;
        B.b.S = S;
        dp::launch_transpose(sl->d_in_sp, B.b.sp_in, S, ns, sl->stream);
        dp::launch_transpose(sl->d_in_tr, B.b.tr_in, S, ns, sl->stream);
        e = cudaStreamSynchronize(sl->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_slot(sl);
        return srv_err(srv, DP_ECUDA, std::string("server buffers: ") + cudaGetErrorString(e));
    }
    if ((st = batch_tune_and_lock(D)) != DP_OK) {
        srv_err(srv, st, dp_last_error(sl->ctx));
        free_slot(sl);
        return st;
    }
    // the forward state of the reference inputs, for batches that use them: one column
    e = dmalloc(sl, &sl->d_ref_pq, (size_t)nn);
    if (e == cudaSuccess) {
        dp_batch &B = D->batch;
        B.S = 1;
        B.b.S = 1;
        if (ns) e = cudaMemcpyAsync(B.b.sp_in, sl->d_ref_sp, sizeof(float) * (size_t)ns, cudaMemcpyDeviceToDevice, sl->stream);
        if (e == cudaSuccess && ns)
            e = cudaMemcpyAsync(B.b.tr_in, sl->d_ref_tr, sizeof(float) * (size_t)ns, cudaMemcpyDeviceToDevice, sl->stream);
        if (e == cudaSuccess) {
            dp::launch_fwdb(D->d, B.b, D->ops, D->lvl_ptr.data(), srv->cfg.analysis.tr_mode, B.fwd_shape, sl->stream);
            e = cudaMemcpyAsync(sl->d_ref_pq, B.b.pq, sizeof(float2) * (size_t)nn, cudaMemcpyDeviceToDevice, sl->stream);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(sl->stream);
    }
    if (e == cudaSuccess) {
        sl->graphs.assign((size_t)bucket_index(S) + 1, std::array<cudaGraphExec_t, 4>{nullptr, nullptr, nullptr, nullptr});
        e = capture_all(srv, sl);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sl->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_slot(sl);
        return srv_err(srv, DP_ECUDA, std::string("batch graphs: ") + cudaGetErrorString(e));
    }
    sl->bytes += D->bytes + D->batch.bytes;
    *out = sl;
    return DP_OK;
}

}  // namespace

extern "C" {

dp_status dp_server_add_design(dp_server *srv, const char *netlist, size_t netlist_len, const char *library,
                               size_t library_len, const float *ref_sp, const float *ref_tr, int32_t *id) {
    if (!srv || !netlist || !library || !id) return srv_err(srv, DP_EINVAL, "NULL argument");
    DeviceGuard g(srv->cfg.device);
    dp_compiled *cp = nullptr;
    char msg[512] = {0};
    dp_status st = dp_compile(netlist, netlist_len, library, library_len, &cp, msg, sizeof msg);
    if (st != DP_OK) return srv_err(srv, st, std::string("compile: ") + msg);
    const int64_t ns = cp->n_start, nc = cp->n_cells, nn = cp->n_nets, ne = cp->n_edges;
    const int64_t S = srv->cfg.max_batch;
    const int nslots = srv->cfg.slots_per_design;
    // device bytes per slot: resident netlist (about 24 B per net, 40 per cell, 8 per edge) and
    // batch buffers
    const double need = 24.0 * nn + 40.0 * nc + 8.0 * ne + 72.0 * nn +
                        (double)S * (8.0 * nn + 4.0 * ne + 16.0 * ns + 4.0 * nn + 4.0 * std::max(nn, nc) +
                                     4.0 * (2 * ns + nc) + 8.0 * ns + 8.0 * dp::kBatchPowerChunks + 8.0 * nc +
                                     4.0 * nn) +
                        (double)(kDeltaEntryBytes * initial_delta_cap(S, nc));
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if ((double)srv->bytes_used + nslots * need > (double)srv->cfg.hbm_budget) {
            dp_compiled_free(cp);
            return srv_err(srv, DP_ENOMEM, "HBM budget: the design needs about " +
                                               std::to_string((long long)(nslots * need)) + " bytes, " +
                                               std::to_string((long long)(srv->cfg.hbm_budget - srv->bytes_used)) +
                                               " left");
        }
    }
    Design *des = new (std::nothrow) Design();
    if (!des) {
        dp_compiled_free(cp);
        return srv_err(srv, DP_ENOMEM, "out of host memory");
    }
    des->ns = ns;
    des->nc = nc;
    des->nn = nn;
    size_t charged = 0;
    for (int k = 0; k < nslots && st == DP_OK; k++) {
        Slot *sl = nullptr;
        st = make_slot(srv, cp, ref_sp, ref_tr, &sl);
        if (st != DP_OK) break;
        sl->des = des;
        des->slots.push_back(sl);
        des->bytes += sl->bytes;
        charged += (size_t)std::max(need, (double)sl->bytes);
    }
    dp_compiled_free(cp);
    if (st != DP_OK) {
        for (Slot *sl : des->slots) free_slot(sl);
        delete des;
        return st;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    des->id = (int)srv->designs.size();
    srv->designs.push_back(des);
    for (Slot *sl : des->slots) srv->slots.push_back(sl);
    srv->bytes_used += charged;
    *id = des->id;
    return DP_OK;
}

dp_status dp_server_design_info(dp_server *srv, int32_t id, dp_info *info) {
    if (!srv || !info) return DP_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (id < 0 || (size_t)id >= srv->designs.size()) return srv_err(srv, DP_EINVAL, "unknown design id");
    const Design *des = srv->designs[(size_t)id];
    dp_status st = dp_design_info(des->slots[0]->D, info);
    info->device_bytes = des->bytes;
    return st;
}

dp_status dp_server_submit(dp_server *srv, const dp_request *r, uint64_t *ticket) {
    if (!srv || !ticket) return DP_EINVAL;
    Design *des = nullptr;
    const dp_status st = check_request(srv, r, &des);
    if (st != DP_OK) return st;
    Req *q = new (std::nothrow) Req();
    if (!q) return srv_err(srv, DP_ENOMEM, "out of host memory");
    q->r = *r;
    q->t_submit = now_s();
    if (srv->cfg.plain) {   // one request at a time on the calling thread
        Slot *sl = des->slots[0];
        std::unique_lock<std::mutex> lk(srv->mu);
        q->ticket = srv->next_ticket++;
        srv->reqs[q->ticket] = q;
        sl->inflight.push_back(q);
        q->state = 1;
        sl->batch_ref = r->sp == nullptr;
        sl->busy = true;
        lk.unlock();
        DeviceGuard g(srv->cfg.device);
        const double t0 = now_s();
        cudaError_t e = launch_batch(srv, sl);
        {
            std::lock_guard<std::mutex> lk2(srv->mu);
            srv->stats.host_launch_s += now_s() - t0;
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(sl->done);
        if (e != cudaSuccess) reset_after_failure(sl);
        complete_batch(srv, sl, e == cudaSuccess ? DP_OK : DP_ECUDA);
        *ticket = q->ticket;
        return DP_OK;
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        q->ticket = srv->next_ticket++;
        srv->reqs[q->ticket] = q;
        des->queue.push_back(q);
        *ticket = q->ticket;
        srv->queued.fetch_add(1, std::memory_order_acq_rel);
    }
    srv->cv_work.notify_one();
    return DP_OK;
}

dp_status dp_server_submit_many(dp_server *srv, const dp_request *reqs, int32_t n, uint64_t *tickets) {
    if (!srv || n < 0 || (n > 0 && (!reqs || !tickets))) return DP_EINVAL;
    if (srv->cfg.plain) {
        for (int32_t i = 0; i < n; i++) {
            const dp_status st = dp_server_submit(srv, &reqs[i], &tickets[i]);
            if (st != DP_OK) return st;
        }
        return DP_OK;
    }
    std::vector<Design *> des((size_t)n, nullptr);
    for (int32_t i = 0; i < n; i++) {
        const dp_status st = check_request(srv, &reqs[i], &des[(size_t)i]);
        if (st != DP_OK) {
            std::lock_guard<std::mutex> lk(srv->emu);
            srv->err = "request " + std::to_string(i) + ": " + srv->err;
            return st;
        }
    }
    std::vector<Req *> qs((size_t)n, nullptr);
    for (int32_t i = 0; i < n; i++) {
        qs[(size_t)i] = new (std::nothrow) Req();
        if (!qs[(size_t)i]) {
            for (Req *q : qs) delete q;
            return srv_err(srv, DP_ENOMEM, "out of host memory");
        }
    }
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (int32_t i = 0; i < n; i++) {
            Req *q = qs[(size_t)i];
            q->r = reqs[i];
            q->t_submit = t;
            q->ticket = srv->next_ticket++;
            srv->reqs[q->ticket] = q;
            des[(size_t)i]->queue.push_back(q);
            tickets[i] = q->ticket;
        }
        srv->queued.fetch_add(n, std::memory_order_acq_rel);
    }
    srv->cv_work.notify_one();
    return DP_OK;
}

dp_status dp_server_wait(dp_server *srv, uint64_t ticket, double timeout_s, double *latency_ms) {
    if (!srv) return DP_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return srv_err(srv, DP_EINVAL, "unknown ticket");
    Req *q = it->second;
    const auto pred = [q] { return q->state == 2; };
    if (timeout_s > 0) {
        if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
            return srv_err(srv, DP_ETIMEOUT, "request not finished within the timeout");
    } else {
        srv->cv_done.wait(lk, pred);
    }
    if (latency_ms) *latency_ms = 1e3 * (q->t_done - q->t_submit);
    const dp_status st = q->status;
    srv->reqs.erase(it);
    delete q;
    if (st != DP_OK) return srv_err(srv, st, "the request's batch failed on the device");
    return DP_OK;
}

dp_status dp_server_get_stats(dp_server *srv, dp_server_stats *out) {
    if (!srv || !out) return DP_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->device_bytes = srv->bytes_used;
    out->designs = (int32_t)srv->designs.size();
    return DP_OK;
}

}  // extern "C"
