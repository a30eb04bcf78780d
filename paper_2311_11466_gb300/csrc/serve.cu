// Batching and serving runtime (include/ptycho_serve.h): many reconstructions
// of the generalised divide-and-concur update on one GPU.
//
// Batch: the contexts' steady-state iteration (re-split prologue, divide,
// concur) is captured once into a CUDA graph with one branch per context
// (fork and join through events on a private stream) and replayed; the first
// iteration, which may start from loaded exit waves, runs directly.
//
// Server: FIFO admission under an HBM budget, a bounded active set, rounds of
// a few iterations of every active request launched concurrently on the
// requests' own streams, and retirement with result copy-back.  New requests
// join between rounds (continuous batching); a finished request frees its
// memory and slot for the next one in the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ptycho.h"
#include "../../include/ptycho_serve.h"
#include "internal.h"
#include "nvtx.h"

using Clock = std::chrono::steady_clock;

namespace {

struct BatchEntry {
    ptycho_ctx* ctx;
    float a, b, c;
};

double seconds(Clock::time_point t0, Clock::time_point t1) {
    return std::chrono::duration<double>(t1 - t0).count();
}

}  // namespace

struct ptycho_batch {
    ptycho_opts opts{};
    std::vector<BatchEntry> e;
    cudaStream_t main = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

extern "C" int ptycho_batch_create(ptycho_batch** out, const ptycho_opts* opts) {
    if (!out) return PTYCHO_EINVAL;
    *out = nullptr;
    ptycho_opts o;
    ptycho_default_opts(&o);
    if (opts) o = *opts;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(o.device) != cudaSuccess) return PTYCHO_EINVAL;
    auto* b = new ptycho_batch();
    b->opts = o;
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaSetDevice(prev);
        delete b;
        return PTYCHO_ECUDA;
    }
    cudaSetDevice(prev);
    *out = b;
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_add(ptycho_batch* b, ptycho_ctx* ctx, float a, float bb, float c) {
    if (!b || !ctx) return PTYCHO_EINVAL;
    if (!std::isfinite(a) || !std::isfinite(bb) || !std::isfinite(c)) return PTYCHO_EINVAL;
    if (!ptycho::ctx_loaded(ctx)) return PTYCHO_ESTATE;
    if (ptycho::ctx_device(ctx) != b->opts.device) return PTYCHO_EINVAL;
    b->e.push_back({ctx, a, bb, c});
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_run(ptycho_batch* b, int32_t n_iter) {
    NvtxRange nvtx_range("ptycho_batch_run");
    if (!b || n_iter < 0) return PTYCHO_EINVAL;
    if (b->e.empty()) return PTYCHO_ESTATE;
    if (n_iter == 0) return PTYCHO_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->opts.device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};

    // first iteration directly (contexts may start from loaded exit waves)
    for (auto& en : b->e) {
        int rc = ptycho_iterate(en.ctx, en.a, en.b, en.c, 1);
        if (rc) return rc;
    }
    if (n_iter == 1) {
        for (auto& en : b->e)
            if (cudaStreamSynchronize(ptycho::ctx_stream(en.ctx)) != cudaSuccess) return PTYCHO_ECUDA;
        return PTYCHO_OK;
    }
    while (b->join.size() < b->e.size()) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return PTYCHO_ECUDA;
        b->join.push_back(ev);
    }
    // the main stream starts after every context's first iteration
    for (size_t i = 0; i < b->e.size(); ++i) {
        if (cudaEventRecord(b->join[i], ptycho::ctx_stream(b->e[i].ctx)) != cudaSuccess ||
            cudaStreamWaitEvent(b->main, b->join[i], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
    }
    // capture one steady-state iteration of every context
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return PTYCHO_ECUDA;
    int rc = PTYCHO_OK;
    cudaEventRecord(b->fork, b->main);
    for (size_t i = 0; i < b->e.size() && rc == PTYCHO_OK; ++i) {
        cudaStream_t s = ptycho::ctx_stream(b->e[i].ctx);
        cudaStreamWaitEvent(s, b->fork, 0);
        rc = ptycho_iterate(b->e[i].ctx, b->e[i].a, b->e[i].b, b->e[i].c, 1);
        cudaEventRecord(b->join[i], s);
        cudaStreamWaitEvent(b->main, b->join[i], 0);
    }
    cudaError_t ce = cudaStreamEndCapture(b->main, &graph);
    if (rc != PTYCHO_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc != PTYCHO_OK ? rc : PTYCHO_ECUDA;
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return PTYCHO_ECUDA;
    // the capture recorded one iteration per context without running it;
    // n_iter - 1 replays run iterations 2 .. n_iter
    for (int it = 1; it < n_iter && ce == cudaSuccess; ++it) ce = cudaGraphLaunch(exec, b->main);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->main);
    cudaGraphExecDestroy(exec);
    if (ce != cudaSuccess) return PTYCHO_ECUDA;
    for (auto& en : b->e) ptycho::ctx_add_iterations(en.ctx, n_iter - 2);
    return PTYCHO_OK;
}

extern "C" void ptycho_batch_destroy(ptycho_batch* b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->opts.device);
    cudaStreamSynchronize(b->main);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    cudaEventDestroy(b->fork);
    cudaStreamDestroy(b->main);
    cudaSetDevice(prev);
    delete b;
}

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------

namespace {

struct Request {
    uint64_t id = 0;
    int32_t J = 0, N = 0, Mr = 0, Mc = 0;
    std::vector<int32_t> pos;
    std::vector<float> inten, obj0, probe0;
    float a = 1, b = 1, c = 1;
    int32_t n_iter = 0, done_iter = 0;
    int32_t state = PTYCHO_REQ_QUEUED;
    ptycho_ctx* ctx = nullptr;
    size_t bytes = 0;
    Clock::time_point t_submit, t_admit, t_done;
    std::vector<float> obj_out, probe_out;
    double final_err = 0.0;
};

}  // namespace

struct ptycho_server {
    ptycho_opts opts{};
    size_t budget = 0;
    int32_t max_active = 1;
    size_t used = 0;
    uint64_t next_id = 1;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
};

extern "C" int ptycho_server_create(ptycho_server** out, size_t budget, int32_t max_active,
                                    const ptycho_opts* opts) {
    if (!out || budget == 0 || max_active < 1) return PTYCHO_EINVAL;
    *out = nullptr;
    auto* s = new ptycho_server();
    ptycho_default_opts(&s->opts);
    if (opts) s->opts = *opts;
    s->opts.stream = nullptr;  // every request gets a private stream
    s->budget = budget;
    s->max_active = max_active;
    *out = s;
    return PTYCHO_OK;
}

extern "C" int ptycho_server_submit(ptycho_server* s, const ptycho_scan_desc* d, float a, float b,
                                    float c, int32_t n_iter, uint64_t* req_id) {
    if (!s || !d || !req_id || n_iter < 0) return PTYCHO_EINVAL;
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c)) return PTYCHO_EINVAL;
    if (d->J < 1 || d->N < 1 || d->M_rows < d->N || d->M_cols < d->N || !d->pos_rc ||
        !d->intensity || !d->obj0 || !d->probe0)
        return PTYCHO_EINVAL;
    const size_t need = ptycho_scan_bytes(d->J, d->N, d->M_rows, d->M_cols, s->opts.precision);
    if (need == 0 || need > s->budget) return PTYCHO_EINVAL;
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->J = d->J;
    r->N = d->N;
    r->Mr = d->M_rows;
    r->Mc = d->M_cols;
    const size_t NN = (size_t)d->N * d->N, M = (size_t)d->M_rows * d->M_cols;
    r->pos.assign(d->pos_rc, d->pos_rc + 2 * (size_t)d->J);
    r->inten.assign(d->intensity, d->intensity + (size_t)d->J * NN);
    r->obj0.assign(d->obj0, d->obj0 + 2 * M);
    r->probe0.assign(d->probe0, d->probe0 + 2 * NN);
    r->a = a;
    r->b = b;
    r->c = c;
    r->n_iter = n_iter;
    r->bytes = need;
    r->t_submit = Clock::now();
    *req_id = r->id;
    s->queue.push_back(r.get());
    s->all[r->id] = std::move(r);
    return PTYCHO_OK;
}

namespace {

void retire(ptycho_server* s, Request* r) {
    const size_t M = (size_t)r->Mr * r->Mc, NN = (size_t)r->N * r->N;
    r->obj_out.resize(2 * M);
    r->probe_out.resize(2 * NN);
    int rc = ptycho_get_object_probe(r->ctx, r->obj_out.data(), r->probe_out.data());
    if (rc == PTYCHO_OK) rc = ptycho_model_error(r->ctx, &r->final_err);
    ptycho_destroy(r->ctx);
    r->ctx = nullptr;
    s->used -= r->bytes;
    r->t_done = Clock::now();
    r->state = rc == PTYCHO_OK ? PTYCHO_REQ_DONE : PTYCHO_REQ_FAILED;
}

}  // namespace

extern "C" int ptycho_server_step(ptycho_server* s, int32_t iters_per_round, int32_t* n_active,
                                  int32_t* n_queued) {
    NvtxRange nvtx_range("ptycho_server_step");
    if (!s || iters_per_round < 1) return PTYCHO_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->opts.device);
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};

    // admission, in arrival order
    while (!s->queue.empty() && (int32_t)s->active.size() < s->max_active) {
        Request* r = s->queue.front();
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PTYCHO_ECUDA;
        const size_t margin = (size_t)1 << 30;
        if (s->used + r->bytes > s->budget || r->bytes + margin > free_b) break;
        s->queue.pop_front();
        ptycho_ctx* ctx = nullptr;
        int rc = ptycho_create(&ctx, &s->opts);
        if (rc == PTYCHO_OK)
            rc = ptycho_load_scan(ctx, r->J, r->N, r->pos.data(), r->inten.data(), r->Mr, r->Mc,
                                  r->obj0.data(), r->probe0.data(), 0);
        if (rc != PTYCHO_OK) {
            if (ctx) ptycho_destroy(ctx);
            r->state = PTYCHO_REQ_FAILED;
            r->t_done = Clock::now();
            continue;
        }
        r->ctx = ctx;
        r->state = PTYCHO_REQ_ACTIVE;
        r->t_admit = Clock::now();
        s->used += r->bytes;
        // the scan now lives on the device
        std::vector<float>().swap(r->inten);
        std::vector<float>().swap(r->obj0);
        std::vector<int32_t>().swap(r->pos);
        std::vector<float>().swap(r->probe0);
        s->active.push_back(r);
    }

    // one round: every active request advances concurrently on its own stream
    for (Request* r : s->active) {
        const int32_t k = std::min(iters_per_round, r->n_iter - r->done_iter);
        if (k > 0) {
            int rc = ptycho_iterate(r->ctx, r->a, r->b, r->c, k);
            if (rc != PTYCHO_OK) return rc;
            r->done_iter += k;
        }
    }
    for (Request* r : s->active)
        if (cudaStreamSynchronize(ptycho::ctx_stream(r->ctx)) != cudaSuccess) return PTYCHO_ECUDA;

    // retirement
    std::vector<Request*> still;
    for (Request* r : s->active) {
        if (r->done_iter >= r->n_iter)
            retire(s, r);
        else
            still.push_back(r);
    }
    s->active.swap(still);
    if (n_active) *n_active = (int32_t)s->active.size();
    if (n_queued) *n_queued = (int32_t)s->queue.size();
    return PTYCHO_OK;
}

extern "C" int ptycho_server_poll(ptycho_server* s, uint64_t id, int32_t* state, float* obj_out,
                                  float* probe_out, double* times) {
    if (!s || !state) return PTYCHO_EINVAL;
    auto it = s->all.find(id);
    if (it == s->all.end()) return PTYCHO_EINVAL;
    Request* r = it->second.get();
    *state = r->state;
    if (r->state == PTYCHO_REQ_DONE) {
        if (obj_out) std::memcpy(obj_out, r->obj_out.data(), r->obj_out.size() * sizeof(float));
        if (probe_out) std::memcpy(probe_out, r->probe_out.data(), r->probe_out.size() * sizeof(float));
        if (times) {
            times[0] = seconds(r->t_submit, r->t_admit);
            times[1] = seconds(r->t_submit, r->t_done);
            times[2] = r->n_iter > 0 ? seconds(r->t_admit, r->t_done) * 100.0 / r->n_iter : 0.0;
            times[3] = r->final_err;
        }
    }
    return PTYCHO_OK;
}

extern "C" void ptycho_server_destroy(ptycho_server* s) {
    if (!s) return;
    for (Request* r : s->active)
        if (r->ctx) ptycho_destroy(r->ctx);
    delete s;
}
