// Batching and serving runtime (include/ptycho_serve.h): many reconstructions
// of the generalised divide-and-concur update on one GPU.
//
// Batch: the contexts' steady-state iteration (re-split prologue, divide,
// concur) is captured once into a CUDA graph and replayed; the first
// iteration, which may start from loaded exit waves, runs directly.  Two
// graph layouts: launch groups (the FP32 cluster-design contexts of one
// pattern side run as one ragged divide launch over the (scan, wave) work
// list of all their scans and one ragged launch per concur kernel; other
// contexts keep a branch of their own), or one branch per context (fork and
// join through events on a private stream).  In the automatic mode both
// graphs are captured, one replay of each is timed, and the faster one is
// replayed.  Every layout runs the same per-scan arithmetic.
//
// Server: FIFO admission under an HBM budget, a bounded active set, rounds of
// a few iterations of every active request on the requests' own streams, and
// retirement with result copy-back.  Rounds are not global: a request gets
// its next round as soon as its previous one has finished, and new requests
// are loaded while the others' rounds run (continuous batching); a finished
// request frees its memory (stream-ordered, without synchronising the
// device) and its slot for the next one in the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <thread>
#include <vector>

#include "../../include/ptycho.h"
#include "../../include/ptycho_serve.h"
#include "internal.h"
#include "nvtx.h"

using Clock = std::chrono::steady_clock;
using namespace ptycho;

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
    int mode = PTYCHO_BATCH_AUTO;
    ptycho_batch_info_t info{};  // of the last run
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

    // first iteration directly (contexts may start from loaded exit waves),
    // and directly too while any context still holds its probe fixed (the
    // captured iteration must be the same in every replay)
    int64_t direct = 1;
    for (auto& en : b->e) direct = std::max<int64_t>(direct, ptycho::ctx_probe_hold(en.ctx));
    direct = std::min<int64_t>(direct, n_iter);
    for (int64_t k = 0; k < direct; ++k)
        for (auto& en : b->e) {
            int rc = ptycho_iterate(en.ctx, en.a, en.b, en.c, 1);
            if (rc) return rc;
        }
    n_iter -= (int32_t)(direct - 1);  // the remaining iterations, counting the first one
    if (n_iter == 1) {
        for (auto& en : b->e)
            if (cudaStreamSynchronize(ptycho::ctx_stream(en.ctx)) != cudaSuccess) return PTYCHO_ECUDA;
        return PTYCHO_OK;
    }
    // Launch groups: the FP32 cluster-design contexts of one pattern side (and
    // launch variant) run each iteration as one ragged divide launch and one
    // ragged launch per concur kernel over all their scans; the others keep a
    // branch of their own in the graph.
    struct Group {
        int N = 0, variant = 0;
        std::vector<size_t> idx;
        cudaStream_t st = nullptr;
        cudaEvent_t join = nullptr;
        void* dev = nullptr;  // device tables of the group
        RaggedConcur rc{};
        const DivideArgs* dtab = nullptr;
        const int* dfirst = nullptr;
        int waves = 0;
    };
    const size_t ne = b->e.size();
    std::vector<DivideArgs> das(ne);
    std::vector<ConcurScan> css(ne);
    std::vector<int> group_of(ne, -1);
    std::vector<Group> groups;
    for (size_t i = 0; i < ne; ++i) {
        const BatchEntry& en = b->e[i];
        int N = 0, v = 0;
        if (!ptycho::ctx_ragged_iteration(en.ctx, en.a, en.b, en.c, &das[i], &css[i], &N, &v)) continue;
        int g = -1;
        for (size_t k = 0; k < groups.size(); ++k)
            if (groups[k].N == N && groups[k].variant == v) g = (int)k;
        if (g < 0) {
            groups.push_back(Group{});
            groups.back().N = N;
            groups.back().variant = v;
            g = (int)groups.size() - 1;
        }
        groups[(size_t)g].idx.push_back(i);
        group_of[i] = g;
    }
    struct Cleanup {
        std::vector<Group>* g;
        ~Cleanup() {
            for (Group& x : *g) {
                if (x.st) cudaStreamDestroy(x.st);
                if (x.join) cudaEventDestroy(x.join);
                if (x.dev) cudaFree(x.dev);
            }
        }
    } cleanup{&groups};
    for (Group& g : groups) {
        // one gather shape and one probe-partial width per group (a launch
        // choice; the results do not depend on it): the first scan's
        const ConcurBufs& c0 = css[g.idx[0]].cb;
        for (size_t k = 1; k < g.idx.size(); ++k) {
            const size_t i = g.idx[k];
            if (css[i].cb.gather_shape != c0.gather_shape || css[i].cb.probe_ppt != c0.probe_ppt) {
                const TileShape sh = kGatherShape[c0.gather_shape];
                int rc = ptycho_set_launch_shapes(b->e[i].ctx, sh.rows, sh.cols, c0.probe_ppt, 0);
                if (rc) return rc;
                int N = 0, v = 0;
                ptycho::ctx_ragged_iteration(b->e[i].ctx, b->e[i].a, b->e[i].b, b->e[i].c, &das[i],
                                             &css[i], &N, &v);
            }
        }
        const int n = (int)g.idx.size();
        std::vector<DivideArgs> dt((size_t)n);
        std::vector<ConcurScan> ct((size_t)n);
        std::vector<int> wfirst((size_t)n + 1, 0);
        for (int k = 0; k < n; ++k) {
            dt[(size_t)k] = das[g.idx[(size_t)k]];
            ct[(size_t)k] = css[g.idx[(size_t)k]];
            wfirst[(size_t)k + 1] = wfirst[(size_t)k] + dt[(size_t)k].J;
        }
        std::vector<int> cfirst, nslice;
        ragged_concur_tables(ct.data(), n, cfirst, nslice, g.rc.totals);
        const size_t b_dt = dt.size() * sizeof(DivideArgs), b_ct = ct.size() * sizeof(ConcurScan);
        const size_t b_wf = wfirst.size() * sizeof(int), b_cf = cfirst.size() * sizeof(int);
        const size_t b_ns = nslice.size() * sizeof(int);
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        const size_t total = up(b_dt) + up(b_ct) + up(b_wf) + up(b_cf) + up(b_ns);
        if (cudaMalloc(&g.dev, total) != cudaSuccess) return PTYCHO_ENOMEM;
        char* p = static_cast<char*>(g.dev);
        char* p_dt = p;
        char* p_ct = p_dt + up(b_dt);
        char* p_wf = p_ct + up(b_ct);
        char* p_cf = p_wf + up(b_wf);
        char* p_ns = p_cf + up(b_cf);
        if (cudaMemcpy(p_dt, dt.data(), b_dt, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p_ct, ct.data(), b_ct, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p_wf, wfirst.data(), b_wf, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p_cf, cfirst.data(), b_cf, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p_ns, nslice.data(), b_ns, cudaMemcpyHostToDevice) != cudaSuccess)
            return PTYCHO_ECUDA;
        g.dtab = reinterpret_cast<const DivideArgs*>(p_dt);
        g.dfirst = reinterpret_cast<const int*>(p_wf);
        g.waves = wfirst.back();
        g.rc.scans = reinterpret_cast<const ConcurScan*>(p_ct);
        g.rc.first = reinterpret_cast<const int*>(p_cf);
        g.rc.n_slice = reinterpret_cast<const int*>(p_ns);
        g.rc.n = n;
        g.rc.gather_shape = ct[0].cb.gather_shape;
        g.rc.probe_ppt = ct[0].cb.probe_ppt;
        if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess)
            return PTYCHO_ECUDA;
    }
    while (b->join.size() < ne) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return PTYCHO_ECUDA;
        b->join.push_back(ev);
    }
    // the main stream starts after every context's direct iterations
    for (size_t i = 0; i < ne; ++i) {
        if (cudaEventRecord(b->join[i], ptycho::ctx_stream(b->e[i].ctx)) != cudaSuccess ||
            cudaStreamWaitEvent(b->main, b->join[i], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
    }
    // Capture one steady-state iteration of every context: with launch groups
    // (groups, plus branches for the other contexts), and with a branch per
    // context.  Both compute the same iteration, bit for bit.
    std::vector<int64_t> base(ne);
    for (size_t i = 0; i < ne; ++i) base[i] = ptycho::ctx_iterations(b->e[i].ctx);
    auto capture = [&](bool use_groups, cudaGraphExec_t* exec) -> int {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return PTYCHO_ECUDA;
        int rc = PTYCHO_OK;
        cudaEventRecord(b->fork, b->main);
        if (use_groups) {
            for (Group& g : groups) {
                cudaStreamWaitEvent(g.st, b->fork, 0);
                if (launch_divide_ragged(g.N, g.variant, g.dtab, g.dfirst, g.rc.n, g.waves, g.st) !=
                        cudaSuccess ||
                    launch_concur_ragged(g.rc, g.st) != cudaSuccess)
                    rc = PTYCHO_ECUDA;
                cudaEventRecord(g.join, g.st);
                cudaStreamWaitEvent(b->main, g.join, 0);
            }
        }
        for (size_t i = 0; i < ne && rc == PTYCHO_OK; ++i) {
            if (use_groups && group_of[i] >= 0) continue;
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
        ce = cudaGraphInstantiate(exec, graph, 0);
        cudaGraphDestroy(graph);
        return ce == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
    };
    const bool have_groups = !groups.empty() && b->mode != PTYCHO_BATCH_BRANCHES;
    const bool try_both = have_groups && b->mode == PTYCHO_BATCH_AUTO && n_iter - 1 >= 3;
    cudaGraphExec_t gexec = nullptr, bexec = nullptr;
    struct ExecGuard {
        cudaGraphExec_t* a;
        cudaGraphExec_t* b;
        ~ExecGuard() {
            if (*a) cudaGraphExecDestroy(*a);
            if (*b) cudaGraphExecDestroy(*b);
        }
    } exec_guard{&gexec, &bexec};
    int rc = PTYCHO_OK;
    if (have_groups && (rc = capture(true, &gexec)) != PTYCHO_OK) return rc;
    if ((!have_groups || try_both) && (rc = capture(false, &bexec)) != PTYCHO_OK) return rc;
    // the captures recorded one iteration per context without running it;
    // n_iter - 1 replays run iterations 2 .. n_iter
    int replays = n_iter - 1;
    cudaError_t ce = cudaSuccess;
    b->info = ptycho_batch_info_t{};
    cudaGraphExec_t use = have_groups ? gexec : bexec;
    if (try_both) {
        // one timed replay of each, then the faster one for the rest
        cudaEvent_t e0, e1, e2;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventCreate(&e2);
        cudaEventRecord(e0, b->main);
        ce = cudaGraphLaunch(gexec, b->main);
        cudaEventRecord(e1, b->main);
        if (ce == cudaSuccess) ce = cudaGraphLaunch(bexec, b->main);
        cudaEventRecord(e2, b->main);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e2);
        float tg = 0.f, tb = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tg, e0, e1);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tb, e1, e2);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        if (ce != cudaSuccess) return PTYCHO_ECUDA;
        b->info.groups_ms = tg;
        b->info.branches_ms = tb;
        use = tg <= tb ? gexec : bexec;
        replays -= 2;
    }
    for (int it = 0; it < replays && ce == cudaSuccess; ++it) ce = cudaGraphLaunch(use, b->main);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->main);
    if (ce != cudaSuccess) return PTYCHO_ECUDA;
    for (size_t i = 0; i < ne; ++i)
        ptycho::ctx_batch_done(b->e[i].ctx, b->e[i].a, b->e[i].b, base[i] + (n_iter - 1));
    b->info.groups = have_groups ? (int32_t)groups.size() : 0;
    int32_t in = 0;
    for (int g : group_of) in += (have_groups && g >= 0) ? 1 : 0;
    b->info.in_groups = in;
    b->info.used = use == gexec && have_groups ? PTYCHO_BATCH_GROUPS : PTYCHO_BATCH_BRANCHES;
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_set_mode(ptycho_batch* b, int mode) {
    if (!b || mode < PTYCHO_BATCH_AUTO || mode > PTYCHO_BATCH_BRANCHES) return PTYCHO_EINVAL;
    b->mode = mode;
    return PTYCHO_OK;
}

extern "C" int ptycho_batch_info(const ptycho_batch* b, ptycho_batch_info_t* out) {
    if (!b || !out) return PTYCHO_EINVAL;
    *out = b->info;
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
    int32_t n_iter = 0, done_iter = 0;  // done_iter: iterations enqueued so far
    int32_t state = PTYCHO_REQ_QUEUED;
    ptycho_ctx* ctx = nullptr;
    cudaEvent_t ev = nullptr;           // recorded after the last enqueued round
    bool pending = false;               // that round may still be running
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
    const size_t need = ptycho::scan_bytes(d->J, d->N, d->M_rows, d->M_cols, s->opts.precision,
                                           s->opts.divide);
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
    ptycho_destroy(r->ctx);  // stream-ordered frees: the other requests keep running
    r->ctx = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    r->ev = nullptr;
    s->used -= r->bytes;
    r->t_done = Clock::now();
    r->state = rc == PTYCHO_OK ? PTYCHO_REQ_DONE : PTYCHO_REQ_FAILED;
}

// 1: the request's last enqueued round has finished (or none is pending);
// 0: still running; < 0: a CUDA error.
int round_done(Request* r) {
    if (!r->pending) return 1;
    const cudaError_t e = cudaEventQuery(r->ev);
    if (e == cudaSuccess) {
        r->pending = false;
        return 1;
    }
    if (e == cudaErrorNotReady) return 0;
    cudaGetLastError();
    return -1;
}

}  // namespace

// The step does not wait for a whole round of every request: it retires
// requests whose work has finished, admits queued ones, and gives every
// request whose previous round has finished its next round, so the device
// keeps running the other requests' rounds while the host loads, admits and
// retires.  When nothing could be done it waits (polling, at most 2 s) until
// some round finishes, and tries once more.
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

    for (int attempt = 0; attempt < 2; ++attempt) {
        bool progressed = false;
        // retirement: every iteration enqueued and the last round finished
        std::vector<Request*> still;
        for (Request* r : s->active) {
            const int d = round_done(r);
            if (d < 0) return PTYCHO_ECUDA;
            if (d == 1 && r->done_iter >= r->n_iter) {
                retire(s, r);
                progressed = true;
            } else {
                still.push_back(r);
            }
        }
        s->active.swap(still);

        // admission, in arrival order
        while (!s->queue.empty() && (int32_t)s->active.size() < s->max_active) {
            Request* r = s->queue.front();
            if (s->used + r->bytes > s->budget) break;
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PTYCHO_ECUDA;
            const size_t margin = (size_t)1 << 30;
            if (r->bytes + margin > free_b) {
                // memory freed by retired requests may still sit in the
                // stream-ordered pool: hand it back to the device, then look again
                cudaMemPool_t pool;
                if (cudaDeviceGetDefaultMemPool(&pool, s->opts.device) == cudaSuccess)
                    cudaMemPoolTrimTo(pool, 0);
                if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return PTYCHO_ECUDA;
                if (r->bytes + margin > free_b) {
                    if (!s->active.empty()) break;  // wait for a request to retire
                    // nothing runs that could free memory: it can never fit
                    s->queue.pop_front();
                    r->state = PTYCHO_REQ_FAILED;
                    r->t_done = Clock::now();
                    progressed = true;
                    continue;
                }
            }
            s->queue.pop_front();
            progressed = true;
            ptycho_ctx* ctx = nullptr;
            int rc = ptycho_create(&ctx, &s->opts);
            if (rc == PTYCHO_OK)
                rc = ptycho_load_scan(ctx, r->J, r->N, r->pos.data(), r->inten.data(), r->Mr, r->Mc,
                                      r->obj0.data(), r->probe0.data(), 0);
            if (rc == PTYCHO_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
                rc = PTYCHO_ECUDA;
            if (rc != PTYCHO_OK) {
                if (ctx) ptycho_destroy(ctx);
                r->ev = nullptr;
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

        // rounds: the next iterations of every request whose previous round finished
        for (Request* r : s->active) {
            const int d = round_done(r);
            if (d < 0) return PTYCHO_ECUDA;
            const int32_t k = std::min(iters_per_round, r->n_iter - r->done_iter);
            if (d == 1 && k > 0) {
                int rc = ptycho_iterate(r->ctx, r->a, r->b, r->c, k);
                if (rc != PTYCHO_OK) return rc;
                r->done_iter += k;
                if (cudaEventRecord(r->ev, ptycho::ctx_stream(r->ctx)) != cudaSuccess) return PTYCHO_ECUDA;
                r->pending = true;
                progressed = true;
            }
        }
        if (progressed || s->active.empty() || attempt == 1) break;
        // nothing to do until a round finishes
        const auto t0 = Clock::now();
        for (bool any = false; !any && seconds(t0, Clock::now()) < 2.0;) {
            for (Request* r : s->active) {
                const int d = round_done(r);
                if (d < 0) return PTYCHO_ECUDA;
                any = any || d == 1;
            }
            if (!any) std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
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
    for (Request* r : s->active) {
        if (r->ctx) ptycho_destroy(r->ctx);
        if (r->ev) cudaEventDestroy(r->ev);
    }
    delete s;
}
