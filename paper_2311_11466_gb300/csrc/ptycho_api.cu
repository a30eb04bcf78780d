// C ABI of the library (declared in include/ptycho.h): context, scan loading,
// the abc iteration loop, state access and error history.
//
// State kept on the device between iterations (lazy re-split): after
// iteration k the context holds y_k = P^c_D x_k, the new object and probe
// (O_{k+1}, P_{k+1}), x_k when a_k != 1, and the pending coefficients (a_k, b_k).
// The next divide kernel forms x_{k+1} = a_k (b_k P O_j + (1 - b_k) y_k) + (1 - a_k) x_k
// on the fly, so the re-split costs no extra pass over memory.  A caller who
// asks for x materialises it with the identical expression.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/ptycho.h"
#include "debug.cuh"
#include "internal.h"
#include "nvtx.h"

using namespace ptycho;

namespace {

constexpr int kRing = 65536;  // error-history entries kept on the device
constexpr int kProfMax = 4096;  // iterations the timing hook can record
// Design of the FP32 divide step that PTYCHO_DIVIDE_AUTO picks at N = 256
// (the faster of the two on the 1024 x 256^2 workload); other N have only the
// cluster design.
constexpr int kAutoDivide256 = PTYCHO_DIVIDE_CLUSTER;

thread_local std::string g_create_error;

}  // namespace

struct ptycho_ctx {
    ptycho_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    bool loaded = false;
    int J = 0, N = 0, Mr = 0, Mc = 0, C = 0;
    int n_part = 0;  // Fourier-error partials the divide design writes per iteration
    double sumI = 0.0;

    float2 *x = nullptr, *y = nullptr, *P = nullptr, *O = nullptr, *tw = nullptr;
    float* sqrtIp = nullptr;
    int divide = PTYCHO_DIVIDE_CLUSTER;  // resolved divide design of the current scan
    int variant = 0;                     // cluster design: launch variant (128^2 tuned)
    float2* scratch = nullptr;  // cluster design: transpose scratch, one slot per exit wave;
                                // two-pass design: a ring of slots (Fourier error only, SP)
    unsigned* ctl = nullptr;    // two-pass design: ticket and completion counts
    // tensor-core path: sqrt(I) in the patterns' layout, two ping-pong operand buffers (hi,
    // lo) and the constant DFT operands (fwd hi, fwd lo, inv hi, inv lo)
    float* sqrtI = nullptr;
    uint16_t* planes[4] = {nullptr, nullptr, nullptr, nullptr};
    uint16_t* Bc[4] = {nullptr, nullptr, nullptr, nullptr};
    int2* pos = nullptr;
    double *e_part = nullptr, *e_ring = nullptr, *e_tmp = nullptr;
    unsigned long long* d_iter = nullptr;  // device-side iteration counter (ring slot)
    int* dflag = nullptr;
    ConcurBufs cb{};
    std::vector<void*> allocs;
    size_t bytes = 0;

    bool have_x = true;    // x_k is in the x buffer (else x_k = re-split(pa, pb), see above)
    float pa = 1.f, pb = 1.f;
    int64_t iters = 0;
    int32_t probe_start = 0;  // iterations k < probe_start hold the probe fixed
    bool tuned = false;         // launch shapes of the concur kernels chosen
    bool tuning = true;         // choose them at the first iteration (ptycho_set_tuning)
    std::vector<int32_t> pos_h; // host copy of the positions (tile lists)

    // measurement: three events per recorded iteration
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    int prof_n = 0;
};

namespace {

int fail(ptycho_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(ptycho_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, PTYCHO_ENOMEM, m);
    }
    return fail(ctx, PTYCHO_ECUDA, m);
}

#define PT_CUDA(ctx, call)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

template <class T>
int dalloc(ptycho_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    const size_t b = count * sizeof(T);
    if (b == 0) return PTYCHO_OK;
    void* q = nullptr;
    // stream-ordered allocation from the device's pool: freeing it later does
    // not synchronise the device (cudaFree would), so a context that is
    // destroyed does not stall the work of other contexts
    cudaError_t e = cudaMallocAsync(&q, b, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PTYCHO_ENOMEM, "device allocation of " + std::to_string(b) +
                                            " bytes failed: " + cudaGetErrorString(e));
    }
    ctx->allocs.push_back(q);
    ctx->bytes += b;
    *p = static_cast<T*>(q);
    return PTYCHO_OK;
}

// The device's stream-ordered pool (context memory) keeps what contexts free
// instead of handing it back to the driver at the next synchronisation, so a
// context that follows another (a served request, a reconstruction after a
// reconstruction) reuses the mapped memory.  A process-local setting of this
// process's pool; the server trims the pool before it refuses a request for
// lack of free device memory.
void keep_pool_memory(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    for (int d : done)
        if (d == device) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(device);
}

void free_scan(ptycho_ctx* ctx) {
    for (void* p : ctx->allocs) cudaFreeAsync(p, ctx->stream);
    ctx->allocs.clear();
    ctx->bytes = 0;
    ctx->x = ctx->y = ctx->P = ctx->O = ctx->tw = nullptr;
    ctx->sqrtIp = nullptr;
    ctx->scratch = nullptr;
    ctx->ctl = nullptr;
    ctx->sqrtI = nullptr;
    for (int i = 0; i < 4; ++i) ctx->planes[i] = ctx->Bc[i] = nullptr;
    ctx->pos = nullptr;
    ctx->e_part = ctx->e_ring = ctx->e_tmp = nullptr;
    ctx->d_iter = nullptr;
    ctx->dflag = nullptr;
    ctx->cb = ConcurBufs{};
    ctx->loaded = false;
    ctx->iters = 0;
}

bool all_finite(const float* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// After a synchronisation: a bounded device wait that expired (bit 0: the
// tensor-core DFT kernel; bit 1: the two-pass divide kernel) leaves a flag;
// report it once.
int check_device_flags(ptycho_ctx* ctx) {
    if (!ctx->dflag || (ctx->opts.precision != PTYCHO_PREC_BF16X3 && ctx->divide != PTYCHO_DIVIDE_TWOPASS))
        return PTYCHO_OK;
    int f = 0;
    PT_CUDA(ctx, cudaMemcpy(&f, ctx->dflag + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        PT_CUDA(ctx, cudaMemset(ctx->dflag + 1, 0, sizeof(int)));
        return fail(ctx, PTYCHO_ETIMEOUT, (f & 1) ? "a bounded wait in the tensor-core DFT kernel expired"
                                                  : "a bounded wait in the two-pass divide kernel expired");
    }
    return PTYCHO_OK;
}

// Arguments of the divide kernels common to every call of a context.
DivideArgs divide_args(ptycho_ctx* ctx) {
    DivideArgs da{};
    da.x = ctx->x;
    da.y = ctx->y;
    da.sqrtIp = ctx->sqrtIp;
    da.P = ctx->P;
    da.O = ctx->O;
    da.pos = ctx->pos;
    da.tw = ctx->tw;
    da.e_part = ctx->e_part;
    da.J = ctx->J;
    da.Mr = ctx->Mr;
    da.Mc = ctx->Mc;
    da.scratch = ctx->scratch;
    da.ctl = ctx->ctl;
    da.lag = divide2p_lag();
    da.ring = ctx->J < divide2p_ring() ? ctx->J : divide2p_ring();
    da.err_flag = ctx->dflag + 1;
    da.variant = ctx->variant;
    return da;
}

ConcurScan concur_scan(ptycho_ctx* ctx, int n_part) {
    ConcurScan cs{};
    cs.y = ctx->y;
    cs.P = ctx->P;
    cs.O = ctx->O;
    cs.pos = ctx->pos;
    cs.cb = ctx->cb;
    cs.J = ctx->J;
    cs.N = ctx->N;
    cs.Mr = ctx->Mr;
    cs.Mc = ctx->Mc;
    cs.alpha = (double)ctx->opts.alpha;
    cs.e_part = ctx->e_part;
    cs.n_part = n_part;
    cs.inv_sumI = ctx->sumI > 0 ? 1.0 / ctx->sumI : 1.0;
    cs.e_ring = ctx->e_ring;
    cs.d_iter = ctx->d_iter;
    cs.ring_cap = kRing;
    return cs;
}

cudaError_t launch_divide_ctx(ptycho_ctx* ctx, const DivideArgs& da) {
    return ctx->divide == PTYCHO_DIVIDE_TWOPASS ? launch_divide2p(da, ctx->stream)
                                                : launch_divide(ctx->N, da, ctx->stream);
}

int materialise(ptycho_ctx* ctx) {
    if (ctx->have_x) return PTYCHO_OK;
    PT_CUDA(ctx, launch_materialise(ctx->x, ctx->y, ctx->P, ctx->O, ctx->pos, ctx->J, ctx->N,
                                    ctx->Mc, ctx->pa, ctx->pb, ctx->stream));
    ctx->have_x = true;
    return PTYCHO_OK;
}

// The divide arguments of the context's next iteration with (a, b, c), from
// its lazy state.
DivideArgs iteration_args(ptycho_ctx* ctx, float a, float b, float c) {
    DivideArgs da = divide_args(ctx);
    da.load_x = ctx->have_x ? 1 : 0;
    da.pa = ctx->pa;
    da.pb = ctx->pb;
    da.c = c;
    da.err_only = 0;
    da.write_x = (!ctx->have_x && a != 1.0f) ? 1 : 0;  // x_k is the next (1 - a) term
    (void)b;
    return da;
}

// The host-side lazy state after an iteration with (a, b).
void iteration_done(ptycho_ctx* ctx, float a, float b) {
    ctx->have_x = false;
    ctx->pa = a;
    ctx->pb = b;
}

}  // namespace

namespace ptycho {
cudaStream_t ctx_stream(const ptycho_ctx* ctx) { return ctx->stream; }
int ctx_device(const ptycho_ctx* ctx) { return ctx->opts.device; }
bool ctx_loaded(const ptycho_ctx* ctx) { return ctx->loaded; }
void ctx_add_iterations(ptycho_ctx* ctx, int64_t n) { ctx->iters += n; }
bool ctx_ragged_iteration(ptycho_ctx* ctx, float a, float b, float c, DivideArgs* da,
                          ConcurScan* cs, int* N, int* variant) {
    if (!ctx->loaded || ctx->have_x || ctx->opts.precision != PTYCHO_PREC_FP32 ||
        ctx->divide != PTYCHO_DIVIDE_CLUSTER || ctx->opts.concur != PTYCHO_CONCUR_DETERMINISTIC ||
        ctx->iters < ctx->probe_start || !ctx->tuned)
        return false;
    *da = iteration_args(ctx, a, b, c);
    *cs = concur_scan(ctx, ctx->n_part);
    *N = ctx->N;
    *variant = ctx->variant;
    return true;
}

void ctx_batch_done(ptycho_ctx* ctx, float a, float b, int64_t n) {
    iteration_done(ctx, a, b);
    ctx->iters = n;
}

int64_t ctx_iterations(const ptycho_ctx* ctx) { return ctx->iters; }

int64_t ctx_probe_hold(const ptycho_ctx* ctx) {
    return ctx->iters < ctx->probe_start ? ctx->probe_start - ctx->iters : 0;
}
}  // namespace ptycho

extern "C" {

void ptycho_default_opts(ptycho_opts* o) {
    if (!o) return;
    o->device = 0;
    o->precision = PTYCHO_PREC_FP32;
    o->concur = PTYCHO_CONCUR_DETERMINISTIC;
    o->alpha = 1e-6f;
    o->stream = nullptr;
    o->divide = PTYCHO_DIVIDE_AUTO;
}

int ptycho_create(ptycho_ctx** out, const ptycho_opts* opts) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return PTYCHO_EINVAL;
    }
    *out = nullptr;
    ptycho_opts o;
    ptycho_default_opts(&o);
    if (opts) o = *opts;
    if (o.precision != PTYCHO_PREC_FP32 && o.precision != PTYCHO_PREC_BF16X3) {
        g_create_error = "unknown precision";
        return PTYCHO_EINVAL;
    }
    if (o.concur != PTYCHO_CONCUR_DETERMINISTIC && o.concur != PTYCHO_CONCUR_ATOMIC) {
        g_create_error = "unknown concur mode";
        return PTYCHO_EINVAL;
    }
    if (!(o.alpha >= 0.0f) || !std::isfinite(o.alpha)) {
        g_create_error = "alpha must be finite and >= 0";
        return PTYCHO_EINVAL;
    }
    if (o.divide != PTYCHO_DIVIDE_AUTO && o.divide != PTYCHO_DIVIDE_CLUSTER &&
        o.divide != PTYCHO_DIVIDE_TWOPASS) {
        g_create_error = "unknown divide design";
        return PTYCHO_EINVAL;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || o.device < 0 || o.device >= ndev) {
        cudaGetLastError();
        g_create_error = std::string("no such CUDA device: ") +
                         (e != cudaSuccess ? cudaGetErrorString(e) : std::to_string(o.device));
        return e != cudaSuccess ? PTYCHO_ECUDA : PTYCHO_EINVAL;
    }
    DeviceGuard dg(o.device);
    keep_pool_memory(o.device);
    ptycho_ctx* ctx = new ptycho_ctx();
    ctx->opts = o;
    if (o.stream) {
        ctx->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            delete ctx;
            return PTYCHO_ECUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return PTYCHO_OK;
}

void ptycho_destroy(ptycho_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard dg(ctx->opts.device);
        cudaStreamSynchronize(ctx->stream);
        free_scan(ctx);
        for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

const char* ptycho_last_error(const ptycho_ctx* ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

size_t ptycho_scan_bytes(int32_t J, int32_t N, int32_t M_rows, int32_t M_cols, int precision) {
    return ptycho::scan_bytes(J, N, M_rows, M_cols, precision, PTYCHO_DIVIDE_AUTO);
}

int ptycho_divide_design(const ptycho_ctx* ctx) { return ctx && ctx->loaded ? ctx->divide : 0; }

}  // extern "C"

int ptycho::resolve_divide(int precision, int divide, int N) {
    if (precision == PTYCHO_PREC_BF16X3 || !divide2p_supported(N)) return PTYCHO_DIVIDE_CLUSTER;
    if (divide == PTYCHO_DIVIDE_TWOPASS || divide == PTYCHO_DIVIDE_CLUSTER) return divide;
    return kAutoDivide256;
}

size_t ptycho::scan_bytes(int J, int N, int M_rows, int M_cols, int precision, int divide) {
    if (J <= 0 || N <= 0 || M_rows <= 0 || M_cols <= 0) return 0;
    const bool two = resolve_divide(precision, divide, N) == PTYCHO_DIVIDE_TWOPASS;
    const size_t NN = (size_t)N * N, M = (size_t)M_rows * M_cols;
    const size_t chunks = (size_t)probe_chunks(J, N);
    size_t b = 0;
    b += 2 * (size_t)J * NN * sizeof(float2);        // x, y
    b += (size_t)J * NN * sizeof(float);             // sqrt(I)
    b += 2 * NN * sizeof(float2) + M * sizeof(float2);  // P, tw, O
    b += (size_t)J * sizeof(int2);
    const size_t parts_fp32 = (size_t)J * (N > 16 ? N : 16);  // either divide design
    b += parts_fp32 * sizeof(double) + (size_t)kRing * sizeof(double) + 64 + 256 * sizeof(double);
    b += M * (sizeof(float2) + sizeof(double)) + 16;
    b += chunks * NN * (sizeof(float2) + sizeof(float));
    b += NN * (sizeof(double2) + sizeof(double));
    b += (size_t)probe_reduce_blocks(N, (int)chunks) * sizeof(double);  // error slice totals
    b += tile_csr_ptr_bound(N, M_rows, M_cols) * sizeof(int) + tile_csr_entries_bound(J, N) * sizeof(int4);
    b += (size_t)J * ((NN + 255) / 256) * sizeof(double);  // load-time partial sums
    b += (size_t)J * (sizeof(int) + sizeof(int4) + sizeof(int2));  // staged-atomic groups (bound)
    if (two) {
        const int ring = J < divide2p_ring() ? J : divide2p_ring();
        b += (size_t)ring * NN * sizeof(float2);                    // scratch ring
        b += divide2p_ctl_words(J) * sizeof(unsigned);              // ticket and counts
    } else {
        b += (size_t)(J > 2 ? J : 2) * NN * sizeof(float2);  // transpose scratch
    }
    if (precision == PTYCHO_PREC_BF16X3) {
        b += (size_t)J * NN * sizeof(float);           // sqrt(I), patterns' layout
        b += 4 * (size_t)J * NN * 2 * sizeof(uint16_t);  // two operand buffers, hi + lo
        b += 4 * 4 * NN * sizeof(uint16_t);            // constant DFT operands
        const size_t parts = (size_t)bf16x3_error_parts(N, J);  // a second, larger error buffer
        if (parts > parts_fp32) b += parts * sizeof(double);
    }
    return b;
}

extern "C" {

int ptycho_load_scan(ptycho_ctx* ctx, int32_t J, int32_t N, const int32_t* pos_rc,
                     const float* intensity, int32_t M_rows, int32_t M_cols, const float* obj0,
                     const float* probe0, uint32_t flags) {
    NvtxRange nvtx_range("ptycho_load_scan");
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (J < 1) return fail(ctx, PTYCHO_EINVAL, "J must be >= 1");
    if (!divide_supported(N))
        return fail(ctx, PTYCHO_EINVAL, "N must be one of 8, 16, 32, 64, 128, 256");
    if (M_rows < N || M_cols < N) return fail(ctx, PTYCHO_EINVAL, "object smaller than the probe");
    const bool tc = ctx->opts.precision == PTYCHO_PREC_BF16X3;
    if (tc && !bf16x3_supported(N))
        return fail(ctx, PTYCHO_EINVAL, "BF16X3 precision needs N = 128 or 256");
    if (!pos_rc || !intensity || !obj0 || !probe0)
        return fail(ctx, PTYCHO_EINVAL, "NULL input pointer");
    if ((size_t)J * N * N > (size_t)1 << 40) return fail(ctx, PTYCHO_EINVAL, "scan too large");
    for (int j = 0; j < J; ++j) {
        const int r = pos_rc[2 * j], c = pos_rc[2 * j + 1];
        if (r < 0 || r > M_rows - N || c < 0 || c > M_cols - N)
            return fail(ctx, PTYCHO_EINVAL, "position " + std::to_string(j) + " = (" +
                                                std::to_string(r) + ", " + std::to_string(c) +
                                                ") outside [0, M - N]");
    }
    const size_t NN = (size_t)N * N, M = (size_t)M_rows * M_cols;
    if (!all_finite(obj0, 2 * M)) return fail(ctx, PTYCHO_EINVAL, "obj0 has a non-finite value");
    if (!all_finite(probe0, 2 * NN)) return fail(ctx, PTYCHO_EINVAL, "probe0 has a non-finite value");

    DeviceGuard dg(ctx->opts.device);
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    free_scan(ctx);
    {
        // fail before any host work or allocation when the scan cannot fit
        const size_t need = scan_bytes(J, N, M_rows, M_cols, ctx->opts.precision, ctx->opts.divide);
        size_t free_b = 0, total_b = 0;
        PT_CUDA(ctx, cudaMemGetInfo(&free_b, &total_b));
        if (need > free_b) {
            // memory freed into the stream-ordered pool counts as used: hand it back, look again
            cudaMemPool_t pool;
            PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            if (cudaDeviceGetDefaultMemPool(&pool, ctx->opts.device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
            cudaGetLastError();
            PT_CUDA(ctx, cudaMemGetInfo(&free_b, &total_b));
            if (need > free_b)
                return fail(ctx, PTYCHO_ENOMEM, "the scan needs " + std::to_string(need) +
                                                    " bytes of device memory; " + std::to_string(free_b) +
                                                    " are free");
        }
    }

    // Object tiles: CSR lists of the positions whose window overlaps each tile,
    // in ascending position order (integer work, done here), for the tile
    // shape the tuner chose for this kind of scan (or the default).
    const TuneChoice tuned = tune_lookup(ctx->opts.device, N, J);
    std::vector<int> tile_cnt;
    std::vector<int4> tile_list;
    build_tile_csr(pos_rc, J, N, M_rows, M_cols, kGatherShape[tuned.gather_shape], tile_cnt, tile_list);
    const TileShape shape = kGatherShape[tuned.gather_shape];
    // staged-atomic concur: position groups (integer work, done here)
    const bool atomic = ctx->opts.concur == PTYCHO_CONCUR_ATOMIC;
    std::vector<int> sc_ord;
    std::vector<int4> sc_groups;
    std::vector<int2> sc_ext;
    int sc_rows = 0, sc_box = 0;
    if (atomic) build_scatter_groups(pos_rc, J, N, sc_ord, sc_groups, sc_ext, &sc_rows, &sc_box);
    const int tiles_r = (M_rows + shape.rows - 1) / shape.rows;
    const int tiles_c = (M_cols + shape.cols - 1) / shape.cols;

    const int C = divide_cluster_size(N);
    const int chunks = probe_chunks(J, N);
    const int design = resolve_divide(ctx->opts.precision, ctx->opts.divide, N);
    const bool two = design == PTYCHO_DIVIDE_TWOPASS;
    {
        cudaError_t pe = divide_prepare(N);
        if (pe == cudaSuccess && two) pe = divide2p_prepare();
        if (pe == cudaSuccess && atomic) pe = concur_prepare();
        if (pe != cudaSuccess) return cuda_fail(ctx, pe, "divide_prepare");
    }
    const int sq_blocks = (int)((NN + 255) / 256);
    double* psum = nullptr;
    int rc;
#define PT_ALLOC(p, n)                           \
    do {                                         \
        if ((rc = dalloc(ctx, &(p), (n))) != 0) { \
            free_scan(ctx);                      \
            return rc;                           \
        }                                        \
    } while (0)
    PT_ALLOC(ctx->x, (size_t)J * NN);
    PT_ALLOC(ctx->y, (size_t)J * NN);
    PT_ALLOC(ctx->sqrtIp, (size_t)J * NN);
    if (two) {
        PT_ALLOC(ctx->scratch, (size_t)(J < divide2p_ring() ? J : divide2p_ring()) * NN);
        PT_ALLOC(ctx->ctl, divide2p_ctl_words(J));
    } else {
        PT_ALLOC(ctx->scratch, (size_t)(J > 2 ? J : 2) * NN);  // SP steps use two slots
    }
    PT_ALLOC(ctx->P, NN);
    PT_ALLOC(ctx->tw, (size_t)N);
    PT_ALLOC(ctx->O, M);
    PT_ALLOC(ctx->pos, (size_t)J);
    const size_t parts_fp32 = (size_t)J * (N > 16 ? N : 16);  // either divide design
    PT_ALLOC(ctx->e_part, parts_fp32);
    PT_ALLOC(ctx->e_ring, (size_t)kRing);
    PT_ALLOC(ctx->e_tmp, (size_t)4 + 256);  // [0]: a result; [4..]: slice totals
    PT_ALLOC(ctx->d_iter, (size_t)1);
    PT_ALLOC(ctx->dflag, (size_t)4);
    PT_ALLOC(ctx->cb.numO, M);
    PT_ALLOC(ctx->cb.denO, M);
    PT_ALLOC(ctx->cb.maxO, (size_t)1);
    PT_ALLOC(ctx->cb.partP, (size_t)chunks * NN);
    PT_ALLOC(ctx->cb.partPd, (size_t)chunks * NN);
    PT_ALLOC(ctx->cb.numP, NN);
    PT_ALLOC(ctx->cb.e_slice, (size_t)probe_reduce_blocks(N, chunks));
    PT_ALLOC(ctx->cb.denP, NN);
    PT_ALLOC(ctx->cb.maxP, (size_t)1);
    // sized for every tile shape, so the tuner can switch shapes in place
    PT_ALLOC(ctx->cb.tile_ptr, tile_csr_ptr_bound(N, M_rows, M_cols));
    PT_ALLOC(ctx->cb.tile_win, tile_csr_entries_bound(J, N) > 0 ? tile_csr_entries_bound(J, N) : 1);
    PT_ALLOC(psum, (size_t)J * sq_blocks);
    if (atomic) {
        PT_ALLOC(ctx->cb.sc_ord, sc_ord.size());
        PT_ALLOC(ctx->cb.sc_groups, sc_groups.size());
        PT_ALLOC(ctx->cb.sc_ext, sc_ext.size());
    }
    if (tc) {
        PT_ALLOC(ctx->sqrtI, (size_t)J * NN);
        for (int i = 0; i < 4; ++i) PT_ALLOC(ctx->planes[i], (size_t)J * NN * 2);
        for (int i = 0; i < 4; ++i) PT_ALLOC(ctx->Bc[i], 4 * NN);
        const int tiles = bf16x3_error_parts(N, J);
        if ((size_t)tiles > parts_fp32) {
            double* more = nullptr;
            PT_ALLOC(more, (size_t)tiles);
            ctx->e_part = more;  // the larger buffer serves both paths
        }
    }
#undef PT_ALLOC
    ctx->cb.tiles_r = tiles_r;
    ctx->cb.tiles_c = tiles_c;
    ctx->cb.chunks = chunks;
    ctx->cb.gather_shape = tuned.gather_shape;
    // the tuner times the deterministic probe pass; the atomic one, with more
    // registers, keeps one pixel per thread unless pinned
    ctx->cb.probe_ppt = atomic ? 1 : tuned.probe_ppt;
    ctx->cb.sc_n = (int)sc_groups.size();
    ctx->cb.sc_rows = sc_rows;
    ctx->cb.sc_box = sc_box;
    ctx->tuned = tuned.valid;
    ctx->pos_h.assign(pos_rc, pos_rc + 2 * (size_t)J);
    ctx->J = J;
    ctx->N = N;
    ctx->Mr = M_rows;
    ctx->Mc = M_cols;
    ctx->C = C;
    ctx->divide = design;
    ctx->n_part = J * divide_error_parts_per_wave(N, two);

    std::vector<float2> tw;
    divide_twiddles(N, tw);
    cudaStream_t st = ctx->stream;
    auto bail = [&](cudaError_t e, const char* where) {
        int r = cuda_fail(ctx, e, where);
        cudaStreamSynchronize(st);
        free_scan(ctx);
        return r;
    };
    cudaError_t e;
#define PT_STEP(call)                                   \
    do {                                                \
        if ((e = (call)) != cudaSuccess) return bail(e, #call); \
    } while (0)
    PT_STEP(divide_prepare(N));
    PT_STEP(cudaMemcpyAsync(ctx->tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st));
    PT_STEP(cudaMemcpyAsync(ctx->pos, pos_rc, (size_t)J * sizeof(int2), cudaMemcpyHostToDevice, st));
    PT_STEP(cudaMemcpyAsync(ctx->O, obj0, M * sizeof(float2), cudaMemcpyHostToDevice, st));
    PT_STEP(cudaMemcpyAsync(ctx->P, probe0, NN * sizeof(float2), cudaMemcpyHostToDevice, st));
    PT_STEP(cudaMemcpyAsync(ctx->cb.tile_ptr, tile_cnt.data(), tile_cnt.size() * sizeof(int),
                            cudaMemcpyHostToDevice, st));
    if (!tile_list.empty())
        PT_STEP(cudaMemcpyAsync(ctx->cb.tile_win, tile_list.data(), tile_list.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, st));
    if (atomic) {
        PT_STEP(cudaMemcpyAsync(ctx->cb.sc_ord, sc_ord.data(), sc_ord.size() * sizeof(int),
                                cudaMemcpyHostToDevice, st));
        PT_STEP(cudaMemcpyAsync(ctx->cb.sc_groups, sc_groups.data(), sc_groups.size() * sizeof(int4),
                                cudaMemcpyHostToDevice, st));
        PT_STEP(cudaMemcpyAsync(ctx->cb.sc_ext, sc_ext.data(), sc_ext.size() * sizeof(int2),
                                cudaMemcpyHostToDevice, st));
    }
    PT_STEP(cudaMemsetAsync(ctx->dflag, 0, 4 * sizeof(int), st));
    PT_STEP(cudaMemsetAsync(ctx->d_iter, 0, sizeof(unsigned long long), st));
    PT_STEP(cudaMemsetAsync(ctx->cb.maxO, 0, sizeof(unsigned long long), st));
    PT_STEP(cudaMemsetAsync(ctx->cb.maxP, 0, sizeof(unsigned long long), st));
    // The intensities pass through the y buffer (twice their size) on their way
    // to the permuted sqrt(I) layout.
    const float* Idev = intensity;
    if (!(flags & PTYCHO_LOAD_INTENSITY_DEVICE)) {
        PT_STEP(cudaMemcpyAsync(ctx->y, intensity, (size_t)J * NN * sizeof(float),
                                cudaMemcpyHostToDevice, st));
        Idev = reinterpret_cast<const float*>(ctx->y);
    }
    // 128^2 cluster shape: the cached choice, or timed now on this scan
    int variant = 0;
    if (N == 128 && !two && !tc) {
        if (tuned.divide_tuned) {
            variant = tuned.divide_variant;
        } else if (ctx->tuning) {
            float ms[2] = {0.f, 0.f};
            for (int v = 0; v < 2; ++v) {
                PT_STEP(launch_sqrt_permute(N, v, Idev, ctx->sqrtIp, psum, ctx->dflag, J, st));
                DivideArgs da = divide_args(ctx);
                da.variant = v;
                da.load_x = 0;
                da.pa = da.pb = da.c = 1.f;
                da.err_only = 1;   // writes only the error partials and the scratch
                cudaEvent_t e0, e1;
                PT_STEP(cudaEventCreate(&e0));
                PT_STEP(cudaEventCreate(&e1));
                e = launch_divide(N, da, st);
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                    if (rep == 1) e = cudaEventRecord(e0, st);
                    if (e == cudaSuccess) e = launch_divide(N, da, st);
                }
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[v], e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (e != cudaSuccess) return bail(e, "128^2 cluster-shape timing");
                ms[v] /= 2.f;
            }
            variant = ms[1] < ms[0] ? 1 : 0;
            tune_store_divide(ctx->opts.device, N, J, variant, ms);
        }
    }
    ctx->variant = variant;
    ctx->C = divide_cluster_size(N, variant);
    if (two)
        PT_STEP(launch_sqrt_permute2p(Idev, ctx->sqrtIp, psum, ctx->dflag, J, st));
    else
        PT_STEP(launch_sqrt_permute(N, variant, Idev, ctx->sqrtIp, psum, ctx->dflag, J, st));
    if (tc) {
        PT_STEP(bf16x3_prepare());
        PT_STEP(launch_sqrt_intensity(N, Idev, ctx->sqrtI, J, st));
        std::vector<uint16_t> Bh[4];
        bf16x3_constants(N, Bh[0], Bh[1], Bh[2], Bh[3]);
        for (int i = 0; i < 4; ++i)
            PT_STEP(cudaMemcpyAsync(ctx->Bc[i], Bh[i].data(), Bh[i].size() * sizeof(uint16_t),
                                    cudaMemcpyHostToDevice, st));
        PT_STEP(cudaStreamSynchronize(st));  // the host vectors go out of scope
    }
    PT_STEP(launch_form_waves(ctx->x, ctx->P, ctx->O, ctx->pos, J, N, M_cols, st));
    std::vector<double> hsum((size_t)J * sq_blocks);
    int bad = 0;
    PT_STEP(cudaMemcpyAsync(hsum.data(), psum, hsum.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    PT_STEP(cudaMemcpyAsync(&bad, ctx->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PT_STEP(cudaStreamSynchronize(st));
#undef PT_STEP
    if (bad) {
        free_scan(ctx);
        return fail(ctx, PTYCHO_EINVAL, "intensity has a negative or non-finite value");
    }
    double s = 0.0;
    for (double v : hsum) s += v;
    ctx->sumI = s;
    ctx->loaded = true;
    ctx->have_x = true;
    ctx->pa = ctx->pb = 1.f;
    ctx->iters = 0;
    return PTYCHO_OK;
}

int ptycho_iterate(ptycho_ctx* ctx, float a, float b, float c, int32_t n_iter) {
    NvtxRange nvtx_range("ptycho_iterate");
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c))
        return fail(ctx, PTYCHO_EINVAL, "a, b, c must be finite");
    if (n_iter < 0) return fail(ctx, PTYCHO_EINVAL, "n_iter must be >= 0");
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    DeviceGuard dg(ctx->opts.device);
    for (int it = 0; it < n_iter; ++it) {
        DivideArgs da = iteration_args(ctx, a, b, c);
        const bool rec = ctx->prof && ctx->prof_n < kProfMax;
        if (rec) PT_CUDA(ctx, cudaEventRecord(ctx->ev[3 * ctx->prof_n], ctx->stream));
        int n_part = ctx->n_part;
        if (ctx->opts.precision == PTYCHO_PREC_BF16X3) {
            PT_CUDA(ctx, launch_divide_bf16x3(da, ctx->N, ctx->sqrtI, ctx->planes, ctx->Bc,
                                              ctx->dflag + 1, ctx->stream));
            n_part = bf16x3_error_parts(ctx->N, ctx->J);
        } else {
            PT_CUDA(ctx, launch_divide_ctx(ctx, da));
        }
        if (rec) PT_CUDA(ctx, cudaEventRecord(ctx->ev[3 * ctx->prof_n + 1], ctx->stream));
        if (!ctx->tuned && ctx->tuning && ctx->opts.concur == PTYCHO_CONCUR_DETERMINISTIC) {
            // launch shapes of the concur kernels: the cached choice, or timed now
            // on this iteration's divided exit waves (not while a graph is captured)
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            PT_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
            if (cs == cudaStreamCaptureStatusNone) {
                TuneChoice tc{};
                ConcurScan cscan = concur_scan(ctx, n_part);
                PT_CUDA(ctx, tune_concur(ctx->opts.device, cscan, ctx->pos_h.data(), ctx->stream, &tc));
                ctx->cb = cscan.cb;
                ctx->tuned = true;
            }
        }
        PT_CUDA(ctx, launch_concur(concur_scan(ctx, n_part), ctx->opts.concur,
                                   ctx->iters >= ctx->probe_start, ctx->stream));
        if (rec) {
            PT_CUDA(ctx, cudaEventRecord(ctx->ev[3 * ctx->prof_n + 2], ctx->stream));
            ctx->prof_n++;
        }
        iteration_done(ctx, a, b);
        ctx->iters++;
    }
    return PTYCHO_OK;
}

int ptycho_debug_build(void) { return PT_DBG_ENABLED; }

int ptycho_debug_flags(int device, uint32_t* flags) {
    if (!flags) return PTYCHO_EINVAL;
    *flags = 0u;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PTYCHO_EINVAL;
    }
    DeviceGuard dg(device);
    if (cudaDeviceSynchronize() != cudaSuccess) return PTYCHO_ECUDA;
    unsigned a = 0, b = 0, c = 0;
    if (debug_flags_divide(&a) != cudaSuccess || debug_flags_divide2p(&b) != cudaSuccess ||
        debug_flags_concur(&c) != cudaSuccess)
        return PTYCHO_ECUDA;
    *flags = a | b | c;
    return PTYCHO_OK;
}

int ptycho_set_tuning(ptycho_ctx* ctx, int enable) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    ctx->tuning = enable != 0;
    return PTYCHO_OK;
}

int ptycho_tuning(const ptycho_ctx* ctx, ptycho_tuning_info* out) {
    if (!ctx || !out) return PTYCHO_EINVAL;
    std::memset(out, 0, sizeof(*out));
    if (!ctx->loaded) return PTYCHO_ESTATE;
    const TuneChoice c = tune_lookup(ctx->opts.device, ctx->N, ctx->J);
    out->tuned = ctx->tuned ? 1 : 0;
    out->gather_rows = kGatherShape[ctx->cb.gather_shape].rows;
    out->gather_cols = kGatherShape[ctx->cb.gather_shape].cols;
    out->probe_ppt = ctx->cb.probe_ppt;
    for (int s = 0; s < kGatherShapes && s < 4; ++s) out->gather_ms[s] = c.gather_ms[s];
    out->probe_ms[0] = c.probe_ms[0];
    out->probe_ms[1] = c.probe_ms[1];
    out->cluster_size = ctx->divide == PTYCHO_DIVIDE_CLUSTER ? ctx->C : 0;
    out->divide_ms[0] = c.divide_ms[0];
    out->divide_ms[1] = c.divide_ms[1];
    return PTYCHO_OK;
}

int ptycho_set_launch_shapes(ptycho_ctx* ctx, int32_t gather_rows, int32_t gather_cols,
                             int32_t probe_ppt, int32_t cluster_size) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    int shape = -1;
    for (int s = 0; s < kGatherShapes; ++s)
        if (kGatherShape[s].rows == gather_rows && kGatherShape[s].cols == gather_cols) shape = s;
    if (shape < 0 || (probe_ppt != 1 && probe_ppt != 2))
        return fail(ctx, PTYCHO_EINVAL, "not a candidate launch shape");
    int variant = ctx->variant;
    if (cluster_size != 0) {
        if (ctx->N != 128 || ctx->divide != PTYCHO_DIVIDE_CLUSTER ||
            ctx->opts.precision != PTYCHO_PREC_FP32 || (cluster_size != 8 && cluster_size != 16))
            return fail(ctx, PTYCHO_EINVAL, "cluster size: 8 or 16, FP32 cluster design at N = 128 only");
        variant = cluster_size == 16 ? 1 : 0;
    }
    DeviceGuard dg(ctx->opts.device);
    if (variant != ctx->variant) {
        // sqrt(I) into the other variant's layout, through the transpose scratch
        // (J slots of N^2 complex values hold the J N^2 floats)
        const size_t n = (size_t)ctx->J * ctx->N * ctx->N;
        PT_CUDA(ctx, cudaMemcpyAsync(ctx->scratch, ctx->sqrtIp, n * sizeof(float),
                                     cudaMemcpyDeviceToDevice, ctx->stream));
        PT_CUDA(ctx, launch_relayout_sqrt(ctx->N, ctx->variant, variant,
                                          reinterpret_cast<const float*>(ctx->scratch), ctx->sqrtIp,
                                          ctx->J, ctx->stream));
        ctx->variant = variant;
        ctx->C = divide_cluster_size(ctx->N, variant);
    }
    PT_CUDA(ctx, tune_apply_shape(ctx->pos_h.data(), ctx->J, ctx->N, ctx->Mr, ctx->Mc, shape, ctx->cb,
                                  ctx->stream));
    ctx->cb.probe_ppt = probe_ppt;
    ctx->tuned = true;   // pinned: no tuning at the next iteration
    return PTYCHO_OK;
}

int ptycho_set_probe_start(ptycho_ctx* ctx, int32_t start) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (start < 0) return fail(ctx, PTYCHO_EINVAL, "start must be >= 0");
    ctx->probe_start = start;
    return PTYCHO_OK;
}

int ptycho_get_object_probe(ptycho_ctx* ctx, float* obj_out, float* probe_out) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    DeviceGuard dg(ctx->opts.device);
    if (obj_out)
        PT_CUDA(ctx, cudaMemcpyAsync(obj_out, ctx->O, (size_t)ctx->Mr * ctx->Mc * sizeof(float2),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    if (probe_out)
        PT_CUDA(ctx, cudaMemcpyAsync(probe_out, ctx->P, (size_t)ctx->N * ctx->N * sizeof(float2),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_flags(ctx);
}

int ptycho_set_object_probe(ptycho_ctx* ctx, const float* obj, const float* probe) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    const size_t M = (size_t)ctx->Mr * ctx->Mc, NN = (size_t)ctx->N * ctx->N;
    if (obj && !all_finite(obj, 2 * M)) return fail(ctx, PTYCHO_EINVAL, "object has a non-finite value");
    if (probe && !all_finite(probe, 2 * NN)) return fail(ctx, PTYCHO_EINVAL, "probe has a non-finite value");
    DeviceGuard dg(ctx->opts.device);
    // the pending re-split uses the object and probe: fix x first
    int rc = materialise(ctx);
    if (rc) return rc;
    if (obj)
        PT_CUDA(ctx, cudaMemcpyAsync(ctx->O, obj, M * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    if (probe)
        PT_CUDA(ctx, cudaMemcpyAsync(ctx->P, probe, NN * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PTYCHO_OK;
}

int ptycho_get_exit_waves(ptycho_ctx* ctx, float* x_out) {
    if (!ctx || !x_out) return ctx ? fail(ctx, PTYCHO_EINVAL, "x_out is NULL") : PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    DeviceGuard dg(ctx->opts.device);
    int rc = materialise(ctx);
    if (rc) return rc;
    PT_CUDA(ctx, cudaMemcpyAsync(x_out, ctx->x, (size_t)ctx->J * ctx->N * ctx->N * sizeof(float2),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_flags(ctx);
}

int ptycho_set_exit_waves(ptycho_ctx* ctx, const float* x) {
    if (!ctx || !x) return ctx ? fail(ctx, PTYCHO_EINVAL, "x is NULL") : PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    const size_t n = (size_t)ctx->J * ctx->N * ctx->N;
    if (!all_finite(x, 2 * n)) return fail(ctx, PTYCHO_EINVAL, "x has a non-finite value");
    DeviceGuard dg(ctx->opts.device);
    PT_CUDA(ctx, cudaMemcpyAsync(ctx->x, x, n * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->have_x = true;
    ctx->pa = ctx->pb = 1.f;
    return PTYCHO_OK;
}

int ptycho_errors(ptycho_ctx* ctx, double* fourier_err, int32_t cap, int32_t* n_written) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (cap < 0 || (cap > 0 && !fourier_err) || !n_written)
        return fail(ctx, PTYCHO_EINVAL, "bad output buffer");
    *n_written = 0;
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    DeviceGuard dg(ctx->opts.device);
    const int64_t have = ctx->iters < kRing ? ctx->iters : kRing;
    const int64_t first = ctx->iters - have;  // oldest kept iteration
    const int32_t n = (int32_t)(have < cap ? have : cap);
    std::vector<double> ring((size_t)(have > 0 ? kRing : 0));
    if (have > 0) {
        PT_CUDA(ctx, cudaMemcpyAsync(ring.data(), ctx->e_ring, (size_t)kRing * sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    }
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int32_t i = 0; i < n; ++i) fourier_err[i] = ring[(size_t)((first + i) % kRing)];
    *n_written = n;
    return check_device_flags(ctx);
}

int64_t ptycho_iteration_count(const ptycho_ctx* ctx) { return ctx && ctx->loaded ? ctx->iters : 0; }

int ptycho_model_error(ptycho_ctx* ctx, double* fourier_err) {
    NvtxRange nvtx_range("ptycho_model_error");
    if (!ctx || !fourier_err) return ctx ? fail(ctx, PTYCHO_EINVAL, "NULL output") : PTYCHO_EINVAL;
    ctx->err.clear();
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    DeviceGuard dg(ctx->opts.device);
    DivideArgs da = divide_args(ctx);
    da.load_x = 0;
    da.pa = 1.f;
    da.pb = 1.f;
    da.c = 1.f;
    da.write_x = 0;
    da.err_only = 1;
    PT_CUDA(ctx, launch_divide_ctx(ctx, da));
    PT_CUDA(ctx, launch_sum_parts(ctx->e_part, ctx->n_part, ctx->sumI > 0 ? 1.0 / ctx->sumI : 1.0,
                                  ctx->e_tmp, ctx->e_tmp + 4, ctx->stream));
    PT_CUDA(ctx, cudaMemcpyAsync(fourier_err, ctx->e_tmp, sizeof(double), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_device_flags(ctx);
}

size_t ptycho_device_bytes(const ptycho_ctx* ctx) { return ctx ? ctx->bytes : 0; }

int ptycho_sp_iterate(ptycho_ctx* ctx, float lam, const int32_t* order, int32_t n_iter) {
    NvtxRange nvtx_range("ptycho_sp_iterate");
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    if (!std::isfinite(lam)) return fail(ctx, PTYCHO_EINVAL, "lam must be finite");
    if (n_iter < 0) return fail(ctx, PTYCHO_EINVAL, "n_iter must be >= 0");
    if (!ctx->loaded) return fail(ctx, PTYCHO_ESTATE, "no scan loaded");
    std::vector<int32_t> ord((size_t)ctx->J);
    if (order) {
        std::vector<char> seen((size_t)ctx->J, 0);
        for (int i = 0; i < ctx->J; ++i) {
            const int32_t v = order[i];
            if (v < 0 || v >= ctx->J || seen[(size_t)v])
                return fail(ctx, PTYCHO_EINVAL, "order is not a permutation of 0..J-1");
            seen[(size_t)v] = 1;
            ord[(size_t)i] = v;
        }
    } else {
        for (int i = 0; i < ctx->J; ++i) ord[(size_t)i] = i;
    }
    if (n_iter == 0) return PTYCHO_OK;
    DeviceGuard dg(ctx->opts.device);
    const double inv_sumI = ctx->sumI > 0 ? 1.0 / ctx->sumI : 1.0;
    DivideArgs da = divide_args(ctx);
    da.P_mut = ctx->P;
    da.O_mut = ctx->O;
    da.load_x = 0;
    da.pa = 1.f;  // the exit wave P * O_j
    da.pb = 1.f;
    da.c = lam;
    da.write_x = 0;
    da.err_only = 0;
    da.sp = 1;
    da.lag = 1;  // one exit wave: its phases back to back
    for (int it = 0; it < n_iter; ++it) {
        for (int i = 0; i < ctx->J; ++i) {
            da.sp_pos = ord[(size_t)i];
            PT_CUDA(ctx, launch_divide_ctx(ctx, da));
        }
        PT_CUDA(ctx, launch_record_error(ctx->e_part, ctx->n_part, inv_sumI, ctx->e_ring,
                                         ctx->d_iter, kRing, ctx->e_tmp + 4, ctx->stream));
        ctx->iters++;
    }
    // the product-space iterate follows the new object and probe
    PT_CUDA(ctx, launch_form_waves(ctx->x, ctx->P, ctx->O, ctx->pos, ctx->J, ctx->N, ctx->Mc,
                                   ctx->stream));
    ctx->have_x = true;
    ctx->pa = ctx->pb = 1.f;
    return PTYCHO_OK;
}

int ptycho_profile_enable(ptycho_ctx* ctx, int enable) {
    if (!ctx) return PTYCHO_EINVAL;
    ctx->err.clear();
    DeviceGuard dg(ctx->opts.device);
    if (enable) {
        while (ctx->ev.size() < (size_t)3 * kProfMax) {
            cudaEvent_t e;
            PT_CUDA(ctx, cudaEventCreate(&e));
            ctx->ev.push_back(e);
        }
        ctx->prof_n = 0;
    }
    ctx->prof = enable != 0;
    return PTYCHO_OK;
}

int ptycho_profile_read(ptycho_ctx* ctx, double* divide_ms, double* concur_ms, int32_t* n_iters) {
    if (!ctx || !divide_ms || !concur_ms || !n_iters) return PTYCHO_EINVAL;
    ctx->err.clear();
    DeviceGuard dg(ctx->opts.device);
    PT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double d = 0.0, c = 0.0;
    for (int i = 0; i < ctx->prof_n; ++i) {
        float a = 0.f, b = 0.f;
        PT_CUDA(ctx, cudaEventElapsedTime(&a, ctx->ev[3 * i], ctx->ev[3 * i + 1]));
        PT_CUDA(ctx, cudaEventElapsedTime(&b, ctx->ev[3 * i + 1], ctx->ev[3 * i + 2]));
        d += a;
        c += b;
    }
    *divide_ms = d;
    *concur_ms = c;
    *n_iters = ctx->prof_n;
    return PTYCHO_OK;
}

}  // extern "C"
