/*
 * ptycho.h — C ABI of the GB300 blind-ptychography set-projection library.
 *
 * Method: W. Mei, A. M. Maiden, "Set projection algorithms for blind
 * ptychographic phase retrieval" (arXiv 2311.11466).  One call of
 * ptycho_iterate runs the paper's generalised divide-and-concur update
 * (Introduction, the displayed equation)
 *
 *     x_{k+1} = a P^b_C P^c_D x_k + (1 - a) x_k
 *
 * over the stack x = [x_0 .. x_{J-1}] of per-position exit waves (the product
 * space of Fig. 3), following the flow of Fig. 4: exit waves for all scan
 * positions -> projections -> updated probe and object.
 *
 *   P_D  (divide, Fig. 3(a)): per position, Psi = F x_j, replace |Psi| by the
 *        measured sqrt(I_j) (phase kept; sqrt(I_j) where Psi = 0), F^{-1}.
 *   P_C  (concur, Fig. 3(b)): least-squares consensus {P * O_j}: the object
 *        from the current probe, then the probe from the new object, each as
 *        sum conj(.) y / (sum |.|^2 + alpha * max(sum |.|^2)), re-split z_j = P * O_j.
 *   P^a_S = a P^1_S + (1 - a) I (relaxed projection, Introduction).
 *
 * DC = (1,1,1), AR = (1,2,2), DR = (1/2,2,2), SF = (1,2,1),
 * RAAR(beta) = (1/2, 2 beta, 2), RRR(beta) = (beta/2, 2, 2) are settings of the
 * same call.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - F is the unnormalised 2-D DFT exp(-2 pi i q.r / N); F^{-1} carries 1/N^2;
 *    no fftshift: intensities are stored with zero frequency at [0][0].
 *  - Complex arrays are interleaved float32 (re, im), row-major:
 *    object [M_rows][M_cols][2], probe [N][N][2], exit waves [J][N][N][2].
 *  - Positions are int32 [J][2] = (row, col) of the window's top-left corner
 *    in the object: O_j(r) = O(s_j + r), r in [0, N)^2.
 *  - Every function returns a ptycho_status; on error, ptycho_last_error()
 *    gives a one-line reason.  Inputs are copied: the caller keeps ownership
 *    of every buffer it passes.  Outputs go to caller-allocated host buffers.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - All device work of a context runs on its stream, asynchronously unless a
 *    function says it synchronises.
 */
#ifndef PTYCHO_H
#define PTYCHO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PTYCHO_OK = 0,
    PTYCHO_EINVAL = -1,    /* bad argument (size, range, non-finite value) */
    PTYCHO_ENOMEM = -2,    /* device allocation failed or exceeds a budget */
    PTYCHO_ECUDA = -3,     /* a CUDA runtime call failed */
    PTYCHO_ETIMEOUT = -4,  /* a bounded device wait expired */
    PTYCHO_ESTATE = -5     /* call not valid in the context's current state */
} ptycho_status;

/* Precision of the divide step's transforms. */
enum { PTYCHO_PREC_FP32 = 0,    /* FP32 shared-memory FFT (default) */
       PTYCHO_PREC_BF16X3 = 1   /* DFT as dense GEMMs on tensor cores, BF16 hi/lo
                                   split with three products, FP32 accumulation */ };

/* How the concur step (Fig. 3(b)) accumulates the object and probe numerators
 * and denominators.  DETERMINISTIC: the object by a position-tiled gather and
 * the probe by an ordered two-level reduction; bitwise reproducible.  ATOMIC:
 * the object by shared-memory-staged atomics (groups of neighbouring
 * positions accumulated band by band in a shared-memory box, then added to the
 * global sums once per box pixel: FP32 numerator, FP64 denominator) and the
 * probe by register-staged FP64 atomics; the same sums in an order that
 * depends on timing, so not bitwise reproducible. */
enum { PTYCHO_CONCUR_DETERMINISTIC = 0,
       PTYCHO_CONCUR_ATOMIC = 1 };

/* Kernel design of the FP32 divide step (Fig. 3(a)); both compute the same
 * update, within FP32 rounding of each other. */
enum { PTYCHO_DIVIDE_AUTO = 0,     /* the faster design for the pattern side */
       PTYCHO_DIVIDE_CLUSTER = 1,  /* one thread-block cluster per exit wave (any N) */
       PTYCHO_DIVIDE_TWOPASS = 2   /* row and column passes through L2 with no
                                      clusters and no transpose buffer (N = 256 only;
                                      other N use the cluster design) */ };

typedef struct {
    int device;      /* CUDA device ordinal */
    int precision;   /* PTYCHO_PREC_* */
    int concur;      /* PTYCHO_CONCUR_* */
    float alpha;     /* denominator regulariser, >= 0 (default 1e-6) */
    void* stream;    /* cudaStream_t to run on, or NULL for a private stream */
    int divide;      /* PTYCHO_DIVIDE_* (default AUTO; the tensor-core precision
                        path always pairs with the cluster design) */
} ptycho_opts;

typedef struct ptycho_ctx ptycho_ctx;

/* Fill *opts with the defaults (device 0, FP32, deterministic, alpha 1e-6,
 * divide design AUTO). */
void ptycho_default_opts(ptycho_opts* opts);

/* Create a context on opts->device.  opts may be NULL for the defaults.
 * Device memory of a context comes from the device's stream-ordered memory
 * pool of this process (allocated and freed on the context's stream); the
 * first context on a device keeps that pool's freed memory mapped for later
 * contexts instead of returning it to the driver at each synchronisation.
 * Errors: EINVAL (bad option), ECUDA. */
int ptycho_create(ptycho_ctx** out, const ptycho_opts* opts);

/* Release every device allocation of the context (back to the pool, without
 * synchronising the device) and its stream if it created one.  NULL is a
 * no-op. */
void ptycho_destroy(ptycho_ctx* ctx);

/* Last error message of the context ("" if none); never NULL.  With
 * ctx == NULL, the last error of ptycho_create on this thread. */
const char* ptycho_last_error(const ptycho_ctx* ctx);

/* Flags of ptycho_load_scan. */
enum { PTYCHO_LOAD_INTENSITY_DEVICE = 1u };  /* intensity is a device pointer */

/* Load one scan and form the initial exit waves x_0,j = P_0 * O_0(s_j + .)
 * (Fig. 4, the first box).  Replaces any scan already loaded.
 *   J          number of positions, >= 1
 *   N          pattern side: 8, 16, 32, 64, 128 or 256
 *   pos_rc     host int32 [J][2]; each must satisfy 0 <= row <= M_rows - N and
 *              0 <= col <= M_cols - N (never clamped: out of range is EINVAL)
 *   intensity  float32 [J][N][N] measured intensities, unshifted, finite, >= 0;
 *              host memory unless flags has PTYCHO_LOAD_INTENSITY_DEVICE
 *   M_rows, M_cols  object size, each >= N
 *   obj0       host complex float32 [M_rows][M_cols], finite (initial object)
 *   probe0     host complex float32 [N][N], finite (initial probe)
 * Synchronises the context's stream.  A scan whose ptycho_scan_bytes exceed
 * the device's free memory fails with ENOMEM before the intensities are read
 * (the context then holds no scan).  Errors: EINVAL, ENOMEM, ECUDA. */
int ptycho_load_scan(ptycho_ctx* ctx, int32_t J, int32_t N, const int32_t* pos_rc,
                     const float* intensity, int32_t M_rows, int32_t M_cols,
                     const float* obj0, const float* probe0, uint32_t flags);

/* Run n_iter iterations of x <- a P^b_C P^c_D x + (1 - a) x, appending the
 * Fourier error E_F(x_k) = sum (|F x_k| - sqrt(I))^2 / sum I of each
 * iteration's input to the context's error history.  Asynchronous on the
 * context's stream.  n_iter = 0 is a no-op.
 * Errors: EINVAL (a, b, c not finite, n_iter < 0), ESTATE (no scan), ECUDA. */
int ptycho_iterate(ptycho_ctx* ctx, float a, float b, float c, int32_t n_iter);

/* Sequential projections (Introduction, Fig. 2): n_iter passes over the
 * positions, each position visited once per pass in the order given
 * (order: host int32 [J], a permutation of 0..J-1, or NULL for ascending).
 * At position j, with psi = P * O_j and psi' = lam P_{S_j}(psi) + (1 - lam) psi
 * (S_j the Fourier-modulus set of position j):
 *     O_j += conj(P) (psi' - psi) / max|P|^2,   P += conj(O_j) (psi' - psi) / max|O_j|^2
 * (O_j before its update on the right).  Appends the Fourier error of each
 * pass to the error history; afterwards the exit waves are P * O_j, so an
 * abc iteration can continue from the result.  Asynchronous.
 * Errors: EINVAL (lam not finite, n_iter < 0, order not a permutation),
 * ESTATE (no scan), ECUDA. */
int ptycho_sp_iterate(ptycho_ctx* ctx, float lam, const int32_t* order, int32_t n_iter);

/* Hold the probe fixed in the concur step of iterations k < start, k counted
 * from 0 at the last ptycho_load_scan: those iterations update the object
 * only (Fig. 3(b), with the probe as known), and the re-split uses the probe
 * as it is.  start = 0 (the default) updates the object and then the probe
 * from the first iteration.  The paper does not say when the probe update
 * begins; this selects the other reading.  The setting stays with the
 * context across loads.  Errors: EINVAL (start < 0). */
int ptycho_set_probe_start(ptycho_ctx* ctx, int32_t start);

/* Launch shapes chosen by the library's autotuner (no counterpart in the
 * paper).  The first iteration of a context whose kind of scan (device, N,
 * floor(log2 J)) this process has not seen times the candidate launch shapes
 * of the concur kernels on the context's data and keeps the fastest; at
 * 128 x 128 the load of such a scan also times two cluster shapes of the
 * divide kernel.  The choice is cached for every later context of that kind.
 * Every candidate computes the same sums in the same order, so results are
 * bit-identical whichever wins. */
typedef struct {
    int32_t tuned;          /* 1 once the concur shapes of this context were chosen */
    int32_t gather_rows;    /* object-gather tile (candidates 16x32, 8x32, 32x32, 8x64) */
    int32_t gather_cols;
    int32_t probe_ppt;      /* probe-partial pixels per thread (1 or 2) */
    float gather_ms[4];     /* measured ms of each gather candidate, in the order above */
    float probe_ms[2];      /* measured ms with 1 and 2 pixels per thread */
    int32_t cluster_size;   /* CTAs per exit wave of the cluster divide kernel (0: two-pass) */
    float divide_ms[2];     /* 128^2: measured ms of clusters of 8 x 128 and 16 x 64 threads */
} ptycho_tuning_info;

/* Enable (default) or disable the autotuner for this context's later loads
 * and first iteration; disabled, it uses the cached choice or the defaults
 * (16 x 32 tiles, 1 pixel per thread, clusters of 8 at 128^2).
 * Errors: EINVAL. */
int ptycho_set_tuning(ptycho_ctx* ctx, int enable);

/* The launch shapes of the context's current scan.  Errors: EINVAL, ESTATE. */
int ptycho_tuning(const ptycho_ctx* ctx, ptycho_tuning_info* out);

/* Pin the launch shapes of the loaded scan -- one of the gather tiles listed
 * above, 1 or 2 probe pixels per thread, and at 128 x 128 with the cluster
 * design the cluster size (8 or 16 CTAs per exit wave; 0 keeps the current
 * one) -- and stop tuning this context, for reproducing a measurement or a
 * chosen configuration.  The results do not change.  Synchronises.
 * Errors: EINVAL (not a candidate), ESTATE (no scan), ECUDA. */
int ptycho_set_launch_shapes(ptycho_ctx* ctx, int32_t gather_rows, int32_t gather_cols,
                             int32_t probe_ppt, int32_t cluster_size);

/* Copy the current object [M_rows][M_cols][2] and probe [N][N][2] to host
 * buffers (either may be NULL).  Synchronises.  Errors: ESTATE, ECUDA. */
int ptycho_get_object_probe(ptycho_ctx* ctx, float* obj_out, float* probe_out);

/* Overwrite the object and/or probe (host buffers, either may be NULL).
 * The exit waves are not changed.  Errors: EINVAL (non-finite), ESTATE, ECUDA. */
int ptycho_set_object_probe(ptycho_ctx* ctx, const float* obj, const float* probe);

/* Copy the current iterate x_k [J][N][N][2] to a host buffer.  Synchronises.
 * Errors: ESTATE, ECUDA. */
int ptycho_get_exit_waves(ptycho_ctx* ctx, float* x_out);

/* Replace the current iterate x_k by a host buffer [J][N][N][2].
 * Errors: EINVAL (non-finite), ESTATE, ECUDA. */
int ptycho_set_exit_waves(ptycho_ctx* ctx, const float* x);

/* Copy up to cap entries of the per-iteration Fourier-error history (oldest
 * first, since the last load) to fourier_err; *n_written receives the count.
 * The history keeps the most recent 65536 iterations.  Synchronises.
 * Errors: EINVAL (cap < 0 or NULL pointers with cap > 0), ESTATE, ECUDA. */
int ptycho_errors(ptycho_ctx* ctx, double* fourier_err, int32_t cap, int32_t* n_written);

/* Number of iterations run since the last load (0 without a scan). */
int64_t ptycho_iteration_count(const ptycho_ctx* ctx);

/* Fourier error of the consensus model, E_F(z) with z_j = P * O(s_j + .),
 * for the current object and probe (the final error of a reconstruction).
 * Synchronises.  Errors: ESTATE, ECUDA. */
int ptycho_model_error(ptycho_ctx* ctx, double* fourier_err);

/* Kernel timing for measurement: with enable = 1 the context records CUDA
 * events on its stream around every later launch of the divide kernel and of
 * the concur step (up to 4096 iterations); enable = 0 stops recording, and a
 * new enable = 1 clears what was recorded.  Errors: EINVAL, ECUDA. */
int ptycho_profile_enable(ptycho_ctx* ctx, int enable);

/* Sum of the recorded divide-kernel and concur-step durations in ms and the
 * number of iterations recorded.  Synchronises.  Errors: EINVAL, ECUDA. */
int ptycho_profile_read(ptycho_ctx* ctx, double* divide_ms, double* concur_ms, int32_t* n_iters);

/* Probe update of the concur step with no device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, for example code whose device memory is all owned
 * by its own allocator or pool, or a pipeline that must not allocate once it
 * is running (an allocation there may fail, fragment a pool sized in advance,
 * or stall the device).  It computes, from caller-provided device buffers,
 *     P(r) = sum_j conj(O(s_j + r)) y_j(r) / (sum_j |O(s_j + r)|^2 + alpha max_r(.))
 * (a regularised denominator of exactly 0 gives 0), the same probe update as
 * the concur step of ptycho_iterate, with the same FP32 partial sums over
 * fixed chunks of positions and FP64 final sums.
 *   y          device complex float32 [J][N][N] (the divided exit waves)
 *   obj        device complex float32 [M_rows][M_cols] (the object)
 *   pos_rc     device int32 [J][2] (row, col) window corners
 *   alpha      regulariser, finite, >= 0
 *   probe_out  device complex float32 [N][N], written on success only
 *   stream     cudaStream_t to run on (NULL: the default stream)
 * All buffers stay owned by the caller.  Scratch lives in one static
 * __device__ array of 8.25 MiB that every GPU loading the library holds until
 * the process exits; it bounds N to 256 (every N from 1 to 256 and every
 * J >= 1 fit).  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress, with the device current),
 * so make that first call before any stream capture.  Every call reuses the
 * same array (the maximum and the status word are cleared at the start of
 * each call): calls whose work overlaps on the GPU race and must not be made.
 * Synchronises the stream before returning (to read the status word).
 * Errors: EINVAL (NULL pointer, J < 1, N < 1 or N > 256, M_rows or M_cols
 * < N, bad alpha, or a position whose window leaves the object: such windows
 * are skipped on the device, probe_out is left untouched), ECUDA. */
int ptycho_probe_update_noalloc(const float* y, const float* obj, const int32_t* pos_rc,
                                int32_t J, int32_t N, int32_t M_rows, int32_t M_cols,
                                float alpha, float* probe_out, void* stream);

/* Diagnostic of the failure handling (no counterpart in the paper): every
 * wait inside the library's kernels is bounded in time and reports expiry to
 * the host instead of hanging the device.  This runs such a wait on device
 * `device` on a flag that nothing sets, bounded by timeout_ms (1..10000);
 * the expected result is PTYCHO_ETIMEOUT, after which the device and every
 * context on it remain usable.  Synchronises the device.
 * Errors: EINVAL (bad device or timeout), ECUDA. */
int ptycho_check_bounded_wait(int device, uint32_t timeout_ms);

/* Checked build (no counterpart in the paper): libptycho_debug.so is the same
 * library compiled with device-side checks of object-window bounds, of the
 * sqrt(I) input and of NaN/Inf in the exit waves, object and probe it writes.
 * A failed check records a bit (1 window, 2 non-finite output, 4 bad sqrt(I))
 * and goes on with a safe value; it never traps.  ptycho_debug_build returns
 * 1 in the checked build and 0 otherwise. */
int ptycho_debug_build(void);

/* Synchronise device `device`, then read and clear its check bits into
 * *flags (always 0 in the normal build).  Errors: EINVAL (bad device or
 * NULL), ECUDA. */
int ptycho_debug_flags(int device, uint32_t* flags);

/* Bytes of device memory the context holds for its current scan. */
size_t ptycho_device_bytes(const ptycho_ctx* ctx);

/* Bytes of device memory a scan of this size would need (for admission),
 * with the default (AUTO) divide design. */
size_t ptycho_scan_bytes(int32_t J, int32_t N, int32_t M_rows, int32_t M_cols, int precision);

/* The divide design a context uses for its current scan (PTYCHO_DIVIDE_CLUSTER
 * or PTYCHO_DIVIDE_TWOPASS; 0 without a scan). */
int ptycho_divide_design(const ptycho_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PTYCHO_H */
