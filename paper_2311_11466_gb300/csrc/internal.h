// Internal interfaces between the library's translation units (not the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ptycho {

// Arguments of the divide kernel (one cluster of CTAs per exit wave).
struct DivideArgs {
    float2* x;            // [J][N][N] current iterate (read in LOADX mode / as x_prev)
    float2* y;            // [J][N][N] divide output y = P^c_D x (in: y_prev for the re-split)
    const float* sqrtIp;  // [J][N*N] sqrt(I_j) in the kernel's frequency order
    const float2* P;      // [N][N] probe
    const float2* O;      // [M_rows][M_cols] object
    const int2* pos;      // [J] (row, col)
    const float2* tw;     // [N] stage twiddles, see divide.cu
    double* e_part;       // per-wave partials of sum (|Psi| - sqrt I)^2 (divide_error_parts_per_wave)
    int J;
    int Mr;               // object rows
    int Mc;               // object row stride (columns)
    int load_x;           // 1: x_k is x[] (no re-split); 0: x_k = re-split(pa, pb)
    float pa, pb;         // re-split coefficients of the previous iteration
    float c;              // divide relaxation
    int write_x;          // store x_k to x[] (needed when this iteration's a != 1)
    int err_only;         // only the Fourier error of x_k (no y written)
    float2* scratch;      // cluster variant: [J][N^2] transpose scratch (row pass -> column
                          // pass); two-pass variant: [ring][N^2] (Fourier error only, SP)
    int sp;               // 1: one sequential-projections step (at position sp_pos)
    int sp_pos;
    float2* P_mut;        // probe and object updated by a sequential-projections step
    float2* O_mut;
    // two-pass variant only
    unsigned* ctl;        // [4 + 2 J] ticket, SP maxima, per-wave completion counts
    int lag;              // waves between the row, column and inverse-row phases
    int ring;             // scratch slots of the Fourier-error-only mode
    int* err_flag;        // set when a bounded wait expires
    int variant;          // cluster design: launch variant (128^2: 0 clusters of 8 CTAs of
                          // 128 threads, 1 clusters of 16 CTAs of 64; same arithmetic)
};

// Supported pattern sides.
bool divide_supported(int N);
// CTAs per exit wave of the cluster design (variant: the launch variant, see
// DivideArgs::variant); also the number of Fourier-error partials per wave.
int divide_cluster_size(int N, int variant = 0);
constexpr int kMaxClusterSize = 16;
// Fourier-error partials per exit wave: one per column frequency (cluster
// design), one per column band (two-pass design, 16).
inline int divide_error_parts_per_wave(int N, bool two_pass) { return two_pass ? 16 : N; }
// Twiddle table of the divide kernel for side N (host, FP64 rounded to FP32).
void divide_twiddles(int N, std::vector<float2>& tw);
cudaError_t divide_prepare(int N);  // one-time kernel attributes
cudaError_t launch_divide(int N, const DivideArgs& a, cudaStream_t st);
// The divide step of n scans of side N (cluster design, launch variant
// `variant`) in one launch: device table[n] of their arguments, first[n + 1]
// the prefix of their wave counts (batching).
cudaError_t launch_divide_ragged(int N, int variant, const DivideArgs* table, const int* first,
                                 int n, int total_waves, cudaStream_t st);
// sqrt of the intensities into the divide kernel's frequency order; flags
// *bad (device int) if any value is negative or not finite; per-pattern sums
// of I in FP64 into psum[J].
cudaError_t launch_sqrt_permute(int N, int variant, const float* I, float* sqrtIp, double* psum,
                                int* bad, int J, cudaStream_t st);
// sqrt(I) from the layout of one launch variant to another's (N = 128).
cudaError_t launch_relayout_sqrt(int N, int from, int to, const float* src, float* dst, int J,
                                 cudaStream_t st);

// Two-pass (row / column through L2, no clusters) divide variant, N = 256
// (divide2p.cu).  Same arguments; sqrt(I) in its own order.
bool divide2p_supported(int N);
int divide2p_lag();
int divide2p_ring();
size_t divide2p_ctl_words(int J);
cudaError_t divide2p_prepare();
cudaError_t launch_divide2p(const DivideArgs& a, cudaStream_t st);
cudaError_t launch_sqrt_permute2p(const float* I, float* sqrtIp, double* psum, int* bad, int J,
                                  cudaStream_t st);

// Checked build: read and clear each translation unit's flag word (debug.cuh).
cudaError_t debug_flags_divide(unsigned* out);
cudaError_t debug_flags_divide2p(unsigned* out);
cudaError_t debug_flags_concur(unsigned* out);

// Concur step and elementwise kernels (concur.cu).
struct ConcurBufs {
    float2* numO;          // [M] object numerator
    double* denO;          // [M] object denominator (FP64 final reduction)
    unsigned long long* maxO;  // bits of max(denO) (double, >= 0)
    float2* partP;         // [chunks][N*N] probe numerator partials
    float* partPd;         // [chunks][N*N] probe denominator partials
    double2* numP;         // [N*N]
    double* denP;          // [N*N]
    unsigned long long* maxP;  // bits of max(denP) (double, >= 0)
    double* e_slice;       // [probe_reduce_blocks(N, chunks)] FP64 slice totals of the Fourier-error partials
    int* tile_ptr;         // [tiles + 1] CSR of positions overlapping each object tile
    int4* tile_win;        // CSR entries (position j, window row, window col, 0)
    int tiles_r, tiles_c, chunks;
    int gather_shape;      // index into kGatherShape (a launch choice; same results)
    int probe_ppt;         // probe-partial pixels per thread, 1 or 2 (same results)
    // staged-atomic object concur (PTYCHO_CONCUR_ATOMIC): positions in a
    // spatial order, grouped so that a group's windows, band by band, fit a
    // shared-memory box
    int* sc_ord;           // [J] position indices, spatial order
    int4* sc_groups;       // [sc_n] {first index into sc_ord, count, row min, col min}
    int2* sc_ext;          // [sc_n] {row max - row min, col max - col min}
    int sc_n;              // number of groups
    int sc_rows;           // window rows per band (one CTA per group and band)
    int sc_box;            // largest box of any group, pixels (shared memory: 12 B each)
};

// Object-gather tile shapes (rows x columns of the object) the tuner chooses
// among; index 0 is the default.
struct TileShape {
    int rows, cols;
};
constexpr int kGatherShapes = 4;
constexpr TileShape kGatherShape[kGatherShapes] = {{16, 32}, {8, 32}, {32, 32}, {8, 64}};
// Host: CSR lists of the positions whose window overlaps each tile of shape s,
// in ascending position order; ptr has tiles + 1 entries.
void build_tile_csr(const int32_t* pos_rc, int J, int N, int Mr, int Mc, TileShape s,
                    std::vector<int>& ptr, std::vector<int4>& list);
// Upper bounds over every shape: tiles + 1 and CSR entries.
size_t tile_csr_ptr_bound(int N, int Mr, int Mc);
size_t tile_csr_entries_bound(int J, int N);
// Host: position groups of the staged-atomic object concur (at most J groups).
// Returns the window rows per band and the largest group box in pixels.
void build_scatter_groups(const int32_t* pos_rc, int J, int N, std::vector<int>& ord,
                          std::vector<int4>& groups, std::vector<int2>& ext, int* rows, int* box);
// Shared-memory limit of the staged-atomic kernel on the current device.
cudaError_t concur_prepare();
// Everything the concur step of one scan needs on the device.
struct ConcurScan {
    const float2* y;
    float2* P;
    float2* O;
    const int2* pos;
    ConcurBufs cb;
    int J, N, Mr, Mc;
    double alpha;
    const double* e_part;      // the divide step's Fourier-error partials
    int n_part;
    double inv_sumI;
    double* e_ring;            // per-iteration error history
    unsigned long long* d_iter;
    int ring_cap;
};
cudaError_t launch_gather(const ConcurScan& cs, cudaStream_t st);
cudaError_t launch_probe_partial(const ConcurScan& cs, cudaStream_t st);
// The concur step of several scans in one launch per kernel (batching): the
// scans must share the gather shape and the probe pixels per thread.
struct RaggedConcur {
    const ConcurScan* scans;   // device [n]
    const int* first;          // device [5][n + 1] block prefixes (gather, object normalise,
                               // probe partial, probe reduce, probe normalise)
    const int* n_slice;        // device [n] probe-reduce blocks of each scan
    int n;
    int totals[5];
    int gather_shape, probe_ppt;
};
void ragged_concur_tables(const ConcurScan* scans, int n, std::vector<int>& first,
                          std::vector<int>& n_slice, int totals[5]);
cudaError_t launch_concur_ragged(const RaggedConcur& rc, cudaStream_t st);
int probe_chunks(int J, int N);
int probe_reduce_blocks(int N, int chunks);  // blocks of the probe reduction (one error slice each)
cudaError_t launch_concur(const ConcurScan& cs, int concur_mode, bool update_probe, cudaStream_t st);

cudaError_t launch_form_waves(float2* x, const float2* P, const float2* O, const int2* pos,
                              int J, int N, int Mc, cudaStream_t st);
cudaError_t launch_materialise(float2* x, const float2* y, const float2* P, const float2* O,
                               const int2* pos, int J, int N, int Mc, float pa, float pb,
                               cudaStream_t st);

// FP64 sum of parts times scale into *out (scratch: 256 doubles for the
// slice totals of a long list).
cudaError_t launch_sum_parts(const double* parts, int n, double scale, double* out,
                             double* scratch, cudaStream_t st);
// FP64 sum of parts times scale into ring[*d_iter % cap], then ++*d_iter.
cudaError_t launch_record_error(const double* parts, int n, double scale, double* ring,
                                unsigned long long* d_iter, int cap, double* scratch,
                                cudaStream_t st);

// Tensor-core (BF16 x 3) divide path (dft_gemm.cu).
bool bf16x3_supported(int N);
int bf16x3_tiles(int N, int J);
int bf16x3_error_parts(int N, int J);
void bf16x3_constants(int N, std::vector<uint16_t>& fwd_hi, std::vector<uint16_t>& fwd_lo,
                      std::vector<uint16_t>& inv_hi, std::vector<uint16_t>& inv_lo);
cudaError_t bf16x3_prepare();
cudaError_t launch_sqrt_intensity(int N, const float* I, float* out, int J, cudaStream_t st);
cudaError_t launch_divide_bf16x3(const DivideArgs& a, int N, const float* sqrtI,
                                 uint16_t* const planes[4], const uint16_t* const B[4],
                                 int* err_flag, cudaStream_t st);

// Divide design resolved for (precision, requested design, N): 1 cluster, 2 two-pass.
int resolve_divide(int precision, int divide, int N);
size_t scan_bytes(int J, int N, int M_rows, int M_cols, int precision, int divide);

// Autotuner of launch shapes (tune.cu); every choice gives bit-identical results.
struct TuneChoice {
    bool valid = false;               // the concur shapes were timed
    int gather_shape = 0;             // index into kGatherShape
    int probe_ppt = 1;                // probe-partial pixels per thread
    float gather_ms[kGatherShapes] = {0.f, 0.f, 0.f, 0.f};
    float probe_ms[2] = {0.f, 0.f};
    bool divide_tuned = false;        // the 128^2 cluster shape was timed
    int divide_variant = 0;           // 128^2: 0 clusters of 8 x 128 threads, 1 of 16 x 64
    float divide_ms[2] = {0.f, 0.f};
};
// The cached choice for (device, N, J bucket), or the defaults (valid = false).
TuneChoice tune_lookup(int device, int N, int J);
// Time the concur candidates on the context's data (once per kind of scan),
// then set cb to the chosen shapes.  Synchronises st.
cudaError_t tune_concur(int device, ConcurScan& cs, const int32_t* pos_rc_host, cudaStream_t st,
                        TuneChoice* out);
void tune_store_divide(int device, int N, int J, int variant, const float ms[2]);
// Upload the tile lists of gather shape `shape` and set cb to it.  Synchronises st.
cudaError_t tune_apply_shape(const int32_t* pos_rc_host, int J, int N, int Mr, int Mc, int shape,
                             ConcurBufs& cb, cudaStream_t st);

// Context internals used by the batching and serving runtime (serve.cu).
}  // namespace ptycho
struct ptycho_ctx;
namespace ptycho {
cudaStream_t ctx_stream(const ptycho_ctx* ctx);
int ctx_device(const ptycho_ctx* ctx);
bool ctx_loaded(const ptycho_ctx* ctx);
// Account for iterations that ran as replays of a captured graph.
void ctx_add_iterations(ptycho_ctx* ctx, int64_t n);
// Iterations still to run with the probe held fixed (0: the probe is updated).
int64_t ctx_probe_hold(const ptycho_ctx* ctx);
// The device arguments of the context's next abc iteration with (a, b, c), for
// a batched launch; false when that iteration cannot join one (tensor-core
// precision, two-pass design, atomic concur, probe held, first iteration).
// *N and *variant give the launch group.
bool ctx_ragged_iteration(ptycho_ctx* ctx, float a, float b, float c, DivideArgs* da,
                          ConcurScan* cs, int* N, int* variant);
// After iterations with (a, b) that ran in a replayed graph: the context's
// host-side state, and its iteration count set to n.
void ctx_batch_done(ptycho_ctx* ctx, float a, float b, int64_t n);
int64_t ctx_iterations(const ptycho_ctx* ctx);

}  // namespace ptycho
