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
    double* e_part;       // [J][C] per-CTA partial of sum (|Psi| - sqrt I)^2
    int J;
    int Mc;               // object row stride (columns)
    int load_x;           // 1: x_k is x[] (no re-split); 0: x_k = re-split(pa, pb)
    float pa, pb;         // re-split coefficients of the previous iteration
    float c;              // divide relaxation
    int write_x;          // store x_k to x[] (needed when this iteration's a != 1)
    int err_only;         // only the Fourier error of x_k (no y written)
    float2* scratch;      // [J][N^2] transpose scratch (row pass -> column pass)
    int reserved;         // unused; keeps the parameter layout below (the divide kernel
                          // measured 1 % slower at 256^2 with this field removed)
    int sp;               // 1: one sequential-projections step (at position sp_pos)
    int sp_pos;
    float2* P_mut;        // probe and object updated by a sequential-projections step
    float2* O_mut;
};

// Supported pattern sides.
bool divide_supported(int N);
int divide_cluster_size(int N);
// Twiddle table of the divide kernel for side N (host, FP64 rounded to FP32).
void divide_twiddles(int N, std::vector<float2>& tw);
cudaError_t divide_prepare(int N);  // one-time kernel attributes
cudaError_t launch_divide(int N, const DivideArgs& a, cudaStream_t st);
// sqrt of the intensities into the divide kernel's frequency order; flags
// *bad (device int) if any value is negative or not finite; per-pattern sums
// of I in FP64 into psum[J].
cudaError_t launch_sqrt_permute(int N, const float* I, float* sqrtIp, double* psum, int* bad,
                                int J, cudaStream_t st);

// Concur step and elementwise kernels (concur.cu).
struct ConcurBufs {
    float2* numO;          // [M] object numerator
    float* denO;           // [M] object denominator
    unsigned* maxO;        // bits of max(denO) (float, >= 0)
    float2* partP;         // [chunks][N*N] probe numerator partials
    float* partPd;         // [chunks][N*N] probe denominator partials
    double2* numP;         // [N*N]
    double* denP;          // [N*N]
    unsigned long long* maxP;  // bits of max(denP) (double, >= 0)
    double* e_slice;       // [probe_reduce_blocks(N, chunks)] FP64 slice totals of the Fourier-error partials
    int* tile_ptr;         // [tiles + 1] CSR of positions overlapping each object tile
    int4* tile_win;        // CSR entries (position j, window row, window col, 0)
    int tiles_r, tiles_c, chunks;
};
#ifndef PTYCHO_OBJ_TILE_R
#define PTYCHO_OBJ_TILE_R 16
#endif
#ifndef PTYCHO_OBJ_TILE_C
#define PTYCHO_OBJ_TILE_C 32
#endif
constexpr int kObjTileR = PTYCHO_OBJ_TILE_R;  // object tile rows of the gather
constexpr int kObjTile = PTYCHO_OBJ_TILE_C;   // object tile columns
int probe_chunks(int J, int N);
int probe_reduce_blocks(int N, int chunks);  // blocks of the probe reduction (one error slice each)
cudaError_t launch_concur(const float2* y, float2* P, float2* O, const int2* pos,
                          const ConcurBufs& cb, int J, int N, int Mr, int Mc, float alpha,
                          const double* e_part, int n_part, double inv_sumI, double* e_ring,
                          unsigned long long* d_iter, int ring_cap, int concur_mode,
                          cudaStream_t st);
cudaError_t launch_form_waves(float2* x, const float2* P, const float2* O, const int2* pos,
                              int J, int N, int Mc, cudaStream_t st);
cudaError_t launch_materialise(float2* x, const float2* y, const float2* P, const float2* O,
                               const int2* pos, int J, int N, int Mc, float pa, float pb,
                               cudaStream_t st);
cudaError_t launch_sum_parts(const double* parts, int n, double scale, double* out,
                             cudaStream_t st);
// FP64 sum of parts times scale into ring[*d_iter % cap], then ++*d_iter.
cudaError_t launch_record_error(const double* parts, int n, double scale, double* ring,
                                unsigned long long* d_iter, int cap, cudaStream_t st);

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

// Context internals used by the batching and serving runtime (serve.cu).
}  // namespace ptycho
struct ptycho_ctx;
namespace ptycho {
cudaStream_t ctx_stream(const ptycho_ctx* ctx);
int ctx_device(const ptycho_ctx* ctx);
bool ctx_loaded(const ptycho_ctx* ctx);
// Account for iterations that ran as replays of a captured graph.
void ctx_add_iterations(ptycho_ctx* ctx, int64_t n);

}  // namespace ptycho
