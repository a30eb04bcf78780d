// Concur step P^1_C of the abc update (Introduction; Fig. 3(b), "concur":
// one consensus from the divided copies) for blind ptychography, plus the
// elementwise kernels around it.
//
// With an unknown probe the consensus set is the set of stacks {P * O_j}.
// One application is one least-squares sweep: the object with the current
// probe, then the probe with the new object,
//   O(m) = sum_j conj(P(m - s_j)) y_j(m - s_j) / (sum_j |P(m - s_j)|^2 + alpha max)
//   P(r) = sum_j conj(O(s_j + r)) y_j(r)       / (sum_j |O(s_j + r)|^2 + alpha max)
// (a regularised denominator of exactly 0 gives 0).  The re-split
// z_j = P * O_j is not stored: the next divide kernel forms it on the fly.
//
// Determinism: the object is a position-tiled gather (each object tile walks
// the ascending list of windows that overlap it); the probe is a two-level
// reduction over positions (FP32 partials over fixed chunks, FP64 final sum
// in a fixed order: chunk order, or with many chunks contiguous groups of
// chunks added in group order).  Maxima use integer atomicMax on the bit patterns of
// non-negative IEEE values, which is order independent.
#include "common.cuh"
#include "internal.h"

namespace ptycho {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ float block_max_float(float v, float* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) scratch[w] = v;
    __syncthreads();
    float m = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, scratch[i]);
    return m;
}

__device__ __forceinline__ double block_max_double(double v, double* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) scratch[w] = v;
    __syncthreads();
    double m = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, scratch[i]);
    return m;
}

// Object numerator/denominator by position-tiled gather.  One CTA per
// kObjTileR x kObjTile object tile walks its list of overlapping windows (each
// entry carries the position index and the window corner, so one load per
// window); thread i owns column i % kObjTile of rows i / kObjTile + kTRG k.
constexpr int kTRG = kT / kObjTile;       // rows covered by one sweep of the CTA
static_assert(kT % kObjTile == 0 && kObjTileR % kTRG == 0, "object tile shape");

__global__ void __launch_bounds__(kT) concur_object_kernel(
    const float2* __restrict__ y, const float2* __restrict__ P, const int4* __restrict__ tile_win,
    const int* __restrict__ tile_ptr, int N, int Mr, int Mc,
    int tiles_c, float2* __restrict__ numO, float* __restrict__ denO, unsigned* __restrict__ maxO) {
    constexpr int KP = kObjTileR / kTRG;  // pixels per thread
    __shared__ float scratch[kT / 32];
    const int tile = blockIdx.x;
    const int ti = tile / tiles_c, tj = tile % tiles_c;
    const int tx = threadIdx.x % kObjTile, ty = threadIdx.x / kObjTile;
    const int mc = tj * kObjTile + tx;
    const int mr0 = ti * kObjTileR + ty;
    float2 acc[KP];
    float den[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        acc[k] = make_float2(0.f, 0.f);
        den[k] = 0.f;
    }
    const size_t NN = (size_t)N * N;
    const int l0 = tile_ptr[tile], l1 = tile_ptr[tile + 1];
    // deep unrolling keeps several windows' loads in flight per thread
#pragma unroll(KP >= 8 ? 1 : 8 / KP)
    for (int l = l0; l < l1; ++l) {
        const int4 w = __ldg(tile_win + l);  // (position j, row, col) of the window
        const int cc = mc - w.z;
        const bool cin = (unsigned)cc < (unsigned)N;
        const float2* yj = y + (size_t)w.x * NN;
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const int rr = mr0 + kTRG * k - w.y;
            if (cin && (unsigned)rr < (unsigned)N) {
                const int o = rr * N + cc;
                const float2 pv = __ldg(P + o);
                const float2 yv = __ldcs(yj + o);
                acc[k] = cadd(acc[k], cconjmul(pv, yv));
                den[k] += cabs2(pv);
            }
        }
    }
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int mr = mr0 + kTRG * k;
        if (mr < Mr && mc < Mc) {
            numO[(size_t)mr * Mc + mc] = acc[k];
            denO[(size_t)mr * Mc + mc] = den[k];
            mx = fmaxf(mx, den[k]);
        }
    }
    const float bm = block_max_float(mx, scratch);
    if (threadIdx.x == 0) atomicMax(maxO, __float_as_uint(bm));
}

// Atomic variant: one CTA row per (position, 256 probe pixels), scatter-add.
__global__ void __launch_bounds__(kT) scatter_object_kernel(
    const float2* __restrict__ y, const float2* __restrict__ P, const int2* __restrict__ pos,
    int N, int Mc, float2* __restrict__ numO, float* __restrict__ denO) {
    const int j = blockIdx.y;
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r >= N * N) return;
    const int rr = r / N, cc = r % N;
    const int2 s = pos[j];
    const float2 pv = __ldg(P + r);
    const float2 yv = __ldcs(y + (size_t)j * N * N + r);
    const size_t m = (size_t)(s.x + rr) * Mc + s.y + cc;
    atomicAdd(numO + m, cconjmul(pv, yv));
    atomicAdd(denO + m, cabs2(pv));
}

__global__ void __launch_bounds__(kT) max_float_kernel(const float* __restrict__ v, size_t n,
                                                       unsigned* __restrict__ out) {
    __shared__ float scratch[kT / 32];
    float m = 0.f;
    for (size_t i = blockIdx.x * (size_t)kT + threadIdx.x; i < n; i += (size_t)gridDim.x * kT)
        m = fmaxf(m, v[i]);
    const float bm = block_max_float(m, scratch);
    if (threadIdx.x == 0) atomicMax(out, __float_as_uint(bm));
}

__global__ void __launch_bounds__(kT) object_normalise_kernel(
    const float2* __restrict__ numO, const float* __restrict__ denO,
    const unsigned* __restrict__ maxO, size_t M, float alpha, float2* __restrict__ O,
    unsigned long long* __restrict__ maxP) {
    const size_t m = blockIdx.x * (size_t)kT + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *maxP = 0ull;  // the probe sweep comes next
    if (m >= M) return;
    const float mx = __uint_as_float(*maxO);
    const float d = denO[m] + alpha * mx;
    const float2 nv = numO[m];
    O[m] = d > 0.f ? make_float2(nv.x / d, nv.y / d) : make_float2(0.f, 0.f);
}

// Probe partial sums over a chunk of positions; thread = one probe pixel.
__global__ void __launch_bounds__(kT) probe_partial_kernel(
    const float2* __restrict__ y, const float2* __restrict__ O, const int2* __restrict__ pos,
    int J, int N, int Mc, int chunks, float2* __restrict__ partP, float* __restrict__ partPd) {
    const int r = blockIdx.x * kT + threadIdx.x;
    const int ch = blockIdx.y;
    if (r >= N * N) return;
    const int rr = r / N, cc = r % N;
    const int j0 = (int)(((long)ch * J) / chunks), j1 = (int)(((long)(ch + 1) * J) / chunks);
    const size_t NN = (size_t)N * N;
    float2 acc = make_float2(0.f, 0.f);
    float den = 0.f;
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const int2 s = pos[j];
        const float2 ov = __ldg(O + (size_t)(s.x + rr) * Mc + s.y + cc);
        const float2 yv = __ldcs(y + (size_t)j * NN + r);
        acc = cadd(acc, cconjmul(ov, yv));
        den += cabs2(ov);
    }
    partP[(size_t)ch * NN + r] = acc;
    partPd[(size_t)ch * NN + r] = den;
}

// FP64 totals of the probe partials: a block takes kT / RG probe pixels, its
// RG thread groups each add a contiguous range of chunks in order, and the
// group totals are added in group order (a fixed order: deterministic; RG = 1
// when there are few chunks, 8 when there are many).  The same blocks also
// add the per-CTA Fourier-error partials of the divide step in fixed slices,
// one FP64 slice total per block, so the final sum (in the normalise kernel)
// is over one value per block.
template <int RG>
__global__ void __launch_bounds__(kT) probe_reduce_kernel(
    const float2* __restrict__ partP, const float* __restrict__ partPd, int NN, int chunks,
    double2* __restrict__ numP, double* __restrict__ denP, unsigned long long* __restrict__ maxP,
    const double* __restrict__ e_part, int n_part, double* __restrict__ e_slice) {
    constexpr int RP = kT / RG;
    __shared__ double gx[RG][RP], gy[RG][RP], gd[RG][RP];
    __shared__ double scratch_s[kT / 32], scratch_m[kT / 32];
    const int px = threadIdx.x % RP, grp = threadIdx.x / RP;
    const int r = blockIdx.x * RP + px;
    const int c0 = (grp * chunks) / RG, c1 = ((grp + 1) * chunks) / RG;
    double nx = 0.0, ny = 0.0, d = 0.0;
    if (r < NN) {
        for (int ch = c0; ch < c1; ++ch) {
            const float2 p = partP[(size_t)ch * NN + r];
            nx += (double)p.x;
            ny += (double)p.y;
            d += (double)partPd[(size_t)ch * NN + r];
        }
    }
    double mx = 0.0;
    if constexpr (RG == 1) {
        if (r < NN) {
            numP[r] = make_double2(nx, ny);
            denP[r] = d;
            mx = d;
        }
    } else {
        gx[grp][px] = nx;
        gy[grp][px] = ny;
        gd[grp][px] = d;
        __syncthreads();
        if (grp == 0 && r < NN) {
            double tx = 0.0, ty = 0.0, td = 0.0;
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                tx += gx[g][px];
                ty += gy[g][px];
                td += gd[g][px];
            }
            numP[r] = make_double2(tx, ty);
            denP[r] = td;
            mx = td;
        }
    }
    const int per = (n_part + (int)gridDim.x - 1) / (int)gridDim.x;
    const int e0 = (int)blockIdx.x * per, e1 = min(n_part, e0 + per);
    double es = 0.0;
    for (int i = e0 + (int)threadIdx.x; i < e1; i += kT) es += e_part[i];
    const double slice = block_sum_double<kT>(es, scratch_s);
    if (threadIdx.x == 0) e_slice[blockIdx.x] = slice;
    const double bm = block_max_double(mx, scratch_m);
    if (threadIdx.x == 0) atomicMax(maxP, (unsigned long long)__double_as_longlong(bm));
}

constexpr int kManyChunks = 8;  // above this the chunks are added by 8 thread groups

// Probe update, plus (block 0) the iteration's Fourier error, stored in the
// ring at the slot of the device-side iteration counter (so a captured graph
// replays correctly), and the reset of the object maximum.
__global__ void __launch_bounds__(kT) probe_normalise_kernel(
    const double2* __restrict__ numP, const double* __restrict__ denP,
    const unsigned long long* __restrict__ maxP, int NN, double alpha, float2* __restrict__ P,
    const double* __restrict__ e_slice, int n_slice, double inv_sumI, double* __restrict__ e_ring,
    unsigned long long* __restrict__ d_iter, int ring_cap, unsigned* __restrict__ maxO) {
    __shared__ double scratch[kT / 32];
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r < NN) {
        const double mx = __longlong_as_double((long long)*maxP);
        const double d = denP[r] + alpha * mx;
        const double2 nv = numP[r];
        P[r] = d > 0.0 ? make_float2((float)(nv.x / d), (float)(nv.y / d)) : make_float2(0.f, 0.f);
    }
    if (blockIdx.x == 0) {
        double s = 0.0;
        for (int i = threadIdx.x; i < n_slice; i += kT) s += e_slice[i];
        const double tot = block_sum_double<kT>(s, scratch);
        if (threadIdx.x == 0) {
            const unsigned long long k = *d_iter;
            e_ring[k % (unsigned long long)ring_cap] = tot * inv_sumI;
            *d_iter = k + 1;
            *maxO = 0u;
        }
    }
}

__global__ void __launch_bounds__(kT) sum_parts_kernel(const double* __restrict__ parts, int n,
                                                       double scale, double* __restrict__ out) {
    __shared__ double scratch[kT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kT) s += parts[i];
    const double tot = block_sum_double<kT>(s, scratch);
    if (threadIdx.x == 0) *out = tot * scale;
}

__global__ void __launch_bounds__(kT) record_error_kernel(const double* __restrict__ parts, int n,
                                                          double scale, double* __restrict__ ring,
                                                          unsigned long long* __restrict__ d_iter,
                                                          int cap) {
    __shared__ double scratch[kT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kT) s += parts[i];
    const double tot = block_sum_double<kT>(s, scratch);
    if (threadIdx.x == 0) {
        const unsigned long long k = *d_iter;
        ring[k % (unsigned long long)cap] = tot * scale;
        *d_iter = k + 1;
    }
}

__global__ void __launch_bounds__(kT) form_waves_kernel(float2* __restrict__ x,
                                                        const float2* __restrict__ P,
                                                        const float2* __restrict__ O,
                                                        const int2* __restrict__ pos, int N,
                                                        int Mc) {
    const int j = blockIdx.y;
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r >= N * N) return;
    const int rr = r / N, cc = r % N;
    const int2 s = pos[j];
    x[(size_t)j * N * N + r] = cmul_rn(P[r], O[(size_t)(s.x + rr) * Mc + s.y + cc]);
}

// x_k from the lazily kept (x_{k-1}, y_{k-1}, P_k, O_k): the same expression,
// operand for operand, as the divide kernel's prologue.
__global__ void __launch_bounds__(kT) materialise_kernel(float2* __restrict__ x,
                                                         const float2* __restrict__ y,
                                                         const float2* __restrict__ P,
                                                         const float2* __restrict__ O,
                                                         const int2* __restrict__ pos, int N,
                                                         int Mc, float pa, float pb) {
    const int j = blockIdx.y;
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r >= N * N) return;
    const int rr = r / N, cc = r % N;
    const int2 s = pos[j];
    const size_t idx = (size_t)j * N * N + r;
    const float2 z = cmul_rn(P[r], O[(size_t)(s.x + rr) * Mc + s.y + cc]);
    const float2 yv = pb != 1.0f ? y[idx] : make_float2(0.f, 0.f);
    const float2 xp = pa != 1.0f ? x[idx] : make_float2(0.f, 0.f);
    x[idx] = resplit_rn(z, yv, xp, pa, pb);
}

}  // namespace

int probe_reduce_blocks(int N, int chunks) {
    const int rp = chunks > kManyChunks ? kT / 8 : kT;
    return (N * N + rp - 1) / rp;
}

int probe_chunks(int J, int N) {
    const int blocks = (N * N + kT - 1) / kT;
    int ch = (2048 + blocks - 1) / blocks;  // about 2048 CTAs in the partial pass
    if (ch > J) ch = J;
    if (ch < 1) ch = 1;
    return ch;
}

cudaError_t launch_concur(const float2* y, float2* P, float2* O, const int2* pos,
                          const ConcurBufs& cb, int J, int N, int Mr, int Mc, float alpha,
                          const double* e_part, int n_part, double inv_sumI, double* e_ring,
                          unsigned long long* d_iter, int ring_cap, int concur_mode,
                          cudaStream_t st) {
    const size_t M = (size_t)Mr * Mc;
    const int NN = N * N;
    if (concur_mode == 0) {
        concur_object_kernel<<<cb.tiles_r * cb.tiles_c, kT, 0, st>>>(
            y, P, cb.tile_win, cb.tile_ptr, N, Mr, Mc, cb.tiles_c, cb.numO, cb.denO, cb.maxO);
    } else {
        cudaMemsetAsync(cb.numO, 0, M * sizeof(float2), st);
        cudaMemsetAsync(cb.denO, 0, M * sizeof(float), st);
        scatter_object_kernel<<<dim3((NN + kT - 1) / kT, J), kT, 0, st>>>(y, P, pos, N, Mc,
                                                                         cb.numO, cb.denO);
        max_float_kernel<<<304, kT, 0, st>>>(cb.denO, M, cb.maxO);
    }
    object_normalise_kernel<<<(unsigned)((M + kT - 1) / kT), kT, 0, st>>>(cb.numO, cb.denO,
                                                                         cb.maxO, M, alpha, O,
                                                                         cb.maxP);
    probe_partial_kernel<<<dim3((NN + kT - 1) / kT, cb.chunks), kT, 0, st>>>(
        y, O, pos, J, N, Mc, cb.chunks, cb.partP, cb.partPd);
    const int n_slice = probe_reduce_blocks(N, cb.chunks);
    if (cb.chunks > kManyChunks)
        probe_reduce_kernel<8><<<n_slice, kT, 0, st>>>(cb.partP, cb.partPd, NN, cb.chunks, cb.numP,
                                                       cb.denP, cb.maxP, e_part, n_part, cb.e_slice);
    else
        probe_reduce_kernel<1><<<n_slice, kT, 0, st>>>(cb.partP, cb.partPd, NN, cb.chunks, cb.numP,
                                                       cb.denP, cb.maxP, e_part, n_part, cb.e_slice);
    probe_normalise_kernel<<<(NN + kT - 1) / kT, kT, 0, st>>>(cb.numP, cb.denP, cb.maxP, NN,
                                                             (double)alpha, P, cb.e_slice, n_slice,
                                                             inv_sumI, e_ring, d_iter, ring_cap,
                                                             cb.maxO);
    return cudaGetLastError();
}

cudaError_t launch_record_error(const double* parts, int n, double scale, double* ring,
                                unsigned long long* d_iter, int cap, cudaStream_t st) {
    record_error_kernel<<<1, kT, 0, st>>>(parts, n, scale, ring, d_iter, cap);
    return cudaGetLastError();
}

cudaError_t launch_form_waves(float2* x, const float2* P, const float2* O, const int2* pos,
                              int J, int N, int Mc, cudaStream_t st) {
    form_waves_kernel<<<dim3((N * N + kT - 1) / kT, J), kT, 0, st>>>(x, P, O, pos, N, Mc);
    return cudaGetLastError();
}

cudaError_t launch_materialise(float2* x, const float2* y, const float2* P, const float2* O,
                               const int2* pos, int J, int N, int Mc, float pa, float pb,
                               cudaStream_t st) {
    materialise_kernel<<<dim3((N * N + kT - 1) / kT, J), kT, 0, st>>>(x, y, P, O, pos, N, Mc,
                                                                      pa, pb);
    return cudaGetLastError();
}

cudaError_t launch_sum_parts(const double* parts, int n, double scale, double* out,
                             cudaStream_t st) {
    sum_parts_kernel<<<1, kT, 0, st>>>(parts, n, scale, out);
    return cudaGetLastError();
}

}  // namespace ptycho
