// Probe update of the concur step for callers that cannot allocate device
// memory: ptycho_probe_update_noalloc (declared in include/ptycho.h).
//
// Some callers own every byte of device memory through their own allocator
// or run inside a pipeline that must not allocate after start-up (a
// cudaMalloc there can fail, fragment a pool sized in advance, or stall the
// device while it synchronises).  This entry point takes device pointers for
// all inputs and the output, and keeps its scratch (the per-chunk partial
// sums of the probe numerator and denominator, their FP64 totals, the running
// maximum and a status word) in one file-scope __device__ array below.  It
// never calls cudaMalloc, cudaFree or any allocating library routine.
//
// The arithmetic is the probe half of the concur step of the general abc
// update, the same as the context-based path computes:
//   P(r) = sum_j conj(O(s_j + r)) y_j(r) / (sum_j |O(s_j + r)|^2 + alpha max_r(.)),
// FP32 partial sums over the same fixed chunks of positions, FP64 final sums.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/ptycho.h"
#include "common.cuh"
#include "internal.h"

namespace {

// Capacity: probe side N <= 256.  The partial sums hold chunks * N^2 values,
// where probe_chunks gives chunks <= ceil(2048 / blocks) with blocks =
// ceil(N^2 / 256); so chunks * N^2 <= chunks * blocks * 256 <= (2048 + blocks - 1)
// * 256 <= (2048 + 255) * 256 for every N <= 256 (N = 256 itself needs 8 * 256^2).
constexpr int kMaxN = 256;
constexpr size_t kMaxPix = (size_t)kMaxN * kMaxN;
constexpr size_t kMaxBlocks = (kMaxPix + 255) / 256;
constexpr size_t kMaxPartial = (2048 + kMaxBlocks - 1) * 256;
static_assert(kMaxPartial >= 8 * kMaxPix, "N = 256 with 8 chunks fits");

// Byte layout of the scratch array.
constexpr size_t kOffPart = 0;                                   // float2 [kMaxPartial]
constexpr size_t kOffPartD = kOffPart + kMaxPartial * 8;         // float  [kMaxPartial]
constexpr size_t kOffNum = kOffPartD + kMaxPartial * 4;          // double2 [kMaxPix]
constexpr size_t kOffDen = kOffNum + kMaxPix * 16;               // double [kMaxPix]
constexpr size_t kOffMax = kOffDen + kMaxPix * 8;                // u64 max bits
constexpr size_t kOffStatus = kOffMax + 8;                       // int status
constexpr size_t kScratchBytes = kOffStatus + 248;               // 8.25 MiB + 256 B
static_assert(kOffNum % 16 == 0 && kOffDen % 8 == 0 && kOffMax % 8 == 0, "scratch alignment");

// The scratch itself: one copy on every device that loads the library, held
// until the process exits.  Host code may not use this name as an address
// (it is a host-side stand-in); the device address comes from
// cudaGetSymbolAddress, looked up once per device below.
static __device__ __align__(256) unsigned char g_probe_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {};

constexpr int kT = 256;

__global__ void __launch_bounds__(kT) na_partial_kernel(
    const float2* __restrict__ y, const float2* __restrict__ O, const int2* __restrict__ pos,
    int J, int N, int Mr, int Mc, int chunks, unsigned char* __restrict__ scratch) {
    float2* partP = reinterpret_cast<float2*>(scratch + kOffPart);
    float* partPd = reinterpret_cast<float*>(scratch + kOffPartD);
    int* status = reinterpret_cast<int*>(scratch + kOffStatus);
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
        // bounds check: a window outside the object is skipped and reported
        if (s.x < 0 || s.y < 0 || s.x > Mr - N || s.y > Mc - N) {
            atomicOr(status, 1);
            continue;
        }
        const float2 ov = __ldg(O + (size_t)(s.x + rr) * Mc + s.y + cc);
        const float2 yv = __ldcs(y + (size_t)j * NN + r);
        acc = ptycho::cadd(acc, ptycho::cconjmul(ov, yv));
        den += ptycho::cabs2(ov);
    }
    partP[(size_t)ch * NN + r] = acc;
    partPd[(size_t)ch * NN + r] = den;
}

__global__ void __launch_bounds__(kT) na_reduce_kernel(int NN, int chunks,
                                                       unsigned char* __restrict__ scratch) {
    __shared__ double sm[kT / 32];
    const float2* partP = reinterpret_cast<const float2*>(scratch + kOffPart);
    const float* partPd = reinterpret_cast<const float*>(scratch + kOffPartD);
    double2* numP = reinterpret_cast<double2*>(scratch + kOffNum);
    double* denP = reinterpret_cast<double*>(scratch + kOffDen);
    unsigned long long* maxP = reinterpret_cast<unsigned long long*>(scratch + kOffMax);
    const int r = blockIdx.x * kT + threadIdx.x;
    double mx = 0.0;
    if (r < NN) {
        double nx = 0.0, ny = 0.0, d = 0.0;
        for (int ch = 0; ch < chunks; ++ch) {
            const float2 p = partP[(size_t)ch * NN + r];
            nx += (double)p.x;
            ny += (double)p.y;
            d += (double)partPd[(size_t)ch * NN + r];
        }
        numP[r] = make_double2(nx, ny);
        denP[r] = d;
        mx = d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < kT / 32; ++i) m = fmax(m, sm[i]);
        atomicMax(maxP, (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void __launch_bounds__(kT) na_normalise_kernel(int NN, double alpha,
                                                          const unsigned char* __restrict__ scratch,
                                                          float2* __restrict__ P) {
    const double2* numP = reinterpret_cast<const double2*>(scratch + kOffNum);
    const double* denP = reinterpret_cast<const double*>(scratch + kOffDen);
    const unsigned long long* maxP = reinterpret_cast<const unsigned long long*>(scratch + kOffMax);
    const int* status = reinterpret_cast<const int*>(scratch + kOffStatus);
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r >= NN || *status != 0) return;   // on a bad position the output is left untouched
    const double mx = __longlong_as_double((long long)*maxP);
    const double d = denP[r] + alpha * mx;
    const double2 nv = numP[r];
    P[r] = d > 0.0 ? make_float2((float)(nv.x / d), (float)(nv.y / d)) : make_float2(0.f, 0.f);
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_on_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_probe_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int ptycho_probe_update_noalloc(const float* y, const float* obj, const int32_t* pos_rc,
                                           int32_t J, int32_t N, int32_t M_rows, int32_t M_cols,
                                           float alpha, float* probe_out, void* stream) {
    if (!y || !obj || !pos_rc || !probe_out) return PTYCHO_EINVAL;
    if (J < 1 || N < 1 || N > kMaxN || M_rows < N || M_cols < N) return PTYCHO_EINVAL;
    if (!(alpha >= 0.0f) || !std::isfinite(alpha)) return PTYCHO_EINVAL;
    const int chunks = ptycho::probe_chunks(J, N);
    const size_t NN = (size_t)N * N;
    if ((size_t)chunks * NN > kMaxPartial) return PTYCHO_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return PTYCHO_ECUDA;
    // the array keeps the previous call's contents: zero the maximum and the status
    if (cudaMemsetAsync(scratch + kOffMax, 0, 16, st) != cudaSuccess) return PTYCHO_ECUDA;
    const unsigned blocks = (unsigned)((NN + kT - 1) / kT);
    // each launch reports its own status (an error left on this thread by
    // earlier, unrelated work is neither returned nor cleared here)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, (unsigned)chunks);
    cfg.blockDim = dim3(kT);
    cfg.stream = st;
    if (cudaLaunchKernelEx(&cfg, na_partial_kernel, reinterpret_cast<const float2*>(y),
                           reinterpret_cast<const float2*>(obj),
                           reinterpret_cast<const int2*>(pos_rc), (int)J, (int)N, (int)M_rows,
                           (int)M_cols, chunks, scratch) != cudaSuccess)
        return PTYCHO_ECUDA;
    cfg.gridDim = dim3(blocks);
    if (cudaLaunchKernelEx(&cfg, na_reduce_kernel, (int)NN, chunks, scratch) != cudaSuccess)
        return PTYCHO_ECUDA;
    if (cudaLaunchKernelEx(&cfg, na_normalise_kernel, (int)NN, (double)alpha,
                           (const unsigned char*)scratch,
                           reinterpret_cast<float2*>(probe_out)) != cudaSuccess)
        return PTYCHO_ECUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, scratch + kOffStatus, sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PTYCHO_ECUDA;
    return status ? PTYCHO_EINVAL : PTYCHO_OK;
}
