// Divide step P^c_D of the abc update (Introduction; Fig. 3(a)) for 256 x 256
// patterns as separate row and column passes through L2, without thread-block
// clusters (the two-pass variant; divide.cu holds the cluster variant).  The
// arithmetic is the same as the cluster kernel's:
//
//   x_k  = a' (b' P O_j + (1 - b') y_{k-1}) + (1 - a') x_{k-1}     (or x_k given)
//   Psi  = F x_k
//   y_k  = F^{-1}( c sqrt(I_j) Psi/|Psi| + (1 - c) Psi )
//   e_j  = sum_q (|Psi| - sqrt(I_j))^2
//
// Every 1-D DFT of length 256 = 16 x 16 is two in-register passes of a
// 16-point DFT with the twiddle W_256^{t k} between them:
//   X[k + 16 q] = sum_t W_16^{t q} W_256^{t k} sum_e W_16^{e k} x[t + 16 e].
//
// Work items, 16 per exit wave and phase, each one band of 16 rows or columns:
//   R  (rows 16 p .. 16 p + 15)    form x_k, row DFT, write the band to T
//   C  (columns 16 p .. 16 p + 15) column DFT, modulus projection with the c
//                                  relaxation and 1/N^2, error partial,
//                                  inverse column DFT, write back to T
//   R' (rows 16 p .. 16 p + 15)    inverse row DFT, write y_k
// T is the exit wave's own y buffer (y_{k-1} of a band is read by the R item
// that then overwrites it), so the intermediate needs no memory of its own;
// it stays in L2 between the phases.
//
// Scheduling: persistent CTAs take items from one ticket counter in a fixed
// order.  Step s of that order holds the R items of wave s, the C items of
// wave s - D and the R' items of wave s - 2 D (D = lag), so an item depends
// only on items with smaller tickets: C(w) on the 16 R(w), R'(w) on the 16
// C(w).  A ticket is taken only by a running CTA, so the earliest unfinished
// item always has its inputs and the schedule cannot deadlock.  Completion
// counts are published with a release fence and atomic add and read with an
// acquire load; intermediates are read with L2-only loads (ld.global.cg).
// Every wait is bounded in time (2 s on %globaltimer): on expiry the kernel
// sets an error flag and the CTA leaves; the host reports PTYCHO_ETIMEOUT.
//
// Modes: the divide step; the Fourier error only (R and C items, T in a ring
// of scratch slots, an R item waiting for the C items of the wave that used
// its slot before); one sequential-projections step (one wave; R items also
// take max|P|^2 and max|O_j|^2, R' items update O and P instead of storing y).
#include <cmath>

#include "common.cuh"
#include "debug.cuh"
#include "internal.h"

PTYCHO_DEBUG_UNIT(divide2p)

namespace ptycho {
namespace {

constexpr int kN = 256;
constexpr int kNN = kN * kN;
constexpr int kBand = 16;                    // rows or columns per work item
constexpr int kItemsPerPhase = kN / kBand;   // 16
constexpr int kItemsPerStep = 3 * kItemsPerPhase;
constexpr int kT = 256;                      // threads: (band row or column) x 16 lanes
constexpr int kSlot = 17;                    // padded stride of 16 elements in shared memory
constexpr int kLine = 16 * kSlot + 1;        // 273: one band row / column in shared memory
constexpr size_t kSmem = (size_t)kBand * kLine * sizeof(float2) + 256 * sizeof(float2) +
                         64 * sizeof(float);
constexpr unsigned long long kWaitNs = 2000000000ull;

enum : int { kModeDivide = 0, kModeErrOnly = 1, kModeSP = 2 };

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Thread 0: wait until *cnt >= target (bounded); false on expiry.
__device__ bool wait_count(const unsigned* cnt, unsigned target, int* err_flag) {
    if (ld_acquire(cnt) >= target) return true;
    const uint64_t t0 = now_ns();
    while (ld_acquire(cnt) < target) {
        __nanosleep(128);
        if (now_ns() - t0 > kWaitNs) {
            atomicOr(err_flag, 2);
            return false;
        }
    }
    return true;
}

struct Item {
    int type, p, w;  // phase (0 R, 1 C, 2 R'), band, wave; w < 0: nothing to do
};

__device__ __forceinline__ Item decode(unsigned ticket, int J, int lag) {
    const int s = (int)(ticket / kItemsPerStep), u = (int)(ticket % kItemsPerStep);
    Item it;
    it.type = u / kItemsPerPhase;
    it.p = u % kItemsPerPhase;
    it.w = s - it.type * lag;
    if (it.w >= J) it.w = -1;
    return it;
}

template <int MODE>
__global__ void __launch_bounds__(kT, 4) divide2p_kernel(const DivideArgs args) {
    constexpr bool ERR_ONLY = MODE == kModeErrOnly;
    constexpr bool SP = MODE == kModeSP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);  // [16][kLine]
    float2* tw = buf + kBand * kLine;                    // tw[t * 16 + k] = W_256^{t k}
    float* red = reinterpret_cast<float*>(tw + 256);     // [64]
    __shared__ unsigned s_ticket[2];  // by iteration parity: written before the barrier
    __shared__ int s_ok[2];           // that the previous parity's readers have passed

    const int tid = threadIdx.x;
    const int hi = tid >> 4, lo = tid & 15;  // band row/column (or k), lane within 16
    for (int i = tid; i < 256; i += kT) tw[i] = args.tw[i];

    const int J = SP ? 1 : args.J;
    const int lag = args.lag;
    const unsigned n_items = (unsigned)(kItemsPerStep * (J + 2 * lag));
    unsigned* ctl = args.ctl;
    unsigned* rdone = ctl + 4;
    unsigned* cdone = ctl + 4 + J;
    const bool load_x = args.load_x != 0, write_x = args.write_x != 0;
    const bool need_y = args.pb != 1.0f, need_xp = args.pa != 1.0f;
    const float inv_n2 = 1.0f / (float)kNN;
    const float cr = args.c, oc = 1.0f - args.c;

    // thread 0: the HBM inputs of an item into L2 ahead of its loads (the rows
    // of x and y of an R item, the sqrt(I) block of a C item)
    auto prefetch_item = [&](unsigned tk) {
        if (tk >= n_items || SP) return;
        const Item nx = decode(tk, J, lag);
        if (nx.w < 0) return;
        const size_t pat = (size_t)nx.w * kNN;
        if (nx.type == 0 && !ERR_ONLY) {
            const size_t off = pat + (size_t)nx.p * kBand * kN;
            constexpr unsigned bb = (unsigned)(kBand * kN * sizeof(float2));
            if (load_x || need_xp) prefetch_l2(args.x + off, bb);
            if (!load_x && need_y) prefetch_l2(args.y + off, bb);
        } else if (nx.type == 1) {
            prefetch_l2(args.sqrtIp + pat + (size_t)nx.p * 4096, 4096 * sizeof(float));
        }
    };

    // Completion is counted per warp (each warp's lane 0 adds 1 once the warp's
    // stores of the item are done), so an item needs no CTA barrier at its end:
    // a wave's phase is complete at kItemsPerPhase * warps counts.
    constexpr unsigned kDone = (unsigned)kItemsPerPhase * (kT / 32);
    unsigned ticket = 0;
    if (tid == 0) {
        ticket = atomicAdd(ctl, 1u);
        prefetch_item(ticket);
    }
    for (unsigned iter = 0;; ++iter) {
        // thread 0: the next item, and a wait for the items it depends on (all
        // of them have smaller tickets, and this CTA's own earlier items were
        // published by its warps as they finished)
        if (tid == 0) {
            const unsigned cur = ticket;
            bool ok = true;
            if (cur < n_items) {
                const Item nx = decode(cur, J, lag);
                if (nx.w >= 0 && !(ERR_ONLY && nx.type == 2)) {
                    if (nx.type == 1) ok = wait_count(rdone + nx.w, kDone, args.err_flag);
                    else if (nx.type == 2) ok = wait_count(cdone + nx.w, kDone, args.err_flag);
                    else if (ERR_ONLY && nx.w >= args.ring)  // the slot's previous wave is done with it
                        ok = wait_count(cdone + (nx.w - args.ring), kDone, args.err_flag);
                }
                // the ticket after it; its latency overlaps this item
                ticket = atomicAdd(ctl, 1u);
            }
            s_ticket[iter & 1] = cur;
            s_ok[iter & 1] = ok ? 1 : 0;
        }
        __syncthreads();  // every warp is done with the previous item's shared memory
        const unsigned cur = s_ticket[iter & 1];
        if (cur >= n_items || !s_ok[iter & 1]) break;
        if (tid == 0) prefetch_item(ticket);
        const Item it = decode(cur, J, lag);
        if (it.w < 0 || (ERR_ONLY && it.type == 2)) continue;
        const int w = it.w, p = it.p;
        const int j = SP ? args.sp_pos : w;
        const size_t pat = (size_t)j * kNN;
        // the intermediate: y_j itself, or a scratch slot
        float2* T = (MODE == kModeDivide) ? args.y + pat
                                          : args.scratch + (size_t)(SP ? 0 : w % args.ring) * kNN;

        if (it.type == 0) {
            // ---- R: form x_k for rows 16 p .. 16 p + 15, two adjacent elements per
            // lane, into slot (n / 16) * 17 + n % 16 of the band row
            int2 s = args.pos[j];
#if PT_DBG_ENABLED
            // checked build: a window outside the object is recorded and clamped
            if (s.x < 0 || s.y < 0 || s.x > args.Mr - kN || s.y > args.Mc - kN) {
                if (tid == 0) PT_DBG_FLAG(kDbgWindow);
                s = make_int2(0, 0);
            }
#endif
            const float2* Ow = args.O + (size_t)s.x * args.Mc + s.y;
            float mp = 0.f, mo = 0.f;
#pragma unroll 4
            for (int i = tid; i < kBand * kN / 2; i += kT) {
                const int row = i >> 7, n = (i & 127) * 2;
                const int r = p * kBand + row;
                const size_t idx = pat + (size_t)r * kN + n;
                float2 x0, x1;
                if (load_x) {
                    const float4 f = __ldcs(reinterpret_cast<const float4*>(args.x + idx));
                    x0 = make_float2(f.x, f.y);
                    x1 = make_float2(f.z, f.w);
                } else {
                    const float4 pv = __ldg(reinterpret_cast<const float4*>(args.P + r * kN + n));
                    const float2* op = Ow + (size_t)r * args.Mc + n;
                    const float2 o0 = __ldg(op), o1 = __ldg(op + 1);
                    const float4 yv = need_y ? __ldcs(reinterpret_cast<const float4*>(args.y + idx))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 xp = need_xp ? __ldcs(reinterpret_cast<const float4*>(args.x + idx))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                    x0 = resplit_rn(cmul_rn(make_float2(pv.x, pv.y), o0), make_float2(yv.x, yv.y),
                                    make_float2(xp.x, xp.y), args.pa, args.pb);
                    x1 = resplit_rn(cmul_rn(make_float2(pv.z, pv.w), o1), make_float2(yv.z, yv.w),
                                    make_float2(xp.z, xp.w), args.pa, args.pb);
                    if (write_x)
                        __stcs(reinterpret_cast<float4*>(args.x + idx), make_float4(x0.x, x0.y, x1.x, x1.y));
                    if constexpr (SP) {
                        mp = fmaxf(mp, fmaxf(cabs2(make_float2(pv.x, pv.y)), cabs2(make_float2(pv.z, pv.w))));
                        mo = fmaxf(mo, fmaxf(cabs2(o0), cabs2(o1)));
                    }
                }
                float2* rb = buf + row * kLine + (n >> 4) * kSlot + (n & 15);
                rb[0] = x0;
                rb[1] = x1;
            }
            if constexpr (SP) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, o));
                    mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, o));
                }
                if ((tid & 31) == 0) {
                    atomicMax(ctl + 1, __float_as_uint(mp));
                    atomicMax(ctl + 2, __float_as_uint(mo));
                }
            }
            __syncthreads();
            {   // pass 1 (lanes over t = lo): DFT over e, twiddle W^{t k}
                float2* q = buf + hi * kLine + lo;
                float2 v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = q[e * kSlot];
                dft_reg<16, false>(v);
#pragma unroll
                for (int k = 0; k < 16; ++k) q[k * kSlot] = cmul(v[k], tw[lo * 16 + k]);
            }
            __syncthreads();
            {   // pass 2 (lanes over k = lo): DFT over t; column frequency k + 16 q
                const float2* q = buf + hi * kLine + lo * kSlot;
                float2 u[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) u[t] = q[t];
                dft_reg<16, false>(u);
                float2* dst = T + (size_t)(p * kBand + hi) * kN + lo;
#pragma unroll
                for (int qq = 0; qq < 16; ++qq) __stcg(dst + 16 * qq, u[qq]);
            }
        } else if (it.type == 1) {
            // ---- C: columns 16 p + c, c = 0..15; element (c, k, t) at c * 273 + k * 17 + t
            {   // pass 1 (thread (t = hi, c = lo)): rows t + 16 e, DFT over e, twiddle
                const float2* src = T + (size_t)hi * kN + p * kBand + lo;
                float2 v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] = __ldcg(src + (size_t)e * 16 * kN);
                dft_reg<16, false>(v);
                float2* q = buf + lo * kLine + hi;
#pragma unroll
                for (int k = 0; k < 16; ++k) q[k * kSlot] = cmul(v[k], tw[hi * 16 + k]);
            }
            __syncthreads();
            float err = 0.f;
            {   // pass 2 (thread (k = hi, c = lo)): DFT over t -> row frequency k + 16 q,
                // modulus projection, inverse DFT over q, conjugate twiddle
                float2* q = buf + lo * kLine + hi * kSlot;
                float2 u[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) u[t] = q[t];
                dft_reg<16, false>(u);
                const float* sp = args.sqrtIp + pat + (size_t)p * 4096 + (size_t)(hi * 16 + lo) * 16;
                float sv[16];
#pragma unroll
                for (int qq = 0; qq < 16; qq += 4) {
                    const float4 f = __ldcs(reinterpret_cast<const float4*>(sp + qq));
                    sv[qq] = f.x; sv[qq + 1] = f.y; sv[qq + 2] = f.z; sv[qq + 3] = f.w;
                }
#pragma unroll
                for (int qq = 0; qq < 16; ++qq) {
#if PT_DBG_ENABLED
                    if (!(sv[qq] >= 0.f) || !isfinite(sv[qq])) PT_DBG_FLAG(kDbgSqrtI);
#endif
                    // |Psi| and Psi/|Psi| from one reciprocal square root
                    const float m2 = cabs2(u[qq]);
                    const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
                    const float d = fmaf(m2, rs, -sv[qq]);
                    err = fmaf(d, d, err);
                    if constexpr (!ERR_ONLY) {
                        // c sqrt(I) Psi/|Psi| + (1 - c) Psi, scaled by 1/N^2; sqrt(I) + 0i where Psi = 0
                        const float g = (cr * sv[qq]) * rs + oc;
                        u[qq] = m2 > 0.f ? make_float2(u[qq].x * (g * inv_n2), u[qq].y * (g * inv_n2))
                                         : make_float2(cr * sv[qq] * inv_n2, 0.f);
                    }
                }
                if constexpr (!ERR_ONLY) {
                    dft_reg<16, true>(u);
#pragma unroll
                    for (int t = 0; t < 16; ++t) q[t] = cconjmul(tw[t * 16 + hi], u[t]);
                }
            }
            // this item's error partial (FP32 within the item; FP64 across items
            // in the concur step's reduction)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) err += __shfl_down_sync(0xffffffffu, err, o);
            if ((tid & 31) == 0) red[tid >> 5] = err;
            __syncthreads();
            if (tid == 0) {
                float tot = 0.f;
#pragma unroll
                for (int i = 0; i < kT / 32; ++i) tot += red[i];
                args.e_part[(size_t)j * kItemsPerPhase + p] = (double)tot;
            }
            if constexpr (!ERR_ONLY) {
                // inverse pass 1 (thread (t = hi, c = lo)): DFT over k -> rows t + 16 e
                const float2* q = buf + lo * kLine + hi;
                float2 v[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = q[k * kSlot];
                dft_reg<16, true>(v);
                float2* dst = T + (size_t)hi * kN + p * kBand + lo;
#pragma unroll
                for (int e = 0; e < 16; ++e) __stcg(dst + (size_t)e * 16 * kN, v[e]);
            }
        } else {
            // ---- R': rows 16 p + row; pass A (thread (row = hi, k = lo)): inverse DFT
            // over q of column frequencies k + 16 q, conjugate twiddle
            {
                const float2* src = T + (size_t)(p * kBand + hi) * kN + lo;
                float2 u[16];
#pragma unroll
                for (int qq = 0; qq < 16; ++qq) u[qq] = __ldcg(src + 16 * qq);
                dft_reg<16, true>(u);
                float2* q = buf + hi * kLine + lo * kSlot;
#pragma unroll
                for (int t = 0; t < 16; ++t) q[t] = cconjmul(tw[t * 16 + lo], u[t]);
            }
            __syncthreads();
            {   // pass B (thread (row = hi, t = lo)): inverse DFT over k -> n = t + 16 e
                const float2* q = buf + hi * kLine + lo;
                float2 v[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = q[k * kSlot];
                dft_reg<16, true>(v);
                const int r = p * kBand + hi;
                if constexpr (SP) {
                    // d = psi' - psi; O_j += conj(P) d / max|P|^2, P += conj(O_j) d / max|O_j|^2
                    const float mp = __uint_as_float(ld_acquire(ctl + 1));
                    const float mo = __uint_as_float(ld_acquire(ctl + 2));
                    const float inv_maxP = mp > 0.f ? 1.0f / mp : 0.f;
                    const float inv_maxO = mo > 0.f ? 1.0f / mo : 0.f;
                    int2 s = args.pos[j];
#if PT_DBG_ENABLED
                    if (s.x < 0 || s.y < 0 || s.x > args.Mr - kN || s.y > args.Mc - kN) s = make_int2(0, 0);
#endif
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int n = lo + 16 * e;
                        const float2 pv = args.P[r * kN + n];
                        float2* op = args.O_mut + (size_t)(s.x + r) * args.Mc + s.y + n;
                        const float2 ov = *op;
                        const float2 d = csub(v[e], cmul_rn(pv, ov));
                        *op = cadd(ov, cscale(cconjmul(pv, d), inv_maxP));
                        args.P_mut[r * kN + n] = cadd(pv, cscale(cconjmul(ov, d), inv_maxO));
                    }
                } else {
                    float2* yo = args.y + pat + (size_t)r * kN + lo;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
#if PT_DBG_ENABLED
                        if (PT_DBG_NONFINITE2(v[e])) PT_DBG_FLAG(kDbgNonFinite);
#endif
                        __stcs(yo + 16 * e, v[e]);
                    }
                }
            }
        }
        // publish this warp's part of an R or C item
        if (it.type < 2) {
            __syncwarp();
            if ((tid & 31) == 0) {
                __threadfence();
                atomicAdd((it.type == 0 ? rdone : cdone) + w, 1u);
            }
        }
    }
}

// sqrt(I) into the order the C items read it: entry p * 4096 + (k * 16 + c) * 16 + q
// holds sqrt(I) at row frequency u = k + 16 q, column frequency v = 16 p + c.
// Flags *bad for a negative or non-finite value; FP64 sums of I over blocks
// of the natural order (the same sums as the cluster design's).
__global__ void __launch_bounds__(256) sqrt_permute2p_kernel(const float* __restrict__ I,
                                                             float* __restrict__ sqrtIp,
                                                             double* __restrict__ psum,
                                                             int* __restrict__ bad) {
    __shared__ double red[8];
    const int j = blockIdx.y;
    const int pidx = blockIdx.x * 256 + threadIdx.x;
    double v64 = 0.0;
    if (pidx < kNN) {
        const int q = pidx & 15, c = (pidx >> 4) & 15, k = (pidx >> 8) & 15, p = pidx >> 12;
        const int u = k + 16 * q, v = 16 * p + c;
        const float val = I[(size_t)j * kNN + (size_t)u * kN + v];
        if (!(val >= 0.0f) || !isfinite(val)) atomicOr(bad, 1);
        sqrtIp[(size_t)j * kNN + pidx] = sqrtf(fmaxf(val, 0.0f));
        v64 = (double)I[(size_t)j * kNN + pidx];  // natural-order block sums
    }
    const double tot = block_sum_double<256>(v64, red);
    if (threadIdx.x == 0) psum[(size_t)j * gridDim.x + blockIdx.x] = tot;
}

int g_grid = 0;

}  // namespace

bool divide2p_supported(int N) { return N == kN; }
int divide2p_lag() { return 16; }
int divide2p_ring() { return 48; }
size_t divide2p_ctl_words(int J) { return 4 + 2 * (size_t)(J > 1 ? J : 1); }

cudaError_t divide2p_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(divide2p_kernel<kModeDivide>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(divide2p_kernel<kModeErrOnly>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(divide2p_kernel<kModeSP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) != cudaSuccess)
        return e;
    if (g_grid == 0) {
        int dev = 0, sms = 0, per = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, divide2p_kernel<kModeDivide>, kT,
                                                               kSmem)) != cudaSuccess)
            return e;
        g_grid = sms * (per > 0 ? per : 1);
    }
    return cudaSuccess;
}

cudaError_t launch_divide2p(const DivideArgs& a, cudaStream_t st) {
    const int J = a.sp ? 1 : a.J;
    cudaError_t e = cudaMemsetAsync(a.ctl, 0, divide2p_ctl_words(J) * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const long items = (long)kItemsPerStep * (J + 2 * a.lag);
    const int grid = (int)(items < g_grid ? items : g_grid);
    if (a.sp) divide2p_kernel<kModeSP><<<grid, kT, kSmem, st>>>(a);
    else if (a.err_only) divide2p_kernel<kModeErrOnly><<<grid, kT, kSmem, st>>>(a);
    else divide2p_kernel<kModeDivide><<<grid, kT, kSmem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sqrt_permute2p(const float* I, float* sqrtIp, double* psum, int* bad, int J,
                                  cudaStream_t st) {
    dim3 grid(kNN / 256, J);
    sqrt_permute2p_kernel<<<grid, 256, 0, st>>>(I, sqrtIp, psum, bad);
    return cudaGetLastError();
}

}  // namespace ptycho
