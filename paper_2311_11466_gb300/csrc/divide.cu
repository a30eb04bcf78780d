// Divide step P^c_D of the abc update (Introduction; Fig. 3(a)), fused with
// the relaxed re-split of the previous iteration's concur step:
//
//   x_k  = a' (b' P O_j + (1 - b') y_{k-1}) + (1 - a') x_{k-1}     (or x_k given)
//   Psi  = F x_k
//   y_k  = F^{-1}( c sqrt(I_j) Psi/|Psi| + (1 - c) Psi )
//   e_j  = sum_q (|Psi| - sqrt(I_j))^2
//
// One thread-block cluster of C CTAs works on one N x N exit wave at a time;
// CTA c holds R = N / C rows in shared memory (FP32 complex).  Every 1-D DFT
// of length N = A * B runs as two in-register passes: pass 1 takes the A
// elements t + B e (e < A) of one thread, a DFT of length A and the twiddle
// W_N^{t k}; pass 2 takes the B elements of one k, a DFT of length B.  The
// spectrum is left in that digit-permuted order (sqrt(I) is stored in the
// same order at load time).
//
// The two transposes of the 2-D DFT (row pass -> column pass and back) go
// through global memory: the row pass's second half stores its outputs in the
// column-major order the other CTAs need, one cluster barrier (release /
// acquire, cluster scope) later the column pass reads them straight into
// registers (L2-cached loads), then drops the lines from L2 without a write
// back; the inverse goes back the same way through the exit wave's own y
// buffer.  Two cluster barriers per exit wave; one cluster per exit wave, so
// clusters start as others finish and their memory and compute phases
// interleave on each SM.
//
// Shared-memory row layout: element t + B e of a row lives at slot e (B + 1) + t
// so both passes are bank-conflict free; the row stride RS keeps the passes
// whose lanes run over rows conflict free as well.
#include <cooperative_groups.h>

#include <cmath>

#include "common.cuh"
#include "debug.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

PTYCHO_DEBUG_UNIT(divide)

namespace ptycho {
namespace {

// A x B radix split, cluster size C, threads T, row stride residue RSM (mod
// 16), and the CTAs per SM the register budget is sized for (MINB).  V selects
// a launch variant with the same radix split (the same arithmetic): at 128^2
// the autotuner times clusters of 8 CTAs of 128 threads (V = 0) against 16 of
// 64 (V = 1).
template <int N, int V = 0> struct Cfg;
template <> struct Cfg<8, 0>   { static constexpr int A = 4,  B = 2,  C = 1, T = 32,  RSM = 9, MINB = 4; };
template <> struct Cfg<16, 0>  { static constexpr int A = 4,  B = 4,  C = 1, T = 64,  RSM = 9, MINB = 4; };
template <> struct Cfg<32, 0>  { static constexpr int A = 8,  B = 4,  C = 1, T = 128, RSM = 9, MINB = 4; };
template <> struct Cfg<64, 0>  { static constexpr int A = 8,  B = 8,  C = 2, T = 256, RSM = 9, MINB = 4; };
template <> struct Cfg<128, 0> { static constexpr int A = 16, B = 8,  C = 8, T = 128, RSM = 9, MINB = 8; };
template <> struct Cfg<128, 1> { static constexpr int A = 16, B = 8,  C = 16, T = 64, RSM = 9, MINB = 16; };
template <> struct Cfg<256, 0> { static constexpr int A = 16, B = 16, C = 16, T = 256, RSM = 1, MINB = 4; };

template <int N, int V = 0>
struct Geo {
    static constexpr int A = Cfg<N, V>::A, B = Cfg<N, V>::B, C = Cfg<N, V>::C, T = Cfg<N, V>::T;
    static constexpr int R = N / C;       // rows per CTA
    static constexpr int KC = A / C;      // pass-2 indices k per CTA
    static constexpr int RS0 = A * (B + 1);
    static constexpr int RS = RS0 + ((Cfg<N, V>::RSM - RS0 % 16) + 16) % 16;  // row stride
    static constexpr int TP2 = (R * A + T - 1) / T;  // pass-2 tasks per thread
    static constexpr size_t SMEM = (size_t)R * RS * sizeof(float2) + 2 * N * sizeof(float2) +
                                   32 * sizeof(double);
    static_assert(A * B == N, "radix split");
    static_assert(A % C == 0, "cluster split");
};

// True when passes 1 and 2 of a row DFT run on the same 16 lanes (A == B == 16
// and one task per thread), so the hand-over between them is warp-local.
template <int N, int V>
constexpr bool kRowPerHalfWarp = Geo<N, V>::A == 16 && Geo<N, V>::B == 16 && Geo<N, V>::R * 16 == Geo<N, V>::T;

// Scratch lines are dropped from L2 once read when a row of the scratch is a
// whole number of 128-byte lines and the lanes sharing a line sit in one warp.
template <int N, int V>
constexpr bool kDiscard = (N % 16 == 0) && (Geo<N, V>::T % 32 == 0) && (32 % Geo<N, V>::B == 0);

// One bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16); it does not wait and brings nothing into the SM.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Drop a 128-byte line from L2 without writing it back (its contents become
// undefined); used on scratch lines once every reader has its data.
__device__ __forceinline__ void discard_l2(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Kernel modes: the divide step; the Fourier error only; one step of
// sequential projections (update O and P from one exit wave).
enum : int { kModeDivide = 0, kModeErrOnly = 1, kModeSP = 2 };

// The work of one CTA of the cluster that handles exit wave j.
template <int N, int MODE, int V>
__device__ __forceinline__ void divide_body(const DivideArgs args, const int j) {
    constexpr bool ERR_ONLY = MODE == kModeErrOnly;
    constexpr bool SP = MODE == kModeSP;
    using G = Geo<N, V>;
    constexpr int A = G::A, B = G::B, C = G::C, T = G::T, R = G::R, RS = G::RS;
    constexpr int TP2 = G::TP2;
    constexpr size_t NN = (size_t)N * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    float2* twA = buf + R * RS;   // twA[k B + t] = W_N^{t k}
    float2* twB = twA + N;        // twB[t A + k] = W_N^{t k}
    float* redf = reinterpret_cast<float*>(twB + N);

    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int tid = threadIdx.x;

    for (int i = tid; i < N; i += T) {
        const float2 w = args.tw[i];
        twA[i] = w;
        twB[(i % B) * A + i / B] = w;
    }

    const bool load_x = args.load_x != 0, write_x = args.write_x != 0;
    const bool need_y = args.pb != 1.0f, need_xp = args.pa != 1.0f;

    const size_t pat = (size_t)j * NN;
    // transpose scratch: S[v'][r] (row pass -> column pass) in this wave's
    // scratch buffer; S2[r][v'] (back) in its y buffer, which holds nothing
    // live between the re-split's read of y_{k-1} (before the first cluster
    // barrier) and the store of y_k (after the second)
    float2* S = SP ? args.scratch : args.scratch + pat;
    float2* S2 = SP ? args.scratch + NN : args.y + pat;  // SP leaves y untouched
    if (tid == 0) {
        // stream this CTA's rows of x, y and sqrt(I) into L2 at once
        const size_t off = pat + (size_t)c * R * N;
        constexpr unsigned cbytes = (unsigned)(R * N * sizeof(float2));
        if (load_x || need_xp) prefetch_l2(args.x + off, cbytes);
        if (!load_x && need_y) prefetch_l2(args.y + off, cbytes);
        prefetch_l2(args.sqrtIp + off, (unsigned)(R * N * sizeof(float)));
    }
    __syncthreads();  // twiddles loaded
    int2 s = args.pos[j];
#if PT_DBG_ENABLED
    // checked build: a window outside the object is recorded and clamped to the
    // corner (every CTA of the cluster still reaches its barriers)
    if (s.x < 0 || s.y < 0 || s.x > args.Mr - N || s.y > args.Mc - N) {
        if (tid == 0) PT_DBG_FLAG(kDbgWindow);
        s = make_int2(0, 0);
    }
#endif
    const float2* Ow = args.O + (size_t)s.x * args.Mc + s.y;

    // Sequential projections, phase 0: max |P|^2 over the probe and max |O_j|^2
    // over the window, each CTA over its rows, then across the cluster.
    float inv_maxP = 0.f, inv_maxO = 0.f;
    if constexpr (SP) {
        float mp = 0.f, mo = 0.f;
        for (int e = tid; e < R * N; e += T) {
            const int r = c * R + e / N, n = e % N;
            mp = fmaxf(mp, cabs2(args.P[r * N + n]));
            mo = fmaxf(mo, cabs2(Ow[(size_t)r * args.Mc + n]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, o));
            mo = fmaxf(mo, __shfl_xor_sync(0xffffffffu, mo, o));
        }
        if ((tid & 31) == 0) {
            redf[2 * (tid >> 5)] = mp;
            redf[2 * (tid >> 5) + 1] = mo;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < T / 32; ++w) {
                mp = fmaxf(mp, redf[2 * w]);
                mo = fmaxf(mo, redf[2 * w + 1]);
            }
            redf[62] = mp;  // this CTA's maxima, read by the whole cluster
            redf[63] = mo;
        }
        cl.sync();
        mp = 0.f;
        mo = 0.f;
        for (int q = 0; q < C; ++q) {
            const float* rq = cl.map_shared_rank(redf, q);
            mp = fmaxf(mp, rq[62]);
            mo = fmaxf(mo, rq[63]);
        }
        inv_maxP = mp > 0.f ? 1.0f / mp : 0.f;
        inv_maxO = mo > 0.f ? 1.0f / mo : 0.f;
    }

    // Phase 1a: form x_k for this CTA's rows, two adjacent elements per lane
    // (16-byte loads, coalesced; few registers live, so many loads in flight),
    // into the row buffer at the slot of element n = t + B e.
    static_assert(N % 2 == 0 && B % 2 == 0, "element pairs");
#pragma unroll 4
    for (int i = tid; i < R * N / 2; i += T) {
        const int row = i / (N / 2), n = 2 * (i % (N / 2));
        const int r = c * R + row;
        const size_t idx = pat + (size_t)r * N + n;
        float2 x0, x1;
        if (load_x) {
            const float4 f = __ldcs(reinterpret_cast<const float4*>(args.x + idx));
            x0 = make_float2(f.x, f.y);
            x1 = make_float2(f.z, f.w);
        } else {
            const float4 pv = __ldg(reinterpret_cast<const float4*>(args.P + r * N + n));
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
            if (write_x) __stcs(reinterpret_cast<float4*>(args.x + idx), make_float4(x0.x, x0.y, x1.x, x1.y));
        }
        float2* rb = buf + row * RS;
        rb[(n / B) * (B + 1) + n % B] = x0;          // n even, B even: n + 1 is
        rb[(n / B) * (B + 1) + n % B + 1] = x1;      // in the same group of B
    }
    __syncthreads();

    // Phase 1b: row DFT pass 1 in place (lanes over t): each thread reads the
    // A slots of its (row, t) and writes its outputs back to the same slots.
#pragma unroll 1
    for (int task = tid; task < R * B; task += T) {
        const int row = task / B, t = task % B;
        float2* p = buf + row * RS + t;
        float2 v[A];
#pragma unroll
        for (int e = 0; e < A; ++e) v[e] = p[e * (B + 1)];
        dft_reg<A, false>(v);
#pragma unroll
        for (int k = 0; k < A; ++k) p[k * (B + 1)] = cmul(v[k], twA[k * B + t]);
    }
    __syncthreads();

    // Phase 2: row DFT pass 2 (lanes over rows); column frequency v' = k B + q
    // of spatial row r goes to S[v'][r].
#pragma unroll
    for (int i = 0; i < TP2; ++i) {
        const int task = tid + i * T;
        if (task < R * A) {
            const int k = task / R, row = task % R;
            const float2* p = buf + row * RS + k * (B + 1);
            float2 u[B];
#pragma unroll
            for (int t = 0; t < B; ++t) u[t] = p[t];
            dft_reg<B, false>(u);
            float2* dst = S + (size_t)(k * B) * N + c * R + row;
#pragma unroll
            for (int q = 0; q < B; ++q) dst[(size_t)q * N] = u[q];
        }
    }
    cl.sync();  // every CTA's rows are in S (release / acquire, cluster scope)

    // Phase 3: column DFT pass 1 over this CTA's column frequencies
    // v' = c R + rho (lanes over t), read from S.
#pragma unroll 1
    for (int task = tid; task < R * B; task += T) {
        const int rho = task / B, t = task % B;
        const float2* src = S + (size_t)(c * R + rho) * N + t;
        float2 v[A];
#pragma unroll
        for (int e = 0; e < A; ++e) v[e] = __ldcg(src + B * e);
        dft_reg<A, false>(v);
        if constexpr (kDiscard<N, V>) {
            // the B lanes of row rho (one warp) have read its N / 16 lines of S
            __syncwarp();
            const float2* line0 = S + (size_t)(c * R + rho) * N;
            for (int l = t; l < N / 16; l += B) discard_l2(line0 + 16 * l);
        }
        float2* p = buf + rho * RS + t;
#pragma unroll
        for (int k = 0; k < A; ++k) p[k * (B + 1)] = cmul(v[k], twA[k * B + t]);
    }
    // With A == B and one task per thread, the 16 lanes that wrote a row in
    // pass 1 are the ones that read it in pass 2: a warp barrier suffices.
    if constexpr (kRowPerHalfWarp<N, V>) __syncwarp(); else __syncthreads();

    // Phase 4: column DFT pass 2, Fourier-modulus projection with the c
    // relaxation and the 1/N^2 of the inverse, inverse pass 2 and conjugate
    // twiddle (lanes over k).
    // Fourier-error partial of each column frequency v' = c R + row (N elements:
    // A tasks of B): each task sums its B terms in order, the A lanes of the
    // row add theirs by a fixed butterfly, and lane k = 0 stores the row's
    // partial at e_part[j N + v'].  The grouping depends on neither the
    // cluster shape nor the thread count, so every launch variant gives the
    // same partials (R * A is a multiple of T: every lane takes every round).
    static_assert((R * A) % T == 0 && T % A == 0 && A <= 32, "error-partial lanes");
    const float* sq = args.sqrtIp + pat + (size_t)c * R * N;
    const float inv_n2 = 1.0f / (float)(N * N);
    const float cr = args.c, oc = 1.0f - args.c;
#pragma unroll 1
    for (int task = tid; task < R * A; task += T) {
        const int row = task / A, k = task % A;
        float2* p = buf + row * RS + k * (B + 1);
        float2 u[B];
#pragma unroll
        for (int t = 0; t < B; ++t) u[t] = p[t];
        dft_reg<B, false>(u);
        float err = 0.f;
        float sv[B];
        const float* sp = sq + (size_t)(row * A + k) * B;
        if constexpr (B % 4 == 0) {
#pragma unroll
            for (int q = 0; q < B; q += 4) {
                const float4 f = __ldcs(reinterpret_cast<const float4*>(sp + q));
                sv[q] = f.x; sv[q + 1] = f.y; sv[q + 2] = f.z; sv[q + 3] = f.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < B; ++q) sv[q] = sp[q];
        }
#pragma unroll
        for (int q = 0; q < B; ++q) {
#if PT_DBG_ENABLED
            if (!(sv[q] >= 0.f) || !isfinite(sv[q])) PT_DBG_FLAG(kDbgSqrtI);
#endif
            // |Psi| and Psi/|Psi| from one reciprocal square root
            const float m2 = cabs2(u[q]);
            const float rs = m2 > 0.f ? rsqrtf(m2) : 0.f;
            const float d = fmaf(m2, rs, -sv[q]);
            err = fmaf(d, d, err);
            if constexpr (!ERR_ONLY) {
                // c sqrt(I) Psi/|Psi| + (1 - c) Psi, scaled by 1/N^2; sqrt(I) + 0i where Psi = 0
                const float g = (cr * sv[q]) * rs + oc;
                u[q] = m2 > 0.f ? make_float2(u[q].x * (g * inv_n2), u[q].y * (g * inv_n2))
                                : make_float2(cr * sv[q] * inv_n2, 0.f);
            }
        }
#pragma unroll
        for (int o = A / 2; o > 0; o >>= 1) err += __shfl_xor_sync(0xffffffffu, err, o, A);
        if (k == 0) args.e_part[(size_t)j * N + c * R + row] = (double)err;
        if constexpr (!ERR_ONLY) {
            dft_reg<B, true>(u);
#pragma unroll
            for (int t = 0; t < B; ++t) p[t] = cconjmul(twB[t * A + k], u[t]);
        }
    }

    if constexpr (!ERR_ONLY) {
        __syncthreads();
        // Phase 5: column inverse pass 1 (lanes over the local rows rho);
        // spatial row r = t + B e of column frequency v' goes to S2[r][v'].
#pragma unroll 1
        for (int task = tid; task < R * B; task += T) {
            const int t = task / R, rho = task % R;
            const float2* p = buf + rho * RS + t;
            float2 v[A];
#pragma unroll
            for (int k = 0; k < A; ++k) v[k] = p[k * (B + 1)];
            dft_reg<A, true>(v);
            float2* dst = S2 + (size_t)t * N + c * R + rho;
#pragma unroll
            for (int e = 0; e < A; ++e) dst[(size_t)(B * e) * N] = v[e];
        }
        cl.sync();  // every CTA's columns are in S2

        // Phase 6: row inverse pass 2 with the conjugate twiddle (lanes over k),
        // this CTA's rows read from S2.
#pragma unroll 1
        for (int task = tid; task < R * A; task += T) {
            const int row = task / A, k = task % A;
            const float2* src = S2 + (size_t)(c * R + row) * N + k * B;
            float2 u[B];
            if constexpr (B % 2 == 0) {
#pragma unroll
                for (int t = 0; t < B; t += 2) {
                    const float4 f = __ldcg(reinterpret_cast<const float4*>(src + t));
                    u[t] = make_float2(f.x, f.y);
                    u[t + 1] = make_float2(f.z, f.w);
                }
            } else {
#pragma unroll
                for (int t = 0; t < B; ++t) u[t] = __ldcg(src + t);
            }
            if constexpr (kDiscard<N, V>) {
                // the lanes reading one 128-byte line are in this warp
                __syncwarp();
                if ((k * B) % 16 == 0) discard_l2(src);
            }
            dft_reg<B, true>(u);
            float2* p = buf + row * RS + k * (B + 1);
#pragma unroll
            for (int t = 0; t < B; ++t) p[t] = cconjmul(twB[t * A + k], u[t]);
        }
        if constexpr (kRowPerHalfWarp<N, V>) __syncwarp(); else __syncthreads();

        // Phase 7: row inverse pass 1, store y_k (lanes over t).
#pragma unroll 1
        for (int task = tid; task < R * B; task += T) {
            const int row = task / B, t = task % B;
            const int r = c * R + row;
            const float2* p = buf + row * RS + t;
            float2 v[A];
#pragma unroll
            for (int k = 0; k < A; ++k) v[k] = p[k * (B + 1)];
            dft_reg<A, true>(v);
            if constexpr (SP) {
                // d = psi' - psi; O_j += conj(P) d / max|P|^2, P += conj(O_j) d / max|O_j|^2
#pragma unroll
                for (int e = 0; e < A; ++e) {
                    const int n = t + B * e;
                    const float2 pv = args.P[r * N + n];
                    float2* op = args.O_mut + (size_t)(s.x + r) * args.Mc + s.y + n;
                    const float2 ov = *op;
                    const float2 d = csub(v[e], cmul_rn(pv, ov));
                    *op = cadd(ov, cscale(cconjmul(pv, d), inv_maxP));
                    args.P_mut[r * N + n] = cadd(pv, cscale(cconjmul(ov, d), inv_maxO));
#if PT_DBG_ENABLED
                    if (PT_DBG_NONFINITE2(*op) || PT_DBG_NONFINITE2(args.P_mut[r * N + n]))
                        PT_DBG_FLAG(kDbgNonFinite);
#endif
                }
            } else {
                float2* yo = args.y + pat + (size_t)r * N + t;
#pragma unroll
                for (int e = 0; e < A; ++e) {
#if PT_DBG_ENABLED
                    if (PT_DBG_NONFINITE2(v[e])) PT_DBG_FLAG(kDbgNonFinite);
#endif
                    __stcs(yo + B * e, v[e]);
                }
            }
        }
    }

}

template <int N, int V>
__global__ void __launch_bounds__(256) sqrt_permute_kernel(const float* __restrict__ I,
                                                           float* __restrict__ sqrtIp,
                                                           double* __restrict__ psum,
                                                           int* __restrict__ bad) {
    using G = Geo<N, V>;
    constexpr int A = G::A, B = G::B, R = G::R, KC = G::KC;
    __shared__ double red[8];
    const int j = blockIdx.y;
    const int pidx = blockIdx.x * 256 + threadIdx.x;
    double v64 = 0.0;
    if (pidx < N * N) {
        // pidx = ((cta * R + rho) * A + k1p) * B + k2p
        const int k2p = pidx % B;
        int tmp = pidx / B;
        const int k1p = tmp % A;
        tmp /= A;
        const int rho = tmp % R;
        const int cta = tmp / R;
        const int u = k1p + A * k2p;                       // row frequency
        const int v = (cta * KC + rho / B) + A * (rho % B);  // column frequency
        const float val = I[(size_t)j * N * N + (size_t)u * N + v];
        if (!(val >= 0.0f) || !isfinite(val)) atomicOr(bad, 1);
        sqrtIp[(size_t)j * N * N + pidx] = sqrtf(fmaxf(val, 0.0f));
        // the sums run over blocks of the natural order, so sum I (and every
        // Fourier error) does not depend on the layout of sqrt(I)
        v64 = (double)I[(size_t)j * N * N + pidx];
    }
    const double tot = block_sum_double<256>(v64, red);
    if (threadIdx.x == 0) psum[(size_t)j * gridDim.x + blockIdx.x] = tot;
}

// One cluster per exit wave; a sequential-projections step works on one given
// position.
template <int N, int MODE, int V>
__global__ void __launch_bounds__(Geo<N, V>::T, Cfg<N, V>::MINB) divide_kernel(const DivideArgs args) {
    pdl_wait();
    divide_body<N, MODE, V>(args, MODE == kModeSP ? args.sp_pos : (int)(blockIdx.x / Geo<N, V>::C));
}

// The divide step of several scans of side N in one launch (batching): the
// clusters are numbered over all their exit waves, scan s owning waves
// first[s] .. first[s + 1] - 1; each cluster runs the same work with its
// scan's arguments, so every scan's result is that of its own launch.
template <int N, int V>
__global__ void __launch_bounds__(Geo<N, V>::T, Cfg<N, V>::MINB)
    divide_ragged_kernel(const DivideArgs* __restrict__ table, const int* __restrict__ first,
                         int n_scans) {
    const int g = (int)(blockIdx.x / Geo<N, V>::C);
    int s = 0;
    while (s + 1 < n_scans && first[s + 1] <= g) ++s;
    divide_body<N, kModeDivide, V>(table[s], g - first[s]);
}

// Index in the permuted sqrt(I) layout of variant V of row frequency u and
// column frequency v (the inverse of the map in sqrt_permute_kernel).
template <int N, int V>
__device__ __forceinline__ int permuted_index(int u, int v) {
    using G = Geo<N, V>;
    constexpr int A = G::A, B = G::B, R = G::R, KC = G::KC;
    const int k1p = u % A, k2p = u / A;
    const int rho = ((v % A) % KC) * B + v / A;
    const int cta = (v % A) / KC;
    return ((cta * R + rho) * A + k1p) * B + k2p;
}

// sqrt(I) from the layout of variant VF (src) to that of variant VT (dst).
template <int N, int VF, int VT>
__global__ void __launch_bounds__(256) relayout_kernel(const float* __restrict__ src,
                                                       float* __restrict__ dst) {
    using G = Geo<N, VT>;
    constexpr int A = G::A, B = G::B, R = G::R, KC = G::KC;
    const int j = blockIdx.y;
    const int pidx = blockIdx.x * 256 + threadIdx.x;
    if (pidx >= N * N) return;
    const int k2p = pidx % B;
    int tmp = pidx / B;
    const int k1p = tmp % A;
    tmp /= A;
    const int rho = tmp % R;
    const int cta = tmp / R;
    const int u = k1p + A * k2p;
    const int v = (cta * KC + rho / B) + A * (rho % B);
    dst[(size_t)j * N * N + pidx] = src[(size_t)j * N * N + permuted_index<N, VF>(u, v)];
}

template <int N, int V = 0>
cudaError_t prepare_t() {
    cudaError_t e = cudaFuncSetAttribute(divide_kernel<N, kModeDivide, V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Geo<N, V>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(divide_ragged_kernel<N, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Geo<N, V>::SMEM);
    if (e != cudaSuccess) return e;
    if constexpr (Geo<N, V>::C > 8) {
        e = cudaFuncSetAttribute(divide_ragged_kernel<N, V>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(divide_kernel<N, kModeSP, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Geo<N, V>::SMEM);
    if (e != cudaSuccess) return e;
    if constexpr (Geo<N, V>::C > 8) {  // clusters above the portable size of 8
        e = cudaFuncSetAttribute(divide_kernel<N, kModeDivide, V>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(divide_kernel<N, kModeErrOnly, V>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(divide_kernel<N, kModeSP, V>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(divide_kernel<N, kModeErrOnly, V>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<N, V>::SMEM);
}

template <int N, int V = 0>
cudaError_t launch_t(const DivideArgs& a, cudaStream_t st) {
    using G = Geo<N, V>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.J * G::C);
    cfg.blockDim = dim3(G::T);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[3];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // Load-balanced placement: with the default (spread: the CTAs of a cluster
    // on distinct SMs) clusters of 16 never land on 16 of the 152 SMs; with
    // load balancing every SM takes CTAs (measured 0.907 -> 0.858 ms, large).
    attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
    // programmatic stream serialisation: the kernel may be launched while the
    // previous one finishes and waits for it in pdl_wait
    attr[2].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[2].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 3;
    if (a.sp) {
        cfg.gridDim = dim3((unsigned)G::C);  // one cluster: one position
        return cudaLaunchKernelEx(&cfg, divide_kernel<N, kModeSP, V>, a);
    }
    if (a.err_only) return cudaLaunchKernelEx(&cfg, divide_kernel<N, kModeErrOnly, V>, a);
    return cudaLaunchKernelEx(&cfg, divide_kernel<N, kModeDivide, V>, a);
}

template <int N, int V = 0>
cudaError_t launch_ragged_t(const DivideArgs* table, const int* first, int n, int total_waves,
                            cudaStream_t st) {
    using G = Geo<N, V>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total_waves * G::C);
    cfg.blockDim = dim3(G::T);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, divide_ragged_kernel<N, V>, table, first, n);
}

template <int N, int V = 0>
cudaError_t sqrt_t(const float* I, float* sqrtIp, double* psum, int* bad, int J, cudaStream_t st) {
    dim3 grid((N * N + 255) / 256, J);
    sqrt_permute_kernel<N, V><<<grid, 256, 0, st>>>(I, sqrtIp, psum, bad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_divide_ragged(int N, int variant, const DivideArgs* table, const int* first,
                                 int n, int total_waves, cudaStream_t st) {
    switch (N) {
        case 8: return launch_ragged_t<8>(table, first, n, total_waves, st);
        case 16: return launch_ragged_t<16>(table, first, n, total_waves, st);
        case 32: return launch_ragged_t<32>(table, first, n, total_waves, st);
        case 64: return launch_ragged_t<64>(table, first, n, total_waves, st);
        case 128:
            return variant == 1 ? launch_ragged_t<128, 1>(table, first, n, total_waves, st)
                                : launch_ragged_t<128, 0>(table, first, n, total_waves, st);
        case 256: return launch_ragged_t<256>(table, first, n, total_waves, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_relayout_sqrt(int N, int from, int to, const float* src, float* dst, int J,
                                 cudaStream_t st) {
    if (N != 128 || from == to || from < 0 || from > 1 || to < 0 || to > 1) return cudaErrorInvalidValue;
    dim3 grid((N * N + 255) / 256, J);
    if (from == 0)
        relayout_kernel<128, 0, 1><<<grid, 256, 0, st>>>(src, dst);
    else
        relayout_kernel<128, 1, 0><<<grid, 256, 0, st>>>(src, dst);
    return cudaGetLastError();
}

bool divide_supported(int N) {
    return N == 8 || N == 16 || N == 32 || N == 64 || N == 128 || N == 256;
}

int divide_cluster_size(int N, int variant) {
    if (N == 128 && variant == 1) return Geo<128, 1>::C;
    switch (N) {
        case 8: return Geo<8>::C;
        case 16: return Geo<16>::C;
        case 32: return Geo<32>::C;
        case 64: return Geo<64>::C;
        case 128: return Geo<128>::C;
        case 256: return Geo<256>::C;
    }
    return 0;
}

static void twiddles_ab(int N, int A, int B, std::vector<float2>& tw) {
    tw.resize((size_t)N);
    for (int k = 0; k < A; ++k)
        for (int t = 0; t < B; ++t) {
            const long m = ((long)t * k) % N;
            const double ang = -2.0 * M_PI * (double)m / (double)N;
            tw[(size_t)k * B + t] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
}

void divide_twiddles(int N, std::vector<float2>& tw) {
    switch (N) {
        case 8: twiddles_ab(N, Geo<8>::A, Geo<8>::B, tw); break;
        case 16: twiddles_ab(N, Geo<16>::A, Geo<16>::B, tw); break;
        case 32: twiddles_ab(N, Geo<32>::A, Geo<32>::B, tw); break;
        case 64: twiddles_ab(N, Geo<64>::A, Geo<64>::B, tw); break;
        case 128: twiddles_ab(N, Geo<128>::A, Geo<128>::B, tw); break;
        case 256: twiddles_ab(N, Geo<256>::A, Geo<256>::B, tw); break;
        default: tw.clear();
    }
}

cudaError_t divide_prepare(int N) {
    switch (N) {
        case 8: return prepare_t<8>();
        case 16: return prepare_t<16>();
        case 32: return prepare_t<32>();
        case 64: return prepare_t<64>();
        case 128: {
            cudaError_t e = prepare_t<128, 0>();
            return e != cudaSuccess ? e : prepare_t<128, 1>();
        }
        case 256: return prepare_t<256>();
    }
    return cudaErrorInvalidValue;
}


cudaError_t launch_divide(int N, const DivideArgs& a, cudaStream_t st) {
    switch (N) {
        case 8: return launch_t<8>(a, st);
        case 16: return launch_t<16>(a, st);
        case 32: return launch_t<32>(a, st);
        case 64: return launch_t<64>(a, st);
        case 128: return a.variant == 1 ? launch_t<128, 1>(a, st) : launch_t<128, 0>(a, st);
        case 256: return launch_t<256>(a, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_sqrt_permute(int N, int variant, const float* I, float* sqrtIp, double* psum,
                                int* bad, int J, cudaStream_t st) {
    if (N == 128 && variant == 1) return sqrt_t<128, 1>(I, sqrtIp, psum, bad, J, st);
    switch (N) {
        case 8: return sqrt_t<8>(I, sqrtIp, psum, bad, J, st);
        case 16: return sqrt_t<16>(I, sqrtIp, psum, bad, J, st);
        case 32: return sqrt_t<32>(I, sqrtIp, psum, bad, J, st);
        case 64: return sqrt_t<64>(I, sqrtIp, psum, bad, J, st);
        case 128: return sqrt_t<128>(I, sqrtIp, psum, bad, J, st);
        case 256: return sqrt_t<256>(I, sqrtIp, psum, bad, J, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ptycho
