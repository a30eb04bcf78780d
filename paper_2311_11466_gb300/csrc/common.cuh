// Device helpers shared by the library's kernels: complex arithmetic with a
// fixed rounding sequence, and small in-register DFTs of length 1..16.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ptycho {

// ---------------------------------------------------------------------------
// Complex float2 arithmetic.  The *_rn forms spell out every rounding step
// (no compiler contraction choice), so two kernels that evaluate the same
// expression produce the same bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cmul_rn(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)),
                       __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// The relaxed re-split of the abc update (Introduction, displayed equation):
//   x = a (b z + (1 - b) y) + (1 - a) x_prev,  z = P * O_j.
// Every kernel that forms x calls this one function, so a materialised x and
// the one formed on the fly inside the divide kernel are bit-identical.
__device__ __forceinline__ float2 resplit_rn(float2 z, float2 y, float2 xp, float a, float b) {
    const float ob = __fsub_rn(1.0f, b), oa = __fsub_rn(1.0f, a);
    const float tx = __fmaf_rn(b, z.x, __fmul_rn(ob, y.x));
    const float ty = __fmaf_rn(b, z.y, __fmul_rn(ob, y.y));
    return make_float2(__fmaf_rn(a, tx, __fmul_rn(oa, xp.x)),
                       __fmaf_rn(a, ty, __fmul_rn(oa, xp.y)));
}

// ---------------------------------------------------------------------------
// In-register DFT of length L in {1, 2, 4, 8, 16}, natural order in and out:
//   v[k] <- sum_e v[e] W_L^{e k},  W_L = exp(-2 pi i / L) (forward) or its
// conjugate (inverse, unscaled).  Radix-2 decimation in time, fully unrolled;
// the twiddles are the exact roots of unity of order 16 written out below.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr float cos16(int m) {
    // cos(2 pi m / 16)
    return (m & 15) == 0 ? 1.0f
         : (m & 15) == 1 ? 0.923879532511286756f
         : (m & 15) == 2 ? 0.707106781186547524f
         : (m & 15) == 3 ? 0.382683432365089772f
         : (m & 15) == 4 ? 0.0f
         : (m & 15) == 5 ? -0.382683432365089772f
         : (m & 15) == 6 ? -0.707106781186547524f
         : (m & 15) == 7 ? -0.923879532511286756f
         : (m & 15) == 8 ? -1.0f
         : (m & 15) == 9 ? -0.923879532511286756f
         : (m & 15) == 10 ? -0.707106781186547524f
         : (m & 15) == 11 ? -0.382683432365089772f
         : (m & 15) == 12 ? 0.0f
         : (m & 15) == 13 ? 0.382683432365089772f
         : (m & 15) == 14 ? 0.707106781186547524f
         : 0.923879532511286756f;
}
__host__ __device__ constexpr float sin16(int m) { return cos16(m - 4); }

// a * exp(-+ 2 pi i K / L); exact for the quarter turns.
template <int L, int K, bool INV>
__device__ __forceinline__ float2 mul_root(float2 a) {
    constexpr int m = ((K * (16 / L)) % 16 + 16) % 16;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 8) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (m == 4) {   // forward: * (-i); inverse: * (+i)
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (m == 12) {  // forward: * (+i); inverse: * (-i)
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float wr = cos16(m);
        constexpr float wi = INV ? sin16(m) : -sin16(m);
        return make_float2(fmaf(a.x, wr, -a.y * wi), fmaf(a.x, wi, a.y * wr));
    }
}

template <int L, bool INV, int K = 0>
__device__ __forceinline__ void dft_combine(float2* v, const float2* ev, const float2* od) {
    if constexpr (K < L / 2) {
        const float2 t = mul_root<L, K, INV>(od[K]);
        v[K] = cadd(ev[K], t);
        v[K + L / 2] = csub(ev[K], t);
        dft_combine<L, INV, K + 1>(v, ev, od);
    }
}

template <int L, bool INV>
__device__ __forceinline__ void dft_reg(float2* v) {
    static_assert(L == 1 || L == 2 || L == 4 || L == 8 || L == 16, "DFT length");
    if constexpr (L > 1) {
        float2 ev[L / 2], od[L / 2];
#pragma unroll
        for (int i = 0; i < L / 2; ++i) {
            ev[i] = v[2 * i];
            od[i] = v[2 * i + 1];
        }
        dft_reg<L / 2, INV>(ev);
        dft_reg<L / 2, INV>(od);
        dft_combine<L, INV>(v, ev, od);
    }
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel in the stream finishes;
// it waits here, before touching memory, until that kernel has completed and
// its writes are visible (a no-op for a kernel launched without it).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Deterministic block reduction of one double per thread (fixed tree order).
// Every thread of the block must call it; the result is valid in thread 0.
template <int THREADS>
__device__ __forceinline__ double block_sum_double(double v, double* scratch /* THREADS/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) scratch[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < THREADS / 32; ++i) s += scratch[i];
    }
    return s;
}

}  // namespace ptycho
