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
//
// The atomic mode builds the same sums with atomics: the object by
// shared-memory-staged atomics (scatter_staged_kernel), the probe by
// register-staged FP64 atomics (the same chunked pass); the order of the
// additions then depends on timing.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "debug.cuh"
#include "internal.h"

PTYCHO_DEBUG_UNIT(concur)

namespace ptycho {
namespace {

constexpr int kT = 256;

// Block maximum of non-negative doubles as the integer maximum of their bit
// patterns (the same order; no FP64 arithmetic).  Valid in thread 0.
__device__ __forceinline__ unsigned long long block_max_bits(unsigned long long v,
                                                             unsigned long long* scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_down_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) scratch[w] = v;
    __syncthreads();
    unsigned long long m = 0ull;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = scratch[i] > m ? scratch[i] : m;
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
// TR x TC object tile walks its list of overlapping windows (each entry
// carries the position index and the window corner, so one load per window);
// thread i owns column i % TC of rows i / TC + (kT / TC) k.  For each pixel the
// windows covering it are added in ascending position order whatever the tile
// shape, the numerator in FP32.  The denominator sum_j |P|^2 is summed like
// the probe's: FP32 partial sums over fixed ranges of positions (j < J/2 and
// j >= J/2) and an FP64 final sum of the partials.  The window list is in
// ascending position order, so the one change of range is a single list
// entry, the same for every thread of the block; FP64 work stays out of the
// loop (this part issues FP64 at a small fraction of the FP32 rate).  Every
// tile shape therefore gives bit-identical results (the shape is a pure
// launch choice).

constexpr int kListStage = 256;  // window-list entries staged in shared memory at a time

template <int TR, int TC>
__device__ __forceinline__ void gather_body(const ConcurScan& cs, const int tile) {
    constexpr int TRG = kT / TC;          // rows covered by one sweep of the CTA
    constexpr int KP = TR / TRG;          // pixels per thread
    static_assert(kT % TC == 0 && TR % TRG == 0, "object tile shape");
    __shared__ unsigned long long scratch[kT / 32];
    const int N = cs.N, Mr = cs.Mr, Mc = cs.Mc;
    const int tiles_c = cs.cb.tiles_c;
    const int ti = tile / tiles_c, tj = tile % tiles_c;
    const int tx = threadIdx.x % TC, ty = threadIdx.x / TC;
    const int mc = tj * TC + tx;
    const int mr0 = ti * TR + ty;
    const float2* __restrict__ y = cs.y;
    const float2* __restrict__ P = cs.P;
    const int4* __restrict__ tile_win = cs.cb.tile_win;
    float2 acc[KP];
    float dg[KP];           // denominator: FP32 partial of the current position range
    double dd[KP];          // and the FP64 total of the ranges done
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        acc[k] = make_float2(0.f, 0.f);
        dg[k] = 0.f;
        dd[k] = 0.0;
    }
    const size_t NN = (size_t)N * N;
    const int l0 = cs.cb.tile_ptr[tile], l1 = cs.cb.tile_ptr[tile + 1];
    const int js = cs.J / 2;   // first position of the second range
    // The windows of one range of list entries, added for every pixel of this
    // thread in list order.  Windows go in groups of kGroup: the loads of a
    // whole group are issued before its arithmetic, so several windows' y and
    // P are in flight at once (a window that misses a pixel loads P[0] and no y).
    auto add_one = [&](const int4 w, const int k, float2 pv, float2 yv) {
        (void)w;
        // conj(P) y and |P|^2 as chains of fused multiply-adds into the sums
        acc[k].x = fmaf(pv.x, yv.x, fmaf(pv.y, yv.y, acc[k].x));
        acc[k].y = fmaf(pv.x, yv.y, fmaf(-pv.y, yv.x, acc[k].y));
        dg[k] = fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, dg[k]));
    };
    auto add_range = [&](const int4* ent, int n) {
        constexpr int kGroup = 8;
        int l = 0;
        for (; l + kGroup <= n; l += kGroup) {
            float2 pv[kGroup][KP], yv[kGroup][KP];
            bool ok[kGroup][KP];
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                const int4 w = ent[l + g];  // (position j, row, col) of the window
                const int cc = mc - w.z;
                const bool cin = (unsigned)cc < (unsigned)N;
                const float2* yj = y + (size_t)w.x * NN;
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    const int rr = mr0 + TRG * k - w.y;
                    ok[g][k] = cin && (unsigned)rr < (unsigned)N;
                    const int o = ok[g][k] ? rr * N + cc : 0;
                    pv[g][k] = __ldg(P + o);
                    yv[g][k] = ok[g][k] ? __ldcs(yj + o) : make_float2(0.f, 0.f);
                }
            }
#pragma unroll
            for (int g = 0; g < kGroup; ++g)
#pragma unroll
                for (int k = 0; k < KP; ++k)
                    if (ok[g][k]) add_one(ent[l + g], k, pv[g][k], yv[g][k]);
        }
        for (; l < n; ++l) {
            const int4 w = ent[l];
            const int cc = mc - w.z;
            const bool cin = (unsigned)cc < (unsigned)N;
            const float2* yj = y + (size_t)w.x * NN;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const int rr = mr0 + TRG * k - w.y;
                if (cin && (unsigned)rr < (unsigned)N) {
                    const int o = rr * N + cc;
                    add_one(w, k, __ldg(P + o), __ldcs(yj + o));
                }
            }
        }
    };
    // The tile's window list is staged in shared memory (kListStage entries at
    // a time), so the loads of y and P depend on a shared-memory load rather
    // than on a global one.  The list is in ascending position order: each
    // batch splits into the entries of the first position range and those of
    // the second (a binary search, the same for every thread), and the
    // denominator's FP32 partial moves to FP64 once, between the two.
    __shared__ int4 list[kListStage];
    bool second = false;
    for (int b0 = l0; b0 < l1; b0 += kListStage) {
        const int nb = min(kListStage, l1 - b0);
        __syncthreads();  // the previous batch is consumed
        for (int i = threadIdx.x; i < nb; i += kT) {
            int4 w = __ldg(tile_win + b0 + i);
#if PT_DBG_ENABLED
            // checked build: an entry whose window leaves the object is recorded
            // and replaced by one that covers no pixel of the tile
            if (w.x < 0 || w.y < 0 || w.z < 0 || w.y > Mr - N || w.z > Mc - N) {
                PT_DBG_FLAG(kDbgWindow);
                w = make_int4(0, -2 * N, -2 * N, 0);
            }
#endif
            list[i] = w;
        }
        __syncthreads();
        int lo = 0, hi = nb;   // first entry of the batch with position >= js
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (list[mid].x < js) lo = mid + 1; else hi = mid;
        }
        add_range(list, lo);
        if (!second && lo < nb) {
            second = true;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                dd[k] = (double)dg[k];
                dg[k] = 0.f;
            }
        }
        add_range(list + lo, nb - lo);
    }
    unsigned long long mx = 0ull;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int mr = mr0 + TRG * k;
        if (mr < Mr && mc < Mc) {
            const double den = dd[k] + (double)dg[k];   // the final sum, FP64
            cs.cb.numO[(size_t)mr * Mc + mc] = acc[k];
            cs.cb.denO[(size_t)mr * Mc + mc] = den;
            const unsigned long long b = (unsigned long long)__double_as_longlong(den);
            mx = b > mx ? b : mx;
        }
    }
    const unsigned long long bm = block_max_bits(mx, scratch);
    if (threadIdx.x == 0) atomicMax(cs.cb.maxO, bm);
}

// Atomic variant: one CTA row per (position, 256 probe pixels), scatter-add.
__global__ void __launch_bounds__(kT) scatter_object_kernel(
    const float2* __restrict__ y, const float2* __restrict__ P, const int2* __restrict__ pos,
    int N, int Mc, float2* __restrict__ numO, double* __restrict__ denO) {
    const int j = blockIdx.y;
    const int r = blockIdx.x * kT + threadIdx.x;
    if (r >= N * N) return;
    const int rr = r / N, cc = r % N;
    const int2 s = pos[j];
    const float2 pv = __ldg(P + r);
    const float2 yv = __ldcs(y + (size_t)j * N * N + r);
    const size_t m = (size_t)(s.x + rr) * Mc + s.y + cc;
    atomicAdd(numO + m, cconjmul(pv, yv));
    atomicAdd(denO + m, (double)cabs2(pv));
}

// Staged-atomic variant (the default of PTYCHO_CONCUR_ATOMIC): one CTA per
// (group of positions, band of window rows).  The group's windows,
// restricted to the band, lie in one box of the object (rows: the band's
// rows plus the group's row spread; columns: N plus its column spread), which
// is accumulated in shared memory and then added to the global numerator
// (FP32 atomics) and denominator (FP64 atomics) once per box pixel instead
// of once per window pixel.  Positions are added one after another with a
// barrier between them, every thread taking the same window pixels of each
// position, so no two threads touch a box pixel at once and the box needs no
// shared-memory atomics; the band's probe values, the same for every
// position of the group, are loaded once per thread.  The global atomics make
// the order of the additions, and so the rounding, depend on timing: this
// mode is not bitwise reproducible (the gather is).
constexpr int kScatterCap = 8192;  // box pixels (float2 + float each: 96 KB of shared memory)
constexpr int kScatterMaxG = 16;   // positions per group
constexpr int kScT = 512;          // threads of the staged kernel (two CTAs per SM)
constexpr int kScatterPx = 4;      // window pixels per thread and band (a band is <= 2048 pixels)

__global__ void __launch_bounds__(kScT, 2) scatter_staged_kernel(const ConcurScan cs) {
    pdl_wait();
    extern __shared__ float4 sc_smem[];
    __shared__ int s_j[kScatterMaxG], s_base[kScatterMaxG];
    const int4 g = cs.cb.sc_groups[blockIdx.x];  // {first, count, row min, col min}
    const int2 ex = cs.cb.sc_ext[blockIdx.x];    // {row spread, col spread}
    const int N = cs.N, RB = cs.cb.sc_rows, band = blockIdx.y;
    const int H = RB + ex.x, W = N + ex.y, HW = H * W;
    const int r0 = g.z + band * RB;              // first object row of the box
#if PT_DBG_ENABLED
    // checked build: a box outside the object or the shared memory is recorded and skipped
    if (r0 + H > cs.Mr || g.w + W > cs.Mc || HW > cs.cb.sc_box || g.y > kScatterMaxG) {
        if (threadIdx.x == 0) PT_DBG_FLAG(kDbgWindow);
        return;
    }
#endif
    float2* snum = reinterpret_cast<float2*>(sc_smem);
    float* sden = reinterpret_cast<float*>(snum + HW);
    // the group's positions and their offsets in the box
    if ((int)threadIdx.x < g.y) {
        const int j = cs.cb.sc_ord[g.x + threadIdx.x];
        const int2 s = cs.pos[j];
        s_j[threadIdx.x] = j;
        s_base[threadIdx.x] = (s.x - g.z) * W + (s.y - g.w);
    }
    for (int i = threadIdx.x; i < HW; i += kScT) {
        snum[i] = make_float2(0.f, 0.f);
        sden[i] = 0.f;
    }
    const int lgN = __ffs(N) - 1;
    const int band_px = RB * N;
    const size_t NN = (size_t)N * N, band0 = (size_t)band * band_px;
    float2 pv[kScatterPx];
    float pd[kScatterPx];
    int boff[kScatterPx];
#pragma unroll
    for (int i = 0; i < kScatterPx; ++i) {
        const int p = threadIdx.x + i * kScT;
        const int rr = p >> lgN, cc = p & (N - 1);
        pv[i] = p < band_px ? __ldg(cs.P + band0 + p) : make_float2(0.f, 0.f);
        pd[i] = cabs2(pv[i]);
        boff[i] = rr * W + cc;
    }
    __syncthreads();  // the box is zeroed, the position table written
    const float2* __restrict__ y = cs.y;
    float2 yv[kScatterPx];
    {
        const int j0 = s_j[0];
#pragma unroll
        for (int i = 0; i < kScatterPx; ++i) {
            const int p = threadIdx.x + i * kScT;
            yv[i] = p < band_px ? __ldcs(y + (size_t)j0 * NN + band0 + p) : make_float2(0.f, 0.f);
        }
    }
    for (int k = 0; k < g.y; ++k) {
        // the next position's y, loaded before this one is added
        float2 yn[kScatterPx];
        const bool more = k + 1 < g.y;
        const int jn = more ? s_j[k + 1] : 0;
#pragma unroll
        for (int i = 0; i < kScatterPx; ++i) {
            const int p = threadIdx.x + i * kScT;
            yn[i] = (more && p < band_px) ? __ldcs(y + (size_t)jn * NN + band0 + p)
                                          : make_float2(0.f, 0.f);
        }
        const int base = s_base[k];
#pragma unroll
        for (int i = 0; i < kScatterPx; ++i) {
            if (threadIdx.x + i * kScT < band_px) {
                const int b = base + boff[i];
                float2 sv = snum[b];
                sv.x = fmaf(pv[i].x, yv[i].x, fmaf(pv[i].y, yv[i].y, sv.x));
                sv.y = fmaf(pv[i].x, yv[i].y, fmaf(-pv[i].y, yv[i].x, sv.y));
                snum[b] = sv;
                sden[b] += pd[i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kScatterPx; ++i) yv[i] = yn[i];
    }
    float2* __restrict__ numO = cs.cb.numO;
    double* __restrict__ denO = cs.cb.denO;
    for (int i = threadIdx.x; i < HW; i += kScT) {
        const float d = sden[i];
        const float2 nv = snum[i];
        if (d != 0.f || nv.x != 0.f || nv.y != 0.f) {
            const int r = i / W, c = i - r * W;
            const size_t m = (size_t)(r0 + r) * cs.Mc + g.w + c;
            atomicAdd(numO + m, nv);
            atomicAdd(denO + m, (double)d);
        }
    }
}

__global__ void __launch_bounds__(kT) max_double_kernel(const double* __restrict__ v, size_t n,
                                                        unsigned long long* __restrict__ out) {
    pdl_wait();
    __shared__ double scratch[kT / 32];
    double m = 0.0;
    for (size_t i = blockIdx.x * (size_t)kT + threadIdx.x; i < n; i += (size_t)gridDim.x * kT)
        m = fmax(m, v[i]);
    const double bm = block_max_double(m, scratch);
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(bm));
}

// O = num / (den + alpha max(den)): the regularised denominator in FP64,
// rounded once to FP32 for the division of the FP32 numerator.  Block 0 also
// clears the probe maximum for the probe sweep that comes next.
__device__ __forceinline__ void onorm_body(const ConcurScan& cs, const int block) {
    const size_t M = (size_t)cs.Mr * cs.Mc;
    const size_t m = block * (size_t)kT + threadIdx.x;
    if (block == 0 && threadIdx.x == 0) *cs.cb.maxP = 0ull;
    if (m >= M) return;
    const double am = cs.alpha * __longlong_as_double((long long)*cs.cb.maxO);
    const float d = (float)(cs.cb.denO[m] + am);
    const float2 nv = cs.cb.numO[m];
    const float2 o = d > 0.f ? make_float2(nv.x / d, nv.y / d) : make_float2(0.f, 0.f);
    cs.O[m] = o;
#if PT_DBG_ENABLED
    if (PT_DBG_NONFINITE2(o)) PT_DBG_FLAG(kDbgNonFinite);
#endif
}

// Probe partial sums over a chunk of positions; thread = PPT adjacent probe
// pixels (PPT = 2: y read with 16-byte loads).  Each pixel adds its chunk's
// positions in ascending order with the same operations for either PPT, so
// both give bit-identical partials (a pure launch choice).  ATOMIC (the
// atomic concur mode): the chunk's sums, staged in registers, are added to
// the FP64 totals with FP64 atomics instead of being stored for the ordered
// reduction.
template <int PPT, bool ATOMIC = false>
__device__ __forceinline__ void ppart_body(const ConcurScan& cs, const int bx, const int ch) {
    static_assert(PPT == 1 || PPT == 2, "pixels per thread");
    const int N = cs.N, Mc = cs.Mc, J = cs.J, chunks = cs.cb.chunks;
    const int r = (bx * kT + threadIdx.x) * PPT;
    if (r >= N * N) return;   // N is even, so with PPT = 2 both pixels are inside
    const int rr = r / N, cc = r % N;
    const int j0 = (int)(((long)ch * J) / chunks), j1 = (int)(((long)(ch + 1) * J) / chunks);
    const size_t NN = (size_t)N * N;
    const float2* __restrict__ y = cs.y;
    const float2* __restrict__ O = cs.O;
    const int2* __restrict__ pos = cs.pos;
    float2 acc[PPT];
    float den[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        acc[i] = make_float2(0.f, 0.f);
        den[i] = 0.f;
    }
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const int2 s = pos[j];
#if PT_DBG_ENABLED
        // checked build: a window outside the object is recorded and skipped
        if (s.x < 0 || s.y < 0 || s.x > cs.Mr - N || s.y > Mc - N) {
            PT_DBG_FLAG(kDbgWindow);
            continue;
        }
#endif
        const float2* op = O + (size_t)(s.x + rr) * Mc + s.y + cc;
        float2 yv[PPT];
        if constexpr (PPT == 2) {
            const float4 f = __ldcs(reinterpret_cast<const float4*>(y + (size_t)j * NN + r));
            yv[0] = make_float2(f.x, f.y);
            yv[1] = make_float2(f.z, f.w);
        } else {
            yv[0] = __ldcs(y + (size_t)j * NN + r);
        }
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
            const float2 ov = __ldg(op + i);
            // conj(O) y and |O|^2 as chains of fused multiply-adds into the sums
            acc[i].x = fmaf(ov.x, yv[i].x, fmaf(ov.y, yv[i].y, acc[i].x));
            acc[i].y = fmaf(ov.x, yv[i].y, fmaf(-ov.y, yv[i].x, acc[i].y));
            den[i] = fmaf(ov.x, ov.x, fmaf(ov.y, ov.y, den[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        if constexpr (ATOMIC) {
            atomicAdd(&cs.cb.numP[r + i].x, (double)acc[i].x);
            atomicAdd(&cs.cb.numP[r + i].y, (double)acc[i].y);
            atomicAdd(cs.cb.denP + r + i, (double)den[i]);
        } else {
            cs.cb.partP[(size_t)ch * NN + r + i] = acc[i];
            cs.cb.partPd[(size_t)ch * NN + r + i] = den[i];
        }
    }
}

// FP64 totals of the probe partials: a block takes kT / RG probe pixels, its
// RG thread groups each add a contiguous range of chunks in order, and the
// group totals are added in group order (a fixed order: deterministic; RG = 1
// when there are few chunks, 8 when there are many).  The same blocks also
// add the per-CTA Fourier-error partials of the divide step in fixed slices,
// one FP64 slice total per block, so the final sum (in the normalise kernel)
// is over one value per block.
constexpr int kManyChunks = 8;  // above this the chunks are added by 8 thread groups

template <int RG>
__device__ __forceinline__ void preduce_body(const ConcurScan& cs, const int block,
                                             const int n_blocks) {
    constexpr int RP = kT / RG;
    __shared__ double gx[RG][RP], gy[RG][RP], gd[RG][RP];
    __shared__ double scratch_s[kT / 32], scratch_m[kT / 32];
    const int NN = cs.N * cs.N, chunks = cs.cb.chunks;
    const int px = threadIdx.x % RP, grp = threadIdx.x / RP;
    const int r = block * RP + px;
    const int c0 = (grp * chunks) / RG, c1 = ((grp + 1) * chunks) / RG;
    double nx = 0.0, ny = 0.0, d = 0.0;
    if (r < NN) {
        for (int ch = c0; ch < c1; ++ch) {
            const float2 p = cs.cb.partP[(size_t)ch * NN + r];
            nx += (double)p.x;
            ny += (double)p.y;
            d += (double)cs.cb.partPd[(size_t)ch * NN + r];
        }
    }
    double mx = 0.0;
    if constexpr (RG == 1) {
        if (r < NN) {
            cs.cb.numP[r] = make_double2(nx, ny);
            cs.cb.denP[r] = d;
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
            cs.cb.numP[r] = make_double2(tx, ty);
            cs.cb.denP[r] = td;
            mx = td;
        }
    }
    const int n_part = cs.n_part;
    const int per = (n_part + n_blocks - 1) / n_blocks;
    const int e0 = block * per, e1 = min(n_part, e0 + per);
    double es = 0.0;
    for (int i = e0 + (int)threadIdx.x; i < e1; i += kT) es += cs.e_part[i];
    const double slice = block_sum_double<kT>(es, scratch_s);
    if (threadIdx.x == 0) cs.cb.e_slice[block] = slice;
    const double bm = block_max_double(mx, scratch_m);
    if (threadIdx.x == 0) atomicMax(cs.cb.maxP, (unsigned long long)__double_as_longlong(bm));
}

// Probe update, plus (block 0) the iteration's Fourier error, stored in the
// ring at the slot of the device-side iteration counter (so a captured graph
// replays correctly), and the reset of the object maximum.
__device__ __forceinline__ void pnorm_body(const ConcurScan& cs, const int block, const int n_slice) {
    __shared__ double scratch[kT / 32];
    const int NN = cs.N * cs.N;
    const int r = block * kT + threadIdx.x;
    if (r < NN) {
        const double mx = __longlong_as_double((long long)*cs.cb.maxP);
        const double d = cs.cb.denP[r] + cs.alpha * mx;
        const double2 nv = cs.cb.numP[r];
        const float2 p = d > 0.0 ? make_float2((float)(nv.x / d), (float)(nv.y / d)) : make_float2(0.f, 0.f);
        cs.P[r] = p;
#if PT_DBG_ENABLED
        if (PT_DBG_NONFINITE2(p)) PT_DBG_FLAG(kDbgNonFinite);
#endif
    }
    if (block == 0) {
        double s = 0.0;
        for (int i = threadIdx.x; i < n_slice; i += kT) s += cs.cb.e_slice[i];
        const double tot = block_sum_double<kT>(s, scratch);
        if (threadIdx.x == 0) {
            const unsigned long long k = *cs.d_iter;
            cs.e_ring[k % (unsigned long long)cs.ring_cap] = tot * cs.inv_sumI;
            *cs.d_iter = k + 1;
            *cs.cb.maxO = 0ull;
        }
    }
}

// ---- one scan per launch -----------------------------------------------------
template <int TR, int TC>
__global__ void __launch_bounds__(kT) concur_object_kernel(const ConcurScan cs) {
    pdl_wait();
    gather_body<TR, TC>(cs, blockIdx.x);
}
__global__ void __launch_bounds__(kT) object_normalise_kernel(const ConcurScan cs) {
    pdl_wait();
    onorm_body(cs, blockIdx.x);
}
template <int PPT>
__global__ void __launch_bounds__(kT) probe_partial_kernel(const ConcurScan cs) {
    pdl_wait();
    ppart_body<PPT>(cs, blockIdx.x, blockIdx.y);
}
template <int PPT>
__global__ void __launch_bounds__(kT) probe_partial_atomic_kernel(const ConcurScan cs) {
    pdl_wait();
    ppart_body<PPT, true>(cs, blockIdx.x, blockIdx.y);
}
template <int RG>
__global__ void __launch_bounds__(kT) probe_reduce_kernel(const ConcurScan cs) {
    pdl_wait();
    preduce_body<RG>(cs, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kT) probe_normalise_kernel(const ConcurScan cs, int n_slice) {
    pdl_wait();
    pnorm_body(cs, blockIdx.x, n_slice);
}

// ---- several scans per launch (batching) ---------------------------------------
// first[s] is the first block of scan s in this launch's numbering; every block
// runs the single-scan work with its scan's arguments, so each scan's results
// are those of its own launches.
__device__ __forceinline__ int find_scan(const int* __restrict__ first, int n, int b) {
    int s = 0;
    while (s + 1 < n && first[s + 1] <= b) ++s;
    return s;
}
template <int TR, int TC>
__global__ void __launch_bounds__(kT) ragged_gather_kernel(const ConcurScan* __restrict__ scans,
                                                           const int* __restrict__ first, int n) {
    const int s = find_scan(first, n, blockIdx.x);
    gather_body<TR, TC>(scans[s], blockIdx.x - first[s]);
}
__global__ void __launch_bounds__(kT) ragged_onorm_kernel(const ConcurScan* __restrict__ scans,
                                                          const int* __restrict__ first, int n) {
    const int s = find_scan(first, n, blockIdx.x);
    onorm_body(scans[s], blockIdx.x - first[s]);
}
template <int PPT>
__global__ void __launch_bounds__(kT) ragged_ppart_kernel(const ConcurScan* __restrict__ scans,
                                                          const int* __restrict__ first, int n) {
    const int s = find_scan(first, n, blockIdx.x);
    const ConcurScan& cs = scans[s];
    const int b = blockIdx.x - first[s];
    const int per_chunk = (cs.N * cs.N / PPT + kT - 1) / kT;
    ppart_body<PPT>(cs, b % per_chunk, b / per_chunk);
}
__global__ void __launch_bounds__(kT) ragged_preduce_kernel(const ConcurScan* __restrict__ scans,
                                                            const int* __restrict__ first, int n) {
    const int s = find_scan(first, n, blockIdx.x);
    const ConcurScan& cs = scans[s];
    const int nb = first[s + 1] - first[s];
    if (cs.cb.chunks > kManyChunks)
        preduce_body<8>(cs, blockIdx.x - first[s], nb);
    else
        preduce_body<1>(cs, blockIdx.x - first[s], nb);
}
__global__ void __launch_bounds__(kT) ragged_pnorm_kernel(const ConcurScan* __restrict__ scans,
                                                          const int* __restrict__ first,
                                                          const int* __restrict__ n_slice, int n) {
    const int s = find_scan(first, n, blockIdx.x);
    pnorm_body(scans[s], blockIdx.x - first[s], n_slice[s]);
}

// Stage 1 of a two-level sum: block b adds the contiguous slice b of parts.
__global__ void __launch_bounds__(kT) slice_sums_kernel(const double* __restrict__ parts, int n,
                                                        double* __restrict__ out) {
    pdl_wait();
    __shared__ double scratch[kT / 32];
    const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int e0 = (int)blockIdx.x * per, e1 = min(n, e0 + per);
    double s = 0.0;
    for (int i = e0 + (int)threadIdx.x; i < e1; i += kT) s += parts[i];
    const double tot = block_sum_double<kT>(s, scratch);
    if (threadIdx.x == 0) out[blockIdx.x] = tot;
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

void build_tile_csr(const int32_t* pos_rc, int J, int N, int Mr, int Mc, TileShape sh,
                    std::vector<int>& ptr, std::vector<int4>& list) {
    const int tr = (Mr + sh.rows - 1) / sh.rows, tc = (Mc + sh.cols - 1) / sh.cols;
    ptr.assign((size_t)tr * tc + 1, 0);
    for (int j = 0; j < J; ++j) {
        const int r = pos_rc[2 * j], c = pos_rc[2 * j + 1];
        for (int ti = r / sh.rows; ti <= (r + N - 1) / sh.rows; ++ti)
            for (int tj = c / sh.cols; tj <= (c + N - 1) / sh.cols; ++tj) ptr[(size_t)ti * tc + tj + 1]++;
    }
    for (size_t t = 1; t < ptr.size(); ++t) ptr[t] += ptr[t - 1];
    list.resize((size_t)ptr.back());
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int j = 0; j < J; ++j) {
        const int r = pos_rc[2 * j], c = pos_rc[2 * j + 1];
        for (int ti = r / sh.rows; ti <= (r + N - 1) / sh.rows; ++ti)
            for (int tj = c / sh.cols; tj <= (c + N - 1) / sh.cols; ++tj)
                list[(size_t)fill[(size_t)ti * tc + tj]++] = make_int4(j, r, c, 0);
    }
}

// Groups for the staged-atomic object concur.  A band of a window is at most
// 2048 pixels (kScatterPx per thread); positions are taken in a spatial
// order -- strips of rows N/16 high (at least 8), by column within a strip --
// and a group grows while its box, band rows + row spread by N + column
// spread, stays within kScatterCap pixels and it has at most kScatterMaxG
// positions.  A raster row of a scan becomes a run of neighbours along the
// columns, whose windows overlap the most.
void build_scatter_groups(const int32_t* pos_rc, int J, int N, std::vector<int>& ord,
                          std::vector<int4>& groups, std::vector<int2>& ext, int* rows, int* box) {
    int rb = 2048 / N;
    if (rb > N) rb = N;
    if (rb < 1) rb = 1;
    *rows = rb;
    const int strip = N / 16 > 8 ? N / 16 : 8;
    ord.resize((size_t)J);
    for (int j = 0; j < J; ++j) ord[(size_t)j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const int sa = pos_rc[2 * a] / strip, sb = pos_rc[2 * b] / strip;
        if (sa != sb) return sa < sb;
        return pos_rc[2 * a + 1] < pos_rc[2 * b + 1];
    });
    groups.clear();
    ext.clear();
    int biggest = 0;
    for (int k = 0; k < J;) {
        const int j0 = ord[(size_t)k];
        int rmin = pos_rc[2 * j0], rmax = rmin, cmin = pos_rc[2 * j0 + 1], cmax = cmin;
        int cnt = 1;
        while (k + cnt < J && cnt < kScatterMaxG) {
            const int j = ord[(size_t)(k + cnt)];
            const int r = pos_rc[2 * j], c = pos_rc[2 * j + 1];
            const int nr0 = r < rmin ? r : rmin, nr1 = r > rmax ? r : rmax;
            const int nc0 = c < cmin ? c : cmin, nc1 = c > cmax ? c : cmax;
            if ((long)(rb + nr1 - nr0) * (N + nc1 - nc0) > kScatterCap) break;
            rmin = nr0, rmax = nr1, cmin = nc0, cmax = nc1;
            ++cnt;
        }
        groups.push_back(make_int4(k, cnt, rmin, cmin));
        ext.push_back(make_int2(rmax - rmin, cmax - cmin));
        const int b = (rb + rmax - rmin) * (N + cmax - cmin);
        biggest = b > biggest ? b : biggest;
        k += cnt;
    }
    *box = biggest;
}

cudaError_t concur_prepare() {
    return cudaFuncSetAttribute(scatter_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kScatterCap * (sizeof(float2) + sizeof(float))));
}

size_t tile_csr_ptr_bound(int N, int Mr, int Mc) {
    (void)N;
    size_t m = 0;
    for (const TileShape& sh : kGatherShape) {
        const size_t t = (size_t)((Mr + sh.rows - 1) / sh.rows) * ((Mc + sh.cols - 1) / sh.cols) + 1;
        m = t > m ? t : m;
    }
    return m;
}

size_t tile_csr_entries_bound(int J, int N) {
    size_t m = 0;
    for (const TileShape& sh : kGatherShape) {
        // a window of side N touches at most ceil(N / s) + 1 tiles of side s along
        // each axis (one more than it fills when it straddles a tile boundary)
        const size_t t = (size_t)((N + sh.rows - 1) / sh.rows + 1) * ((N + sh.cols - 1) / sh.cols + 1);
        m = t > m ? t : m;
    }
    return (size_t)J * m;
}

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

// A kernel of the deterministic concur step, launched with programmatic stream
// serialisation: its launch overlaps the end of the previous kernel, and it
// waits in pdl_wait before touching memory (measured: concur 0.229 -> 0.220 ms
// per 1024 x 256^2 iteration).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, cudaStream_t st, Args... args) {
    return launch_pdl_ex(kern, grid, dim3(kT), 0, st, args...);
}

cudaError_t launch_gather(const ConcurScan& cs, cudaStream_t st) {
    const unsigned grid = (unsigned)(cs.cb.tiles_r * cs.cb.tiles_c);
    switch (cs.cb.gather_shape) {
        case 0: return launch_pdl(concur_object_kernel<16, 32>, dim3(grid), st, cs);
        case 1: return launch_pdl(concur_object_kernel<8, 32>, dim3(grid), st, cs);
        case 2: return launch_pdl(concur_object_kernel<32, 32>, dim3(grid), st, cs);
        case 3: return launch_pdl(concur_object_kernel<8, 64>, dim3(grid), st, cs);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_probe_partial(const ConcurScan& cs, cudaStream_t st) {
    const int NN = cs.N * cs.N;
    if (cs.cb.probe_ppt == 2)
        return launch_pdl(probe_partial_kernel<2>, dim3((NN / 2 + kT - 1) / kT, cs.cb.chunks), st, cs);
    return launch_pdl(probe_partial_kernel<1>, dim3((NN + kT - 1) / kT, cs.cb.chunks), st, cs);
}

cudaError_t launch_concur(const ConcurScan& cs, int concur_mode, bool update_probe, cudaStream_t st) {
    const size_t M = (size_t)cs.Mr * cs.Mc;
    const int NN = cs.N * cs.N;
    const ConcurBufs& cb = cs.cb;
    if (concur_mode == 0) {
        cudaError_t e = launch_gather(cs, st);
        if (e != cudaSuccess) return e;
    } else {
        cudaMemsetAsync(cb.numO, 0, M * sizeof(float2), st);
        cudaMemsetAsync(cb.denO, 0, M * sizeof(double), st);
        if (cb.sc_n > 0) {
            const size_t smem = (size_t)cb.sc_box * (sizeof(float2) + sizeof(float));
            cudaError_t e = launch_pdl_ex(scatter_staged_kernel, dim3(cb.sc_n, cs.N / cb.sc_rows), dim3(kScT),
                                          smem, st, cs);
            if (e != cudaSuccess) return e;
        } else {
            scatter_object_kernel<<<dim3((NN + kT - 1) / kT, cs.J), kT, 0, st>>>(
                cs.y, cs.P, cs.pos, cs.N, cs.Mc, cb.numO, cb.denO);
        }
        cudaError_t e = launch_pdl(max_double_kernel, dim3(304), st, (const double*)cb.denO, M, cb.maxO);
        if (e != cudaSuccess) return e;
    }
    {
        cudaError_t e = launch_pdl(object_normalise_kernel, dim3((unsigned)((M + kT - 1) / kT)), st, cs);
        if (e != cudaSuccess) return e;
    }
    if (!update_probe) {
        // the probe is held: the iteration's Fourier error from the divide
        // kernel's partials (slices summed into the probe-reduce slice buffer,
        // unused in this iteration), and the object maximum cleared for the
        // next gather
        const int nb = probe_reduce_blocks(cs.N, cb.chunks);
        slice_sums_kernel<<<nb, kT, 0, st>>>(cs.e_part, cs.n_part, cb.e_slice);
        record_error_kernel<<<1, kT, 0, st>>>(cb.e_slice, nb, cs.inv_sumI, cs.e_ring, cs.d_iter,
                                              cs.ring_cap);
        cudaMemsetAsync(cb.maxO, 0, sizeof(unsigned long long), st);
        return cudaGetLastError();
    }
    const int n_slice = probe_reduce_blocks(cs.N, cb.chunks);
    if (concur_mode != 0) {
        // atomic mode: FP64 atomics of the register-staged chunk sums, then the
        // probe maximum and the error slices (the probe maximum was cleared by
        // the object normalisation)
        cudaMemsetAsync(cb.numP, 0, NN * sizeof(double2), st);
        cudaMemsetAsync(cb.denP, 0, NN * sizeof(double), st);
        cudaError_t e =
            cb.probe_ppt == 2
                ? launch_pdl(probe_partial_atomic_kernel<2>, dim3((NN / 2 + kT - 1) / kT, cb.chunks), st, cs)
                : launch_pdl(probe_partial_atomic_kernel<1>, dim3((NN + kT - 1) / kT, cb.chunks), st, cs);
        if (e == cudaSuccess)
            e = launch_pdl(max_double_kernel, dim3((NN + kT - 1) / kT < 304 ? (NN + kT - 1) / kT : 304), st,
                           (const double*)cb.denP, (size_t)NN, cb.maxP);
        if (e == cudaSuccess)
            e = launch_pdl(slice_sums_kernel, dim3(n_slice), st, (const double*)cs.e_part, cs.n_part,
                           cb.e_slice);
        if (e == cudaSuccess) e = launch_pdl(probe_normalise_kernel, dim3((NN + kT - 1) / kT), st, cs, n_slice);
        return e;
    }
    {
        cudaError_t e = launch_probe_partial(cs, st);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cb.chunks > kManyChunks ? launch_pdl(probe_reduce_kernel<8>, dim3(n_slice), st, cs)
                                            : launch_pdl(probe_reduce_kernel<1>, dim3(n_slice), st, cs);
    if (e != cudaSuccess) return e;
    e = launch_pdl(probe_normalise_kernel, dim3((NN + kT - 1) / kT), st, cs, n_slice);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

void ragged_concur_tables(const ConcurScan* scans, int n, std::vector<int>& first,
                          std::vector<int>& n_slice, int totals[5]) {
    first.assign(5 * (size_t)(n + 1), 0);
    n_slice.assign((size_t)n, 0);
    for (int s = 0; s < n; ++s) {
        const ConcurScan& cs = scans[s];
        const int NN = cs.N * cs.N;
        const size_t M = (size_t)cs.Mr * cs.Mc;
        n_slice[s] = probe_reduce_blocks(cs.N, cs.cb.chunks);
        const int blocks[5] = {cs.cb.tiles_r * cs.cb.tiles_c, (int)((M + kT - 1) / kT),
                               ((NN / cs.cb.probe_ppt + kT - 1) / kT) * cs.cb.chunks, n_slice[s],
                               (NN + kT - 1) / kT};
        for (int k = 0; k < 5; ++k)
            first[(size_t)k * (n + 1) + s + 1] = first[(size_t)k * (n + 1) + s] + blocks[k];
    }
    for (int k = 0; k < 5; ++k) totals[k] = first[(size_t)k * (n + 1) + n];
}

cudaError_t launch_concur_ragged(const RaggedConcur& rc, cudaStream_t st) {
    const int n = rc.n;
    const int* f = rc.first;
    switch (rc.gather_shape) {
        case 0: ragged_gather_kernel<16, 32><<<rc.totals[0], kT, 0, st>>>(rc.scans, f, n); break;
        case 1: ragged_gather_kernel<8, 32><<<rc.totals[0], kT, 0, st>>>(rc.scans, f, n); break;
        case 2: ragged_gather_kernel<32, 32><<<rc.totals[0], kT, 0, st>>>(rc.scans, f, n); break;
        case 3: ragged_gather_kernel<8, 64><<<rc.totals[0], kT, 0, st>>>(rc.scans, f, n); break;
        default: return cudaErrorInvalidValue;
    }
    ragged_onorm_kernel<<<rc.totals[1], kT, 0, st>>>(rc.scans, f + (n + 1), n);
    if (rc.probe_ppt == 2)
        ragged_ppart_kernel<2><<<rc.totals[2], kT, 0, st>>>(rc.scans, f + 2 * (n + 1), n);
    else
        ragged_ppart_kernel<1><<<rc.totals[2], kT, 0, st>>>(rc.scans, f + 2 * (n + 1), n);
    ragged_preduce_kernel<<<rc.totals[3], kT, 0, st>>>(rc.scans, f + 3 * (n + 1), n);
    ragged_pnorm_kernel<<<rc.totals[4], kT, 0, st>>>(rc.scans, f + 4 * (n + 1), rc.n_slice, n);
    return cudaGetLastError();
}

// Many partials are summed in two levels (fixed slices, then the slice
// totals in order) so the single final block has little to add.
constexpr int kSliceBlocks = 256;

cudaError_t launch_record_error(const double* parts, int n, double scale, double* ring,
                                unsigned long long* d_iter, int cap, double* scratch,
                                cudaStream_t st) {
    if (n > 16 * kT) {
        slice_sums_kernel<<<kSliceBlocks, kT, 0, st>>>(parts, n, scratch);
        record_error_kernel<<<1, kT, 0, st>>>(scratch, kSliceBlocks, scale, ring, d_iter, cap);
    } else {
        record_error_kernel<<<1, kT, 0, st>>>(parts, n, scale, ring, d_iter, cap);
    }
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
                             double* scratch, cudaStream_t st) {
    if (n > 16 * kT) {
        slice_sums_kernel<<<kSliceBlocks, kT, 0, st>>>(parts, n, scratch);
        sum_parts_kernel<<<1, kT, 0, st>>>(scratch, kSliceBlocks, scale, out);
    } else {
        sum_parts_kernel<<<1, kT, 0, st>>>(parts, n, scale, out);
    }
    return cudaGetLastError();
}

}  // namespace ptycho
