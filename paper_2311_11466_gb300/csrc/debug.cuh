// Checked build of the library (compiled with -DPTYCHO_DEBUG into
// libptycho_debug.so).  Device-side checks of object-window bounds, of the
// sqrt(I) input and of non-finite outputs record what they saw in a flag word
// of their translation unit and go on with a safe value (a clamped window, a
// skipped entry) instead of trapping, so a failed check never faults or hangs
// the device and a kernel whose CTAs meet at a barrier still meets there.
// ptycho_debug_flags() reads and clears the words.  In the normal build the
// checks compile to nothing and the flags read as 0.
#pragma once

#include <cuda_runtime.h>

namespace ptycho {

enum : unsigned {
    kDbgWindow = 1u,      // an object window outside the object
    kDbgNonFinite = 2u,   // a NaN or Inf written to y, the object or the probe
    kDbgSqrtI = 4u,       // a negative or non-finite sqrt(I) read by the divide step
};

}  // namespace ptycho

#ifdef PTYCHO_DEBUG
// One flag word per translation unit (no relocatable device code needed) and
// its host accessor ptycho::debug_flags_<name>(), which reads and clears it on
// the current device.
#define PTYCHO_DEBUG_UNIT(name)                                                          \
    namespace ptycho {                                                                   \
    static __device__ unsigned g_debug_flags;                                            \
    cudaError_t debug_flags_##name(unsigned* out) {                                      \
        unsigned zero = 0u;                                                              \
        cudaError_t e = cudaMemcpyFromSymbol(out, g_debug_flags, sizeof(unsigned));      \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_debug_flags, &zero, sizeof(zero)); \
        return e;                                                                        \
    }                                                                                    \
    }
#define PT_DBG_FLAG(bit) atomicOr(&::ptycho::g_debug_flags, (unsigned)(bit))
#define PT_DBG_ENABLED 1
#else
#define PTYCHO_DEBUG_UNIT(name)                                                          \
    namespace ptycho {                                                                   \
    cudaError_t debug_flags_##name(unsigned* out) {                                      \
        *out = 0u;                                                                       \
        return cudaSuccess;                                                              \
    }                                                                                    \
    }
#define PT_DBG_FLAG(bit) ((void)0)
#define PT_DBG_ENABLED 0
#endif

// v has a NaN or Inf component (for the output checks).
#define PT_DBG_NONFINITE2(v) (!isfinite((v).x) || !isfinite((v).y))
