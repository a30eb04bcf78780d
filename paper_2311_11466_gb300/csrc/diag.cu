// Diagnostic for the library's failure handling (include/ptycho.h):
// every wait inside a kernel is bounded in time and reports its expiry to
// the host through a status word instead of hanging the device.  This entry
// point runs such a wait on a device flag that nothing ever sets, so the
// bound must fire; the host reads the status and returns PTYCHO_ETIMEOUT,
// and the context and device remain usable.
#include <cuda_runtime.h>

#include "../../include/ptycho.h"

namespace {

__global__ void bounded_wait_kernel(const volatile int* flag, unsigned long long timeout_ns,
                                    int* status) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (*flag == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > timeout_ns) {
            atomicOr(status, 1);
            return;
        }
        __nanosleep(1000);
    }
}

}  // namespace

extern "C" int ptycho_check_bounded_wait(int device, uint32_t timeout_ms) {
    if (timeout_ms == 0 || timeout_ms > 10000) return PTYCHO_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return PTYCHO_EINVAL;
    int* buf = nullptr;  // [0] the flag nobody sets, [1] the status
    int rc = PTYCHO_ECUDA;
    if (cudaMalloc(&buf, 2 * sizeof(int)) == cudaSuccess &&
        cudaMemset(buf, 0, 2 * sizeof(int)) == cudaSuccess) {
        bounded_wait_kernel<<<1, 1>>>(buf, (unsigned long long)timeout_ms * 1000000ull, buf + 1);
        int status = 0;
        if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
            cudaMemcpy(&status, buf + 1, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
            rc = status ? PTYCHO_ETIMEOUT : PTYCHO_OK;
    }
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    return rc;
}
