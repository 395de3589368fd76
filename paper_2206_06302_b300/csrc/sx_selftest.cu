// sx_selftest.cu -- self-test of the device-side failure path (sx_target_selftest).
//
// Kernels of this library never trap: a device-side wait that runs out records a code in the
// target's device error word and returns, and the host reports SX_ERR_DEVICE at its next
// synchronisation.  This kernel exercises that path on demand.
#include "sx_device.cuh"
#include "sx_internal.h"

namespace sx {
namespace {

constexpr int kSelfTestCode = 0x201;

// Waits, bounded by %globaltimer, on err[1], which nothing writes; on expiry records
// kSelfTestCode in err[0] and returns.  The loop reads the flag with volatile loads and always
// ends.
__global__ void k_selftest_wait(int *err, uint64_t limit_ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    volatile int *flag = err + 1;
    const uint64_t t0 = dev::global_ns();
    while (*flag == 0) {
        if (dev::global_ns() - t0 > limit_ns) {
            atomicExch(err, kSelfTestCode);
            return;
        }
    }
}

}  // namespace

int launch_selftest(const sx_target *t, cudaStream_t s, int64_t limit_us) {
    k_selftest_wait<<<1, 32, 0, s>>>(t->d_err, (uint64_t)limit_us * 1000ull);
    SX_CUDA(cudaGetLastError());
    return SX_OK;
}

}  // namespace sx
