// tc_common.cuh -- small device helpers shared by the tensor-core
// contraction kernels (tc.cu, tc64.cu): packed spectral offsets, the device
// error word and the bounded mbarrier wait.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.cuh"

namespace sht {
namespace tcc {

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s

// Records the first error code of a launch (0 = none).
__device__ __forceinline__ void raise_err(int *err, int code)
{
    if (err) atomicCAS(err, 0, code);
}

// Bounded wait that also gives up when another thread of the CTA gave up.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    const uint64_t t0 = tc::globaltimer();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u) {
            if (*abort) return false;
            if (tc::globaltimer() - t0 > kWaitNs) {
                *abort = 1;
                return false;
            }
        }
    }
    *abort = 1;
    return false;
}

}  // namespace tcc
}  // namespace sht
