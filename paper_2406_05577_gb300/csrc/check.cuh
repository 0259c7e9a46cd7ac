// check.cuh -- device bounds checks of the checked build (FFTB_CHECK).
//
// Built with -DFFTB_CHECK (build.build(check=True) makes libfftb_check.so),
// the stick and plane kernels test every global index they compute -- sphere
// entries, stick rows, cube points, the potential -- and every slab-plane
// index against the extent of its buffer before the access. An index outside
// sets the STATUS_BOUNDS bit of the plan's status word and the access is
// skipped (a load reads zero), so fftb_plan_check reports
// FFTB_ERR_DEVICE_BOUNDS instead of a fault. Without FFTB_CHECK every check
// is the constant true and costs nothing.
#pragma once

#include <stdint.h>

namespace fftb {

// Device status bit (plan status word): a checked build found an index
// outside its buffer.
constexpr int STATUS_BOUNDS = 2;

#ifdef FFTB_CHECK
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t n, int32_t* status) {
  if ((uint64_t)i < (uint64_t)n) return true;
  atomicOr(status, STATUS_BOUNDS);
  return false;
}
#define FFTB_IN(i, n, status) (::fftb::in_bounds((int64_t)(i), (int64_t)(n), (status)))
#else
#define FFTB_IN(i, n, status) true
#endif

}  // namespace fftb
