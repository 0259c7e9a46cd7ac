// k_tc.cu -- MIXED_TC instantiations: float storage and arithmetic, radix-8
// passes on the tensor cores in split FP16 precision.
#include "kernels.cuh"

namespace fftb {
FFTB_INSTANTIATE(float, true)
}  // namespace fftb
