// k_f64.cu -- double instantiations of the stick and plane kernels.
#include "kernels.cuh"

namespace fftb {
FFTB_INSTANTIATE(double, false)
}  // namespace fftb
