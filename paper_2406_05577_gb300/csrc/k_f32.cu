// k_f32.cu -- float instantiations of the stick and plane kernels.
#include "kernels.cuh"

namespace fftb {
FFTB_INSTANTIATE(float, false)
}  // namespace fftb
