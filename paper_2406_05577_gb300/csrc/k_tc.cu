// k_tc.cu -- MIXED_TC instantiations: float storage and arithmetic, radix-8
// passes on the tensor cores in split FP16 precision.
#include "kernels.cuh"

namespace fftb {
FFTB_INSTANTIATE(float, true)

namespace {
template <int N> constexpr bool has_tc_pass() {
  using L = Line<N>;
  bool r = false;
  for (int p = 0; p < L::NP; ++p) r = r || (LP<N>::R[p] == 8 && L::G > 1);
  return r;
}
}  // namespace

// The length's line schedule has a radix-8 pass the tensor cores take
// (run_tc); without one a MIXED_TC stage of that length is FP32 arithmetic.
bool tc_pass_in_schedule(int n) {
  switch (n) {
#define C_(N) case N: return has_tc_pass<N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return false;
}
}  // namespace fftb
