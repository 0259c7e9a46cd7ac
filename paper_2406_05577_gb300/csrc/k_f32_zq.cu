// k_f32_zq.cu -- float z-stage kernels for launches whose sphere entries all
// have |z| <= N2/4 (KF_Z_QUARTER; cutoff spheres of the cube-width-twice-
// the-diameter rule): the middle half of every z line is dropped at compile
// time (k_stick with QZ), default radix schedule.
#include "kernels.cuh"

namespace fftb {
namespace {

template <int N2, int MODE> const void* zq_fn() { return (const void*)k_stick<float, N2, MODE, false, 0, true>; }

template <int N2> cudaError_t go_zq(int mode, const Launch& L, int ctas) {
  const size_t smem = stick_smem_c<float, N2>();
  const int gpb = (L.g.smax + (32 / Line<N2>::G) - 1) / (32 / Line<N2>::G);
  const int need = (L.nb * gpb + STICK_NW - 1) / STICK_NW;  // one task per warp
  const dim3 grid(ctas > 0 ? min(ctas, need) : need);
  if (mode == M_G2R) return launch_k(k_stick<float, N2, M_G2R, false, 0, true>, grid, STICK_NW * 32, smem, L, L);
  return launch_k(k_stick<float, N2, M_R2G, false, 0, true>, grid, STICK_NW * 32, smem, L, L);
}
template <int N2> cudaError_t prep_zq() {
  const int s = (int)stick_smem_c<float, N2>();
  cudaError_t e = raise_smem_limit(zq_fn<N2, M_G2R>(), s);
  return e == cudaSuccess ? raise_smem_limit(zq_fn<N2, M_R2G>(), s) : e;
}

}  // namespace

cudaError_t prepare_stick_zq(int n2) {
  switch (n2) {
#define C_(N) case N: return prep_zq<N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_stick_zq(int mode, const Launch& L, int ctas) {
  switch (L.g.n2) {
#define C_(N) case N: return go_zq<N>(mode, L, ctas);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
