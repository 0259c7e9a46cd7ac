// k_f32_zq.cu -- float z-stage kernels for launches whose sphere entries all
// have |z| <= N2/4 (KF_Z_QUARTER; cutoff spheres of the cube-width-twice-
// the-diameter rule): the middle half of every z line is dropped at compile
// time (k_stick with QZ). The 160-point lines run the two-pass 40 x 4
// schedule (one exchange, 8 sticks a warp, one CTA per SM; measured at
// 160^3 with one persistent wave: G->r 2.67 -> 2.29, r->G 2.90 -> 1.97 us per
// band against the default 4 x 4 x 2 x 5), the others their default schedule.
#include "kernels.cuh"

namespace fftb {
namespace {

template <int N2> constexpr int VZ = N2 == 160 ? 2 : 0;
template <int N2, int MODE> const void* zq_fn() { return (const void*)k_stick<float, N2, MODE, false, VZ<N2>, true>; }

template <int N2> cudaError_t go_zq(int mode, const Launch& L, int ctas) {
  using LZ = Line<N2, VZ<N2>>;
  const size_t smem = stick_smem_c<float, N2, VZ<N2>>();
  const int gpb = (L.g.smax + (32 / LZ::G) - 1) / (32 / LZ::G);
  const int need = (L.nb * gpb + STICK_NW - 1) / STICK_NW;  // one task per warp
  const dim3 grid(ctas > 0 ? min(ctas, need) : need);
  if (mode == M_G2R) return launch_k(k_stick<float, N2, M_G2R, false, VZ<N2>, true>, grid, STICK_NW * 32, smem, L, L);
  return launch_k(k_stick<float, N2, M_R2G, false, VZ<N2>, true>, grid, STICK_NW * 32, smem, L, L);
}
template <int N2> cudaError_t prep_zq() {
  const int s = (int)stick_smem_c<float, N2, VZ<N2>>();
  cudaError_t e = raise_smem_limit(zq_fn<N2, M_G2R>(), s);
  return e == cudaSuccess ? raise_smem_limit(zq_fn<N2, M_R2G>(), s) : e;
}
// resident CTAs per SM of both directions' kernels
template <int N2> int occ_zq() {
  const size_t s = stick_smem_c<float, N2, VZ<N2>>();
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_stick<float, N2, M_G2R, false, VZ<N2>, true>, STICK_NW * 32, s) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_stick<float, N2, M_R2G, false, VZ<N2>, true>, STICK_NW * 32, s) !=
          cudaSuccess)
    return 0;
  return a < b ? a : b;
}

}  // namespace

int stick_zq_occupancy(int n2) {
  switch (n2) {
#define C_(N) case N: return occ_zq<N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}

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
