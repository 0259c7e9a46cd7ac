// k_f32_alt.cu -- float stick and plane kernels with the alternative radix
// schedule of the lengths that have one (LPV<N, 1>; the plane stages of 160
// take the two-pass schedule LPV<160, 2>); the autotuner chooses between them
// and the default schedule.
#include <algorithm>

#include "kernels.cuh"

namespace fftb {
namespace {

#define FFTB_ALT_SIZES(X) X(64) X(96) X(128) X(160)

// schedule variant of the alternative plane kernels (160: the two-pass
// schedule), and of their line-pruned versions for launches whose k-points
// all have every occupied stick within a quarter of the grid (160: variant 3;
// the others: the same schedule with QP)
template <int N> constexpr int plane_v() { return N == 160 ? 2 : 1; }
template <int N> constexpr int plane_vq() { return N == 160 ? 3 : plane_v<N>(); }
template <int N> constexpr bool plane_qp() { return N != 160; }

template <int N, int MODE, bool Q = false> const void* plane_fn() {
  if constexpr (Q) return (const void*)k_plane<float, N, N, MODE, false, false, false, plane_vq<N>(), plane_qp<N>()>;
  else return (const void*)k_plane<float, N, N, MODE, false, false, false, plane_v<N>()>;
}
template <int N, int MODE> const void* stick_fn() { return (const void*)k_stick<float, N, MODE, false, 1>; }

template <int N, int V, bool QP> cudaError_t go_plane_vv(int mode, const Launch& L) {
  const size_t smem = plane_smem_c<float, N, N, V>(L.g.xmax, L.a_bufs);
  const int nplanes = L.nb * L.g.n2;
  const dim3 grid(L.plane_ctas > 0 ? min(L.plane_ctas, nplanes) : nplanes);
  constexpr int NT = PlaneCfg<float>::NW * 32;
  if (mode == M_G2R) return launch_k(k_plane<float, N, N, M_G2R, false, false, false, V, QP>, grid, NT, smem, L, L);
  if (mode == M_R2G) return launch_k(k_plane<float, N, N, M_R2G, false, false, false, V, QP>, grid, NT, smem, L, L);
  return launch_k(k_plane<float, N, N, M_APPLY, false, false, false, V, QP>, grid, NT, smem, L, L);
}
template <int N> cudaError_t go_plane_v(int mode, const Launch& L) {
  if (L.xq) return go_plane_vv<N, plane_vq<N>(), plane_qp<N>()>(mode, L);
  return go_plane_vv<N, plane_v<N>(), false>(mode, L);
}
template <int N> cudaError_t go_stick_v(int mode, const Launch& L, int ctas) {
  constexpr int WZ = 32 / Line<N, 1>::G;
  const size_t smem = stick_smem_c<float, N, 1>();
  const int gpb = (L.g.smax + WZ - 1) / WZ;
  const int need = (L.nb * gpb + STICK_NW - 1) / STICK_NW;  // one task per warp
  const dim3 grid(ctas > 0 ? min(ctas, need) : need);
  if (mode == M_G2R) return launch_k(k_stick<float, N, M_G2R, false, 1>, grid, STICK_NW * 32, smem, L, L);
  return launch_k(k_stick<float, N, M_R2G, false, 1>, grid, STICK_NW * 32, smem, L, L);
}
template <int N> cudaError_t prep_plane_v(int xmax, int a_bufs) {
  const int s = (int)plane_smem_c<float, N, N, plane_v<N>()>(xmax, a_bufs);
  cudaError_t e = raise_smem_limit(plane_fn<N, M_G2R>(), s);
  if (e == cudaSuccess) e = raise_smem_limit(plane_fn<N, M_R2G>(), s);
  if (e == cudaSuccess) e = raise_smem_limit(plane_fn<N, M_APPLY>(), s);
  const int sq = (int)plane_smem_c<float, N, N, plane_vq<N>()>(xmax, a_bufs);
  if (e == cudaSuccess) e = raise_smem_limit(plane_fn<N, M_G2R, true>(), sq);
  if (e == cudaSuccess) e = raise_smem_limit(plane_fn<N, M_R2G, true>(), sq);
  if (e == cudaSuccess) e = raise_smem_limit(plane_fn<N, M_APPLY, true>(), sq);
  return e;
}
template <int N> cudaError_t prep_stick_v() {
  const int s = (int)stick_smem_c<float, N, 1>();
  cudaError_t e = raise_smem_limit(stick_fn<N, M_G2R>(), s);
  if (e == cudaSuccess) e = raise_smem_limit(stick_fn<N, M_R2G>(), s);
  return e;
}
template <int N> int occ_plane_v(int mode, int xmax, int a_bufs) {
  const size_t s = plane_smem_c<float, N, N, plane_v<N>()>(xmax, a_bufs);
  const void* fn = mode == M_G2R ? plane_fn<N, M_G2R>() : mode == M_R2G ? plane_fn<N, M_R2G>() : plane_fn<N, M_APPLY>();
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, PlaneCfg<float>::NW * 32, s) != cudaSuccess) return 0;
  {  // the line-pruned variant must be resident the same way
    const void* fq = mode == M_G2R   ? plane_fn<N, M_G2R, true>()
                     : mode == M_R2G ? plane_fn<N, M_R2G, true>()
                                     : plane_fn<N, M_APPLY, true>();
    int nq = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nq, fq, PlaneCfg<float>::NW * 32, s) != cudaSuccess) return 0;
    nb = std::min(nb, nq);
  }
  return nb;
}
template <int N> int occ_stick_v() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, stick_fn<N, M_G2R>(), STICK_NW * 32,
                                                       stick_smem_c<float, N, 1>()) == cudaSuccess
             ? nb
             : 0;
}

}  // namespace

bool alt_schedule(int n) {
  switch (n) {
#define C_(N) case N: return true;
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return false;
}

size_t plane_alt_smem(int n, int xmax, int a_bufs) {
  switch (n) {
#define C_(N) case N: return plane_smem_c<float, N, N, plane_v<N>()>(xmax, a_bufs);
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t prepare_alt(int n0, int n2, int xmax, int a_bufs) {
  cudaError_t e = cudaSuccess;
  switch (n0) {
#define C_(N) case N: e = prep_plane_v<N>(xmax, a_bufs); break;
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  if (e != cudaSuccess) return e;
  switch (n2) {
#define C_(N) case N: e = prep_stick_v<N>(); break;
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return e;
}

int plane_alt_occupancy(int mode, int n, int xmax, int a_bufs) {
  switch (n) {
#define C_(N) case N: return occ_plane_v<N>(mode, xmax, a_bufs);
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return 0;
}

int stick_alt_occupancy(int n) {
  switch (n) {
#define C_(N) case N: return occ_stick_v<N>();
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t launch_plane_alt(int mode, const Launch& L) {
  if (L.g.n0 != L.g.n1) return cudaErrorInvalidValue;
  switch (L.g.n0) {
#define C_(N) case N: return go_plane_v<N>(mode, L);
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_stick_alt(int mode, const Launch& L, int ctas) {
  switch (L.g.n2) {
#define C_(N) case N: return go_stick_v<N>(mode, L, ctas);
    FFTB_ALT_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
