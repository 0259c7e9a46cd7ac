// k_f32_pf.cu -- float plane kernels whose inputs arrive by bulk asynchronous
// copies (k_plane with PF), in a translation unit of their own.
#include "kernels.cuh"

namespace fftb {
namespace {
// the prefetch staging fits shared memory beside the slab planes up to 160;
// with the slab planes in global memory (AG) from 128 to 256
#define FFTB_PF_SIZES(X) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(96) X(128) X(160)
#define FFTB_PF_AG_SIZES(X) X(128) X(160) X(256)

template <int N, int MODE> constexpr bool pf_has() { return MODE != M_R2G || rows_prefetchable<float, N, N>(); }

template <int N, int MODE, bool AG, bool QP = false> auto pf_kernel() {
  return k_plane<float, N, N, MODE, false, AG, pf_has<N, MODE>(), 0, QP>;
}

template <int N, bool AG, bool QP = false> cudaError_t go(int mode, const Launch& L) {
  if constexpr (!QP && qp_variant<float, false, N>()) {
    if (L.xq) return go<N, AG, true>(mode, L);  // every sphere within a quarter of the grid
  }
  const size_t smem = plane_smem_c<float, N, N>(L.g.xmax, L.a_bufs, AG, mode, L.g.smax);
  const int nplanes = L.nb * L.g.n2;
  // AG: persistent CTAs only, never more than the slab-plane blocks allocated
  const int ctas = AG ? min(min(L.plane_ctas, nplanes), L.a_blocks) : (L.plane_ctas > 0 ? min(L.plane_ctas, nplanes) : nplanes);
  if (ctas < 1) return cudaErrorInvalidValue;
  const dim3 grid(ctas);
  constexpr int NT = PlaneCfg<float>::NW * 32;
  if (mode == M_G2R) return launch_k(pf_kernel<N, M_G2R, AG, QP>(), grid, NT, smem, L, L);
  if (mode == M_R2G) return launch_k(pf_kernel<N, M_R2G, AG, QP>(), grid, NT, smem, L, L);
  return launch_k(pf_kernel<N, M_APPLY, AG, QP>(), grid, NT, smem, L, L);
}
template <int N, bool AG, bool QP = false> cudaError_t prep(int mode, int xmax, int a_bufs, int tp) {
  if constexpr (!QP && qp_variant<float, false, N>()) {
    cudaError_t e = prep<N, AG, true>(mode, xmax, a_bufs, tp);
    if (e != cudaSuccess) return e;
  }
  const int s = (int)plane_smem_c<float, N, N>(xmax, a_bufs, AG, mode, tp);
  if (mode == M_G2R) return raise_smem_limit((const void*)pf_kernel<N, M_G2R, AG, QP>(), s);
  if (mode == M_R2G) return raise_smem_limit((const void*)pf_kernel<N, M_R2G, AG, QP>(), s);
  return raise_smem_limit((const void*)pf_kernel<N, M_APPLY, AG, QP>(), s);
}
template <int N, bool AG, bool QP = false> int occ(int mode, int xmax, int a_bufs, int tp) {
  constexpr int NT = PlaneCfg<float>::NW * 32;
  const size_t s = plane_smem_c<float, N, N>(xmax, a_bufs, AG, mode, tp);
  int nb = 0, nq = 1 << 30;  // the line-pruned variant must be resident the same way
  if constexpr (!QP && qp_variant<float, false, N>()) nq = occ<N, AG, true>(mode, xmax, a_bufs, tp);
  cudaError_t e;
  if (mode == M_G2R) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pf_kernel<N, M_G2R, AG, QP>(), NT, s);
  else if (mode == M_R2G) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pf_kernel<N, M_R2G, AG, QP>(), NT, s);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pf_kernel<N, M_APPLY, AG, QP>(), NT, s);
  return e == cudaSuccess ? min(nb, nq) : 0;
}

bool size_listed(int n, bool ag) {
  if (ag) {
    switch (n) {
#define C_(N) case N:
      FFTB_PF_AG_SIZES(C_)
#undef C_
      return true;
      default: return false;
    }
  }
  switch (n) {
#define C_(N) case N:
    FFTB_PF_SIZES(C_)
#undef C_
    return true;
    default: return false;
  }
}

}  // namespace

bool plane_pf_supported(int mode, int n0, int n1, bool ag) {
  if (n0 != n1 || !size_listed(n0, ag)) return false;
  switch (n0) {
#define C_(N) case N: return mode == M_G2R || mode == M_APPLY || (mode == M_R2G && rows_prefetchable<float, N, N>());
    FFTB_PF_SIZES(C_)
    case 256: return mode == M_G2R || mode == M_APPLY || (mode == M_R2G && rows_prefetchable<float, 256, 256>());
#undef C_
  }
  return false;
}
size_t plane_pf_smem(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag) {
  if (!plane_pf_supported(mode, n0, n1, ag)) return 0;
  if (ag) {
    switch (n0) {
#define C_(N) case N: return plane_smem_c<float, N, N>(xmax, a_bufs, true, mode, tp);
      FFTB_PF_AG_SIZES(C_)
#undef C_
    }
    return 0;
  }
  switch (n0) {
#define C_(N) case N: return plane_smem_c<float, N, N>(xmax, a_bufs, false, mode, tp);
    FFTB_PF_SIZES(C_)
#undef C_
  }
  return 0;
}
cudaError_t prepare_plane_pf(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag) {
  if (!plane_pf_supported(mode, n0, n1, ag)) return cudaErrorInvalidValue;
  if (ag) {
    switch (n0) {
#define C_(N) case N: return prep<N, true>(mode, xmax, a_bufs, tp);
      FFTB_PF_AG_SIZES(C_)
#undef C_
    }
    return cudaErrorInvalidValue;
  }
  switch (n0) {
#define C_(N) case N: return prep<N, false>(mode, xmax, a_bufs, tp);
    FFTB_PF_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}
int plane_pf_occupancy(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag) {
  if (!plane_pf_supported(mode, n0, n1, ag)) return 0;
  if (ag) {
    switch (n0) {
#define C_(N) case N: return occ<N, true>(mode, xmax, a_bufs, tp);
      FFTB_PF_AG_SIZES(C_)
#undef C_
    }
    return 0;
  }
  switch (n0) {
#define C_(N) case N: return occ<N, false>(mode, xmax, a_bufs, tp);
    FFTB_PF_SIZES(C_)
#undef C_
  }
  return 0;
}
cudaError_t launch_plane_pf(int mode, const Launch& L) {
  if (L.g.n0 != L.g.n1) return cudaErrorInvalidValue;
  if (L.a_glob) {
    switch (L.g.n0) {
#define C_(N) case N: return go<N, true>(mode, L);
      FFTB_PF_AG_SIZES(C_)
#undef C_
    }
    return cudaErrorInvalidValue;
  }
  switch (L.g.n0) {
#define C_(N) case N: return go<N, false>(mode, L);
    FFTB_PF_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
