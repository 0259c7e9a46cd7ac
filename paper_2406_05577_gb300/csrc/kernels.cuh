// kernels.cuh -- the staged, pruned sphere <-> cube kernels (Fig. 3: pad one
// dimension, transform it, then the next).
//
//   k_stick  (z stage)  G -> r: gather each occupied (x,y) stick's sphere
//            entries into a zero-padded length-N2 column and run its z-DFT;
//            write the stick buffer T[band][z][s].
//            r -> G: z-DFT of each stick of T, then scatter the sphere
//            entries back to the coefficient list (pruned output).
//   k_plane  (y and x stages) one CTA per (band, z) plane.
//            G -> r: place the plane's S stick values into the occupied
//            x-slab columns A[y][xi], y-DFT each of the X columns, then
//            zero-extend each row to N0 and x-DFT it; write the cube plane.
//            r -> G: x-DFT each cube row keeping only the X occupied outputs,
//            y-DFT the X columns, keep the S occupied sticks.
//            apply: G -> r of the plane, multiply by V(r) (Sec. 2.3 fusion of
//            pad, FFT and a pointwise product), r -> G; the cube never
//            reaches global memory.
//
// The processor-grid all-to-alls of the paper's distributed version (Sec.
// 3.1, 4.1) become the stick -> plane regrouping through T and the
// shared-memory transposes inside k_plane.
#pragma once

#include "fft_core.cuh"
#include "fftb_internal.h"

namespace fftb {

template <typename T> struct Cfg;
template <> struct Cfg<float> { static constexpr int NT = 256, EPT = 16; };
template <> struct Cfg<double> { static constexpr int NT = 256, EPT = 8; };

template <typename T, int N> __host__ __device__ constexpr int line_cap() {
  return (Cfg<T>::NT * Cfg<T>::EPT) / N;
}
template <typename T, int N2> __host__ __device__ constexpr int stick_tile_c() {
  return line_cap<T, N2>() > 128 ? 128 : line_cap<T, N2>();
}
template <typename T, int N0, int N1> __host__ __device__ constexpr int row_chunk_c() {
  return line_cap<T, N0>() > N1 ? N1 : line_cap<T, N0>();
}

template <typename T, int N2> constexpr size_t stick_smem_c() {
  using C = typename cplx<T>::type;
  return sizeof(C) * ((size_t)N2 * odd_pitch(stick_tile_c<T, N2>()) + N2);
}
template <typename T, int N0, int N1> size_t plane_smem_c(int xmax) {
  using C = typename cplx<T>::type;
  const int xp = odd_pitch(xmax > 0 ? xmax : 1);
  return sizeof(C) * ((size_t)N1 * xp + (size_t)N0 * odd_pitch(row_chunk_c<T, N0, N1>()) + N0 + N1) +
         sizeof(int) * N0;
}

// ------------------------------------------------------------------ z stage
template <typename T, int N2, int MODE>
__global__ void __launch_bounds__(Cfg<T>::NT) k_stick(const Launch L) {
  using C = typename cplx<T>::type;
  constexpr int NT = Cfg<T>::NT, EPT = Cfg<T>::EPT;
  constexpr int TS = stick_tile_c<T, N2>();
  constexpr int TSP = odd_pitch(TS);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw = buf + N2 * TSP;

  const int bl = blockIdx.y;
  const int gb = L.band0 + bl;
  const int k = L.g.band_k[gb];
  const KInfo ki = L.g.kinfo[k];
  const int s0 = blockIdx.x * TS;
  if (s0 >= ki.S) return;
  const int ns = min(TS, ki.S - s0);

  const C* tw_g = static_cast<const C*>(L.g.tw2);
  for (int m = threadIdx.x; m < N2; m += NT) tw[m] = tw_g[m];
  C* Tb = static_cast<C*>(L.T) + (size_t)bl * N2 * L.g.smax + s0;
  const int smax = L.g.smax;
  const int32_t* sent = L.g.stick_ent + ki.stick_base + k;
  const int e0 = sent[s0], e1 = sent[s0 + ns];
  const int64_t sph = L.g.band_sph[gb];

  auto mid_ld = [&](int line, int e) -> C { return buf[e * TSP + line]; };
  auto mid_st = [&](int line, int e, C v) { buf[e * TSP + line] = v; };

  if constexpr (MODE == M_G2R) {
    const C* in = static_cast<const C*>(L.sph_in) + sph;
    for (int m = threadIdx.x; m < N2 * TSP; m += NT) buf[m] = czero<C>();
    __syncthreads();
    for (int e = e0 + threadIdx.x; e < e1; e += NT) {
      const uint32_t zs = (uint32_t)L.g.ent_zs[e];
      buf[(int)(zs >> 24) * TSP + ((int)(zs & 0xFFFFFFu) - s0)] = in[L.g.ent_pos[e]];
    }
    __syncthreads();
    auto last = [&](int line, int e, C v) { Tb[(size_t)e * smax + line] = v; };
    fft_lines<N2, +1, NT, EPT, false, C>(ns, tw, mid_ld, mid_ld, mid_st, last);
  } else {
    __syncthreads();
    auto first = [&](int line, int e) -> C { return Tb[(size_t)e * smax + line]; };
    fft_lines<N2, -1, NT, EPT, false, C>(ns, tw, first, mid_ld, mid_st, mid_st);
    C* out = static_cast<C*>(L.sph_out) + sph;
    for (int e = e0 + threadIdx.x; e < e1; e += NT) {
      const uint32_t zs = (uint32_t)L.g.ent_zs[e];
      out[L.g.ent_pos[e]] = buf[(int)(zs >> 24) * TSP + ((int)(zs & 0xFFFFFFu) - s0)];
    }
  }
}

// ------------------------------------------------------------- y, x stages
template <typename T, int N0, int N1, int MODE>
__global__ void __launch_bounds__(Cfg<T>::NT) k_plane(const Launch L) {
  using C = typename cplx<T>::type;
  constexpr int NT = Cfg<T>::NT, EPT = Cfg<T>::EPT;
  constexpr int LCY = line_cap<T, N1>();          // y-DFT columns per pass set
  constexpr int YC = row_chunk_c<T, N0, N1>();    // x-DFT rows per pass set
  constexpr int YCP = odd_pitch(YC);
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int z = blockIdx.x;
  const int bl = blockIdx.y;
  const int gb = L.band0 + bl;
  const int n2 = L.g.n2;
  const int k = L.g.band_k[gb];
  const KInfo ki = L.g.kinfo[k];
  const int X = ki.X, S = ki.S;
  const int XP = odd_pitch(X > 0 ? X : 1);

  C* A = reinterpret_cast<C*>(smem_raw);
  C* B = A + N1 * XP;
  C* tw0 = B + N0 * YCP;
  C* tw1 = tw0 + N0;
  int* xm = reinterpret_cast<int*>(tw1 + N1);
  {
    const C* t0 = static_cast<const C*>(L.g.tw0);
    const C* t1 = static_cast<const C*>(L.g.tw1);
    for (int m = threadIdx.x; m < N0; m += NT) {
      tw0[m] = t0[m];
      xm[m] = L.g.xmap[ki.xmap_base + m];
    }
    for (int m = threadIdx.x; m < N1; m += NT) tw1[m] = t1[m];
  }
  C* Tz = static_cast<C*>(L.T) + ((size_t)bl * n2 + z) * L.g.smax;
  const int32_t* sxy = L.g.stick_xy + ki.stick_base;
  const size_t plane = ((size_t)gb * n2 + z) * (size_t)(N1 * N0);

  auto b_ld = [&](int line, int e) -> C { return B[e * YCP + line]; };
  auto b_st = [&](int line, int e, C v) { B[e * YCP + line] = v; };

  if constexpr (MODE == M_G2R || MODE == M_APPLY) {
    for (int m = threadIdx.x; m < N1 * XP; m += NT) A[m] = czero<C>();
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += NT) {
      const int xy = sxy[s];
      A[(xy & 0xFFFF) * XP + (xy >> 16)] = Tz[s];
    }
    __syncthreads();
    // y-DFT (+) of each occupied x-slab column
    for (int c0 = 0; c0 < X; c0 += LCY) {
      const int nl = min(LCY, X - c0);
      auto a_ld = [&](int line, int e) -> C { return A[e * XP + c0 + line]; };
      auto a_st = [&](int line, int e, C v) { A[e * XP + c0 + line] = v; };
      fft_lines<N1, +1, NT, EPT, false, C>(nl, tw1, a_ld, a_ld, a_st, a_st);
    }
    // x-DFT (+) of every row, zero-extended from the X occupied columns
    for (int y0 = 0; y0 < N1; y0 += YC) {
      const int nl = min(YC, N1 - y0);
      auto first = [&](int line, int x) -> C {
        const int xi = xm[x];
        return xi >= 0 ? A[(y0 + line) * XP + xi] : czero<C>();
      };
      if constexpr (MODE == M_G2R) {
        C* out = static_cast<C*>(L.cube_out) + plane + (size_t)y0 * N0;
        auto last = [&](int line, int x, C v) { out[line * N0 + x] = v; };
        fft_lines<N0, +1, NT, EPT, true, C>(nl, tw0, first, b_ld, b_st, last);
      } else {
        const T* V = static_cast<const T*>(L.V) + (size_t)z * (N1 * N0) + (size_t)y0 * N0;
        auto last = [&](int line, int x, C v) { B[x * YCP + line] = scale(v, V[line * N0 + x]); };
        fft_lines<N0, +1, NT, EPT, true, C>(nl, tw0, first, b_ld, b_st, last);
        auto back = [&](int line, int x, C v) {
          const int xi = xm[x];
          if (xi >= 0) A[(y0 + line) * XP + xi] = v;
        };
        fft_lines<N0, -1, NT, EPT, true, C>(nl, tw0, b_ld, b_ld, b_st, back);
      }
    }
  }
  if constexpr (MODE == M_R2G) {
    __syncthreads();
    for (int y0 = 0; y0 < N1; y0 += YC) {
      const int nl = min(YC, N1 - y0);
      const C* in = static_cast<const C*>(L.cube_in) + plane + (size_t)y0 * N0;
      auto first = [&](int line, int x) -> C { return in[line * N0 + x]; };
      auto last = [&](int line, int x, C v) {
        const int xi = xm[x];
        if (xi >= 0) A[(y0 + line) * XP + xi] = v;
      };
      fft_lines<N0, -1, NT, EPT, true, C>(nl, tw0, first, b_ld, b_st, last);
    }
  }
  if constexpr (MODE == M_R2G || MODE == M_APPLY) {
    // y-DFT (-) of each occupied column, then keep the occupied sticks
    for (int c0 = 0; c0 < X; c0 += LCY) {
      const int nl = min(LCY, X - c0);
      auto a_ld = [&](int line, int e) -> C { return A[e * XP + c0 + line]; };
      auto a_st = [&](int line, int e, C v) { A[e * XP + c0 + line] = v; };
      fft_lines<N1, -1, NT, EPT, false, C>(nl, tw1, a_ld, a_ld, a_st, a_st);
    }
    for (int s = threadIdx.x; s < S; s += NT) {
      const int xy = sxy[s];
      Tz[s] = A[(xy & 0xFFFF) * XP + (xy >> 16)];
    }
  }
}

// ---------------------------------------------------------------- dispatch
#define FFTB_SIZES(X) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(96) X(128) X(160)

template <typename T> size_t stick_smem_t(int n2) {
  switch (n2) {
#define C_(N) case N: return stick_smem_c<T, N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}
template <typename T> size_t plane_smem_t(int n0, int n1, int xmax) {
  if (n0 != n1) return 0;
  switch (n0) {
#define C_(N) case N: return plane_smem_c<T, N, N>(xmax);
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}
template <typename T> int stick_tile_t(int n2) {
  switch (n2) {
#define C_(N) case N: return stick_tile_c<T, N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}

template <typename T, int N2> cudaError_t go_stick(int mode, const Launch& L, int tiles) {
  const size_t smem = stick_smem_c<T, N2>();
  const dim3 grid(tiles, L.nb);
  if (mode == M_G2R) k_stick<T, N2, M_G2R><<<grid, Cfg<T>::NT, smem, L.stream>>>(L);
  else k_stick<T, N2, M_R2G><<<grid, Cfg<T>::NT, smem, L.stream>>>(L);
  return cudaGetLastError();
}
template <typename T, int N> cudaError_t go_plane(int mode, const Launch& L) {
  const size_t smem = plane_smem_c<T, N, N>(L.g.xmax);
  const dim3 grid(L.g.n2, L.nb);
  if (mode == M_G2R) k_plane<T, N, N, M_G2R><<<grid, Cfg<T>::NT, smem, L.stream>>>(L);
  else if (mode == M_R2G) k_plane<T, N, N, M_R2G><<<grid, Cfg<T>::NT, smem, L.stream>>>(L);
  else k_plane<T, N, N, M_APPLY><<<grid, Cfg<T>::NT, smem, L.stream>>>(L);
  return cudaGetLastError();
}
template <typename T, int N2> cudaError_t prep_stick() {
  const int s = (int)stick_smem_c<T, N2>();
  cudaError_t e = cudaFuncSetAttribute(k_stick<T, N2, M_G2R>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_stick<T, N2, M_R2G>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  return e;
}
template <typename T, int N> cudaError_t prep_plane(int xmax) {
  const int s = (int)plane_smem_c<T, N, N>(xmax);
  cudaError_t e = cudaFuncSetAttribute(k_plane<T, N, N, M_G2R>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane<T, N, N, M_R2G>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_plane<T, N, N, M_APPLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  return e;
}

template <typename T> cudaError_t launch_stick_t(int mode, const Launch& L, int tiles) {
  switch (L.g.n2) {
#define C_(N) case N: return go_stick<T, N>(mode, L, tiles);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}
template <typename T> cudaError_t launch_plane_t(int mode, const Launch& L) {
  if (L.g.n0 != L.g.n1) return cudaErrorInvalidValue;
  switch (L.g.n0) {
#define C_(N) case N: return go_plane<T, N>(mode, L);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}
template <typename T> cudaError_t prepare_t(int n0, int n1, int n2, int xmax) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (n2) {
#define C_(N) case N: e = prep_stick<T, N>(); break;
    FFTB_SIZES(C_)
#undef C_
  }
  if (e != cudaSuccess || n0 != n1) return e == cudaSuccess ? cudaErrorInvalidValue : e;
  switch (n0) {
#define C_(N) case N: return prep_plane<T, N>(xmax);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

#define FFTB_INSTANTIATE(T)                                                        \
  template size_t stick_smem_t<T>(int);                                            \
  template size_t plane_smem_t<T>(int, int, int);                                  \
  template int stick_tile_t<T>(int);                                               \
  template cudaError_t launch_stick_t<T>(int, const Launch&, int);                 \
  template cudaError_t launch_plane_t<T>(int, const Launch&);                      \
  template cudaError_t prepare_t<T>(int, int, int, int);

}  // namespace fftb
