// k_generic.cu -- the staged pruned transform for grid extents outside the
// compiled list, N0 != N1 included: every extent whose prime factors are
// 2, 3 and 5 (up to 512; N2 up to 256, the entry records hold z in 8 bits).
//
// The same stages as the compiled kernels (Fig. 3: pad one dimension, run its
// 1D DFTs, then the next), one kernel per axis and direction:
//   z  G -> r: sphere entries of each occupied stick -> zero-padded z line ->
//              z-DFT -> stick buffer T[band][z][stick]
//   y  G -> r: the sticks of each occupied x-slab (from T) -> zero-padded y
//              line -> y-DFT -> slab buffer S[band][z][slab][y]
//   x  G -> r: each (z, y) row gathered from S at the occupied x values ->
//              zero-padded x line -> x-DFT -> cube row
// and the reverse with outputs pruned to the occupied slabs and sticks; the
// fused apply runs x-DFT (+), V(r) * psi(r), x-DFT (-) on each row in one
// kernel, so the cube never reaches global memory. The line lengths are
// runtime values: a CTA holds a group of lines in shared memory and runs
// Stockham passes over them (radices chosen on the host from 8, 4, 2, 3, 5;
// Sec. 2.1 factorisation), ping-ponging between two line buffers.
#include "kernels.cuh"

namespace fftb {
namespace {

constexpr int GEN_NT = 256;

// One Stockham pass of runtime radix R over nl lines of length n (line l at
// src + l * pitch), written to dst: butterfly i of a line takes the inputs
// i + j n/R, twiddles them by w^{j k} (k = i mod L, L = the radices before
// this pass), and stores its outputs at (i - k) R + k + j L.
template <int R, int S, typename C>
__device__ __forceinline__ void gen_pass(const C* src, C* dst, int nl, int n, int pitch, int L, const C* tw) {
  const int nb = n / R;
  const int step = n / (L * R);
  for (int w = threadIdx.x; w < nl * nb; w += GEN_NT) {
    const int line = w / nb, i = w - line * nb, k = i % L;
    C v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = src[line * pitch + i + j * nb];
    if (L > 1) {
#pragma unroll
      for (int j = 1; j < R; ++j) {
        const C t = tw[j * k * step];
        v[j] = S > 0 ? cmul(v[j], t) : cmulc(v[j], t);
      }
    }
    dft<R, S>(v);
    const int base = (i - k) * R + k;
#pragma unroll
    for (int j = 0; j < R; ++j) dst[line * pitch + base + j * L] = v[j];
  }
}

// All passes of a length-n DFT (sign S) of nl lines in a; returns the buffer
// holding the result (a or b). Every thread of the CTA must call it.
template <int S, typename C>
__device__ C* gen_fft(C* a, C* b, int nl, int n, int pitch, const GenAxis& ax, const C* tw) {
  int L = 1;
  for (int p = 0; p < ax.np; ++p) {
    const int R = ax.r[p];
    switch (R) {
      case 2: gen_pass<2, S>(a, b, nl, n, pitch, L, tw); break;
      case 3: gen_pass<3, S>(a, b, nl, n, pitch, L, tw); break;
      case 4: gen_pass<4, S>(a, b, nl, n, pitch, L, tw); break;
      case 5: gen_pass<5, S>(a, b, nl, n, pitch, L, tw); break;
      default: gen_pass<8, S>(a, b, nl, n, pitch, L, tw); break;
    }
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    L *= R;
  }
  return a;
}

enum { GEN_Z = 0, GEN_Y = 1, GEN_X = 2, GEN_XAPPLY = 3 };

template <typename T, int STAGE, int S>
__global__ void __launch_bounds__(GEN_NT) k_gen(const Launch L, const GenParams P) {
  using C = typename cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int AX = STAGE == GEN_Z ? 2 : STAGE == GEN_Y ? 1 : 0;
  const GenAxis& ax = P.ax[AX];
  const int n = ax.n, lpc = P.lpc, pitch = P.pitch;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* b0 = tw + n;
  C* b1 = b0 + (size_t)lpc * pitch;
  {
    const C* src = static_cast<const C*>(AX == 2 ? L.g.tw2 : AX == 1 ? L.g.tw1 : L.g.tw0);
    for (int m = threadIdx.x; m < n; m += GEN_NT) tw[m] = src[m];
  }
  __syncthreads();
  const int n0 = L.g.n0, n1 = L.g.n1, n2 = L.g.n2, smax = L.g.smax, xmax = L.g.xmax;
  C* Sb = static_cast<C*>(P.S);
  C* Tb = static_cast<C*>(L.T);
  // line groups: sticks per band (z), slabs per (band, z) plane (y), rows per plane (x)
  const int per = STAGE == GEN_Z ? (smax + lpc - 1) / lpc : STAGE == GEN_Y ? (xmax + lpc - 1) / lpc
                                                                          : (n1 + lpc - 1) / lpc;
  const int64_t ntask = STAGE == GEN_Z ? (int64_t)L.nb * per : (int64_t)L.nb * n2 * per;
  for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
    const int grp = (int)(task % per);
    const int64_t rest = task / per;
    const int bl = STAGE == GEN_Z ? (int)rest : (int)(rest / n2);
    const int z = STAGE == GEN_Z ? 0 : (int)(rest % n2);
    const BandInfo bi = L.g.band[L.band0 + bl];
    const KInfo ki = bi.ki;
    const int first = grp * lpc;
    const int nl = STAGE == GEN_Z ? min(lpc, ki.S - first) : STAGE == GEN_Y ? min(lpc, ki.X - first)
                                                                           : min(lpc, n1 - first);
    if (nl <= 0) continue;  // uniform: dead group (a k-point with fewer sticks or slabs)
    const int st = ki.bstride;
    const size_t trow = ((size_t)bl * n2 + z) * smax;                // T row of (band, z)
    const size_t srow = ((size_t)bl * n2 + z) * xmax;                // S block of (band, z), in lines of n1
    // ---- inputs, zero-padded
    // G -> r inputs are sparse (zero-padded lines); r -> G inputs are whole lines
    if (S > 0 || STAGE == GEN_XAPPLY)
      for (int q = threadIdx.x; q < nl * pitch; q += GEN_NT) b0[q] = czero<C>();
    __syncthreads();
    if constexpr (STAGE == GEN_Z) {
      const int4* si = L.g.stick_info + ki.stick_base;
      if constexpr (S > 0) {
        const int ea = si[first].x, eb = si[first + nl - 1].y;
        const C* in = static_cast<const C*>(L.sph_in);
        for (int e = ea + threadIdx.x; e < eb; e += GEN_NT) {
          const uint32_t zs = (uint32_t)L.g.ent_zs[e];
          const int64_t pos = bi.sph + (int64_t)L.g.ent_pos[e] * st;
          if (FFTB_IN(pos, L.lim_sph, L.status))
            b0[((int)(zs & 0xFFFFFFu) - first) * pitch + (int)(zs >> 24)] = in[pos];
        }
      } else {
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q % nl, zz = q / nl;
          const size_t idx = ((size_t)bl * n2 + zz) * smax + first + l;
          b0[l * pitch + zz] = FFTB_IN(idx, L.lim_T, L.status) ? Tb[idx] : czero<C>();
        }
      }
    } else if constexpr (STAGE == GEN_Y) {
      const int4* ci = L.g.col_info + ki.col_base;
      if constexpr (S > 0) {
        const int sa = ci[first].x, sb = ci[first + nl - 1].x + ci[first + nl - 1].y;
        for (int s = sa + threadIdx.x; s < sb; s += GEN_NT) {
          const int xy = L.g.stick_xy[ki.stick_base + s];
          if (FFTB_IN(trow + s, L.lim_T, L.status)) b0[((xy >> 16) - first) * pitch + (xy & 0xFFFF)] = Tb[trow + s];
        }
      } else {
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q / n, y = q - l * n;
          const size_t idx = (srow + first + l) * n1 + y;
          b0[l * pitch + y] = FFTB_IN(idx, P.lim_S, L.status) ? Sb[idx] : czero<C>();
        }
      }
    } else {
      const int16_t* xm = L.g.xmap + ki.xmap_base;
      if (S > 0 || STAGE == GEN_XAPPLY) {
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q % nl, x = q / nl;
          const int xi = xm[x];
          if (xi >= 0) {
            const size_t idx = (srow + xi) * n1 + first + l;
            if (FFTB_IN(idx, P.lim_S, L.status)) b0[l * pitch + x] = Sb[idx];
          }
        }
      } else {
        const C* in = static_cast<const C*>(L.cube_in);
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q / n, x = q - l * n;
          const int64_t idx = bi.cube + (((int64_t)z * n1 + first + l) * n0 + x) * st;
          if (FFTB_IN(idx, L.lim_cube, L.status)) b0[l * pitch + x] = in[idx];
        }
      }
    }
    __syncthreads();
    // ---- the line DFTs
    C* res = gen_fft<S>(b0, b1, nl, n, pitch, ax, tw);
    if constexpr (STAGE == GEN_XAPPLY) {
      // V(r) psi(r) on each row, then back (Sec. 2.3 fusion)
      const T* V = static_cast<const T*>(L.V);
      for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
        const int l = q / n, x = q - l * n;
        const int64_t vi = ((int64_t)z * n1 + first + l) * n0 + x;
        res[l * pitch + x] = scale(res[l * pitch + x], FFTB_IN(vi, L.lim_V, L.status) ? V[vi] : T(0));
      }
      __syncthreads();
      C* other = res == b0 ? b1 : b0;
      res = gen_fft<-1>(res, other, nl, n, pitch, ax, tw);
    }
    // ---- outputs, pruned for r -> G
    if constexpr (STAGE == GEN_Z) {
      if constexpr (S > 0) {
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q % nl, zz = q / nl;
          const size_t idx = ((size_t)bl * n2 + zz) * smax + first + l;
          if (FFTB_IN(idx, L.lim_T, L.status)) Tb[idx] = res[l * pitch + zz];
        }
      } else {
        const int4* si = L.g.stick_info + ki.stick_base;
        const int ea = si[first].x, eb = si[first + nl - 1].y;
        C* out = static_cast<C*>(L.sph_out);
        for (int e = ea + threadIdx.x; e < eb; e += GEN_NT) {
          const uint32_t zs = (uint32_t)L.g.ent_zs[e];
          const int64_t pos = bi.sph + (int64_t)L.g.ent_pos[e] * st;
          if (FFTB_IN(pos, L.lim_sph, L.status)) out[pos] = res[((int)(zs & 0xFFFFFFu) - first) * pitch + (int)(zs >> 24)];
        }
      }
    } else if constexpr (STAGE == GEN_Y) {
      if constexpr (S > 0) {
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q / n, y = q - l * n;
          const size_t idx = (srow + first + l) * n1 + y;
          if (FFTB_IN(idx, P.lim_S, L.status)) Sb[idx] = res[l * pitch + y];
        }
      } else {
        const int4* ci = L.g.col_info + ki.col_base;
        const int sa = ci[first].x, sb = ci[first + nl - 1].x + ci[first + nl - 1].y;
        for (int s = sa + threadIdx.x; s < sb; s += GEN_NT) {
          const int xy = L.g.stick_xy[ki.stick_base + s];
          if (FFTB_IN(trow + s, L.lim_T, L.status)) Tb[trow + s] = res[((xy >> 16) - first) * pitch + (xy & 0xFFFF)];
        }
      }
    } else {
      if (S > 0 && STAGE == GEN_X) {
        C* out = static_cast<C*>(L.cube_out);
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q / n, x = q - l * n;
          const int64_t idx = bi.cube + (((int64_t)z * n1 + first + l) * n0 + x) * st;
          if (FFTB_IN(idx, L.lim_cube, L.status)) out[idx] = res[l * pitch + x];
        }
      } else {
        const int16_t* xm = L.g.xmap + ki.xmap_base;
        for (int q = threadIdx.x; q < nl * n; q += GEN_NT) {
          const int l = q % nl, x = q / nl;
          const int xi = xm[x];
          if (xi >= 0) {
            const size_t idx = (srow + xi) * n1 + first + l;
            if (FFTB_IN(idx, P.lim_S, L.status)) Sb[idx] = res[l * pitch + x];
          }
        }
      }
    }
    __syncthreads();  // the line buffers are reused by the next group
  }
}

template <typename T, int STAGE, int S> cudaError_t go(const Launch& L, const GenParams& P, int ctas) {
  using C = typename cplx<T>::type;
  const int axis = STAGE == GEN_Z ? 2 : STAGE == GEN_Y ? 1 : 0;
  const size_t smem = sizeof(C) * ((size_t)P.ax[axis].n + 2 * (size_t)P.lpc * P.pitch);
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit((const void*)k_gen<T, STAGE, S>, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gen<T, STAGE, S><<<ctas, GEN_NT, smem, L.stream>>>(L, P);
  return cudaGetLastError();
}

template <typename T> cudaError_t go_t(int stage, int sign, const Launch& L, const GenParams& P, int ctas) {
  if (stage == GEN_Z) return sign > 0 ? go<T, GEN_Z, 1>(L, P, ctas) : go<T, GEN_Z, -1>(L, P, ctas);
  if (stage == GEN_Y) return sign > 0 ? go<T, GEN_Y, 1>(L, P, ctas) : go<T, GEN_Y, -1>(L, P, ctas);
  if (stage == GEN_X) return sign > 0 ? go<T, GEN_X, 1>(L, P, ctas) : go<T, GEN_X, -1>(L, P, ctas);
  return go<T, GEN_XAPPLY, 1>(L, P, ctas);
}

}  // namespace

cudaError_t launch_generic(bool fp64, int stage, int sign, const Launch& L, const GenParams& P, int ctas) {
  return fp64 ? go_t<double>(stage, sign, L, P, ctas) : go_t<float>(stage, sign, L, P, ctas);
}

}  // namespace fftb
