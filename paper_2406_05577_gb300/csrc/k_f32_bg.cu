// k_f32_bg.cu -- float y and x stages for batch-fastest plans (Sec. 3.3, the
// batch dimension declared first): a CTA takes BG bands of one k-point at
// one z together, so the cube row I/O of the x stage is band-contiguous.
//
// In the batch-fastest cube, point (z, y, x) of band b_local is element
// ((z N1 + y) N0 + x) B_k + b_local: the bands of one point are adjacent and
// one band's consecutive x are B_k elements apart. A CTA that handles one
// (band, z) plane therefore moves one 8-byte element per 32-byte sector.
// Here a CTA handles a group of BG bands of the same k-point at one z: the
// y stage fills BG slab planes (one per band) in shared memory, and in the x
// stage a warp's lines are BG bands x (lines / BG) rows with the band index
// fastest across the line groups, so the lanes that hold one x of one row
// for the BG bands touch BG adjacent elements (a full sector for BG = 4).
//
// Groups never straddle a k-point; the plan lists them (first band, count)
// and launches whole groups per band chunk. Slab planes are single-buffered
// (a block barrier ends each phase); no prefetch, no tensor cores. The
// arithmetic per line is the band-major kernel's, so both give the same
// results bit for bit.
#include "kernels.cuh"

namespace fftb {
namespace {

// warps per CTA and resident CTAs per SM the register allocation allows
#ifndef FFTB_BG_NW
#define FFTB_BG_NW 8
#endif
constexpr int BG_NW = FFTB_BG_NW;
template <int N> __host__ __device__ constexpr int bg_minb() {
#ifdef FFTB_BG_MINB
  return FFTB_BG_MINB;
#else
  return plane_minb<float, N>();
#endif
}

// lines per warp of the length-N engine (both plane lengths are N)
template <int N> __host__ __device__ constexpr int bg_wx() { return 32 / Line<N>::G; }

// Elements from one band's slab plane to the next: N rows of a_pitch(xmax),
// rounded up to 8 past a multiple of 16, so that the lanes of two bands that
// read one x-task position (a half warp of 8-byte accesses) fall on the two
// halves of the banks.
__host__ __device__ constexpr int bg_abuf(int n, int xmax) {
  return n * a_pitch(xmax) + ((8 - (n * a_pitch(xmax)) % 16) + 16) % 16;
}

template <int N, int BG> size_t bg_smem(int xmax) {
  constexpr int SCR = bg_wx<N>() * Line<N>::PITCH;
  return sizeof(float2) * ((size_t)BG * bg_abuf(N, xmax) + (size_t)BG_NW * SCR + N);
}

// QP: every k-point's sticks lie within a quarter of the grid per axis
// (KF_XY_QUARTER for all of the plan's k-points): the middle half of every y
// and x line is dropped at compile time, as in the band-major kernels.
template <int N, int MODE, int BG, bool QP = false>
__global__ void __launch_bounds__(BG_NW * 32, (bg_minb<N>())) k_plane_bg(const Launch L) {
  using C = float2;
  using LN = Line<N>;
  constexpr int NW = BG_NW, NT = NW * 32;
  constexpr int W = bg_wx<N>(), E = LN::E;
  constexpr int RPT = W / BG;  // rows per x task
  static_assert(W % BG == 0, "a warp's lines must hold whole band groups");
  constexpr int SCR = W * LN::PITCH;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int n2 = L.g.n2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane % LN::G, l = lane / LN::G;
  const int abuf = bg_abuf(N, L.g.xmax);
  C* A0 = reinterpret_cast<C*>(smem_raw);
  C* scr = A0 + BG * abuf + warp * SCR;
  C* tw = A0 + BG * abuf + NW * SCR;
  {
    const C* t0 = static_cast<const C*>(L.g.tw0);  // N0 == N1: one table serves both stages
    for (int m = threadIdx.x; m < N; m += NT) tw[m] = t0[m];
  }
  pdl_launch_dependents();
  __syncthreads();
  pdl_wait();
  C* lrow = scr + l * LN::PITCH;
  typename LN::template TwCache<C> tc;
  tc.load(g, tw);
  auto ysigned = [](int y) { return y < N - N / 2 ? y : y - N; };
  // x task line: band j of the group, row r of the task
  const int xj = l % BG, xr = l / BG;

  const int nunits = L.ngrp * n2;
  int cur_k = -1;
  XiPack<E> xin, xout;
#pragma unroll 1
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int gi = u / n2, z = u - gi * n2;
    const int2 gr = L.groups[L.grp0 + gi];  // first band (plan-global), bands in the group
    const BandInfo bi = L.g.band[gr.x];
    const KInfo ki = bi.ki;
    const int X = ki.X, XP = a_pitch(X), cst = ki.bstride, cnt = gr.y;
    if (ki.xmap_base != cur_k) {  // a new k-point (uniform across the CTA)
      cur_k = ki.xmap_base;
      const int16_t* xm = L.g.xmap + ki.xmap_base;
#pragma unroll
      for (int q = 0; q < (E + 3) / 4; ++q) { xin.w[q] = 0; xout.w[q] = 0; }
#pragma unroll
      for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
        for (int j = 0; j < LN::R0; ++j) {
          const int q = m * LN::R0 + j, xi = xm[LN::first_pos(g, m, j)];
          xin.w[q >> 2] |= (uint32_t)(xi < 0 ? 255 : xi) << (8 * (q & 3));
        }
#pragma unroll
      for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
        for (int j = 0; j < LN::RL; ++j) {
          const int q = m * LN::RL + j, xi = xm[LN::last_pos(g, m, j)];
          xout.w[q >> 2] |= (uint32_t)(xi < 0 ? 255 : xi) << (8 * (q & 3));
        }
    }
    const int4* __restrict__ cinfo = L.g.col_info + ki.col_base;
    const int32_t* sxy = L.g.stick_xy + ki.stick_base;
    const int bl0 = gr.x - L.band0;  // the group's first band within this launch's chunk
    // cube element of (first band of the group, z, 0, 0)
    const size_t plane = (size_t)bi.cube + (size_t)z * (size_t)(N * N) * (size_t)cst;
    const int ty = (X + W - 1) / W;  // y tasks per band
    const int tx = (N + RPT - 1) / RPT;  // x tasks, each RPT rows of the BG bands

    // y stage of band j, column task ct: G -> r (sign +) from the stick row into A_j,
    // r -> G (sign -) from A_j into the stick row
    auto y_task = [&](int j, int ct) {
      C* A = A0 + j * abuf;
      C* Tz = static_cast<C*>(L.T) + ((size_t)(bl0 + j) * n2 + z) * L.g.smax;
      const int c0 = ct * W, nl = min(W, X - c0);
      const int col = c0 + (l < nl ? l : 0);
      const int4 ci = cinfo[col];  // first stick, sticks, signed gy of the first
      C v[E];
      if constexpr (MODE == M_G2R) {
        if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j2 = 0; j2 < LN::R0; ++j2) {
              if (QP && x_mid<N, LN::G, LN::R0>(m * LN::R0 + j2)) {  // no occupied y there
                v[m * LN::R0 + j2] = czero<C>();
                continue;
              }
              const int d = ysigned(LN::first_pos(g, m, j2)) - ylo;
              v[m * LN::R0 + j2] = (unsigned)d < (unsigned)len ? Tz[sa + d] : czero<C>();
            }
        } else {
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LN::G);
          for (int q = lane; q < W * LN::PITCH; q += 32) scr[q] = czero<C>();
          __syncwarp();
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            scr[((xy >> 16) - c0) * LN::PITCH + wpad(xy & 0xFFFF)] = Tz[s];
          }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j2 = 0; j2 < LN::R0; ++j2)
              v[m * LN::R0 + j2] = QP && x_mid<N, LN::G, LN::R0>(m * LN::R0 + j2) ? czero<C>()  // no stick there
                                                                                 : lrow[wpad(LN::first_pos(g, m, j2))];
          __syncwarp();
        }
        LN::template run<+1>(v, g, lrow, tw, tc);
        if (l < nl) {
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j2 = 0; j2 < LN::RL; ++j2) A[LN::last_pos(g, m, j2) * XP + c0 + l] = v[m * LN::RL + j2];
        }
      } else {
#pragma unroll
        for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
          for (int j2 = 0; j2 < LN::R0; ++j2) v[m * LN::R0 + j2] = A[LN::first_pos(g, m, j2) * XP + col];
        LN::template run<-1>(v, g, lrow, tw, tc);
        if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          if (l < nl) {
            const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
            for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
              for (int j2 = 0; j2 < LN::RL; ++j2) {
                if (QP && x_mid<N, LN::G, LN::RL>(m * LN::RL + j2)) continue;  // no occupied y there
                const int d = ysigned(LN::last_pos(g, m, j2)) - ylo;
                if ((unsigned)d < (unsigned)len) Tz[sa + d] = v[m * LN::RL + j2];
              }
          }
        } else {
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j2 = 0; j2 < LN::RL; ++j2) {
              if (QP && x_mid<N, LN::G, LN::RL>(m * LN::RL + j2)) continue;  // no stick there
              lrow[wpad(LN::last_pos(g, m, j2))] = v[m * LN::RL + j2];
            }
          __syncwarp();
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LN::G);
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            Tz[s] = scr[((xy >> 16) - c0) * LN::PITCH + wpad(xy & 0xFFFF)];
          }
          __syncwarp();
        }
      }
    };

    if constexpr (MODE == M_G2R) {
#pragma unroll 1
      for (int t = warp; t < cnt * ty; t += NW) y_task(t / ty, t - (t / ty) * ty);
      __syncthreads();
      // x-DFT (+) of every row of the BG slab planes, zero-extended from the X occupied columns
#pragma unroll 1
      for (int t = warp; t < tx; t += NW) {
        const int row = t * RPT + xr;
        const bool live = row < N && xj < cnt;
        const C* A = A0 + xj * abuf + (live ? row : 0) * XP;
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
          if (QP && x_mid<N, LN::G, LN::R0>(q)) {  // no occupied x there
            v[q] = czero<C>();
            continue;
          }
          const int xi = xin.get(q);
          v[q] = (live && xi != 255) ? A[xi] : czero<C>();
        }
        LN::template run<+1>(v, g, lrow, tw, tc);
        if (live) {
          C* out = static_cast<C*>(L.cube_out) + plane + (size_t)row * N * cst + xj;
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j2 = 0; j2 < LN::RL; ++j2) out[(size_t)LN::last_pos(g, m, j2) * cst] = v[m * LN::RL + j2];
        }
      }
      __syncthreads();
    } else {
      // x-DFT (-) of every row, kept at the X occupied columns of A_j
#pragma unroll 1
      for (int t = warp; t < tx; t += NW) {
        const int row = t * RPT + xr;
        const bool live = row < N && xj < cnt;
        const C* in = static_cast<const C*>(L.cube_in) + plane + (size_t)(live ? row : 0) * N * cst + xj;
        C v[E];
#pragma unroll
        for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
          for (int j2 = 0; j2 < LN::R0; ++j2)
            v[m * LN::R0 + j2] = live ? in[(size_t)LN::first_pos(g, m, j2) * cst] : czero<C>();
        LN::template run<-1>(v, g, lrow, tw, tc);
        if (live) {
          C* A = A0 + xj * abuf + row * XP;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            if (QP && x_mid<N, LN::G, LN::RL>(q)) continue;  // no occupied x there
            const int xi = xout.get(q);
            if (xi != 255) A[xi] = v[q];
          }
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int t = warp; t < cnt * ty; t += NW) y_task(t / ty, t - (t / ty) * ty);
      __syncthreads();
    }
  }
}

template <int N> constexpr bool bg_qp() { return N == 64 || N == 96 || N == 128; }
template <int N, int BG, bool QP = false> const void* bg_fn(int mode) {
  return mode == M_G2R ? (const void*)k_plane_bg<N, M_G2R, BG, QP> : (const void*)k_plane_bg<N, M_R2G, BG, QP>;
}
template <int N, int BG, bool QP = false> cudaError_t go_bg(int mode, const Launch& L) {
  if constexpr (!QP && bg_qp<N>()) {
    if (L.xq) return go_bg<N, BG, true>(mode, L);
  }
  const size_t smem = bg_smem<N, BG>(L.g.xmax);
  const int units = L.ngrp * L.g.n2;
  const dim3 grid(L.plane_ctas > 0 ? min(L.plane_ctas, units) : units);
  constexpr int NT = BG_NW * 32;
  if (mode == M_G2R) return launch_k(k_plane_bg<N, M_G2R, BG, QP>, grid, NT, smem, L, L);
  return launch_k(k_plane_bg<N, M_R2G, BG, QP>, grid, NT, smem, L, L);
}

template <int N> cudaError_t prep_bg(int xmax);
template <int N> int occ_bg(int mode, int xmax);

// the band group of each length: 4 (a full 32-byte sector of FP32 complex) up
// to 96 points, 2 above, where four slab planes no longer fit shared memory
template <int N> __host__ __device__ constexpr int bg_of() { return (N <= 96 && bg_wx<N>() % 4 == 0) ? 4 : 2; }

#define FFTB_BG_SIZES(X) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(96) X(128) X(160) X(256)

template <int N> cudaError_t prep_bg(int xmax) {
  const int s = (int)bg_smem<N, bg_of<N>()>(xmax);
  cudaError_t e = raise_smem_limit(bg_fn<N, bg_of<N>()>(M_G2R), s);
  if (e == cudaSuccess) e = raise_smem_limit(bg_fn<N, bg_of<N>()>(M_R2G), s);
  if constexpr (bg_qp<N>()) {
    if (e == cudaSuccess) e = raise_smem_limit(bg_fn<N, bg_of<N>(), true>(M_G2R), s);
    if (e == cudaSuccess) e = raise_smem_limit(bg_fn<N, bg_of<N>(), true>(M_R2G), s);
  }
  return e;
}
// resident CTAs per SM, the line-pruned variant included (the plan sizes one grid for both)
template <int N> int occ_bg(int mode, int xmax) {
  const size_t s = bg_smem<N, bg_of<N>()>(xmax);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bg_fn<N, bg_of<N>()>(mode), BG_NW * 32, s) != cudaSuccess)
    return 0;
  if constexpr (bg_qp<N>()) {
    int nq = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nq, bg_fn<N, bg_of<N>(), true>(mode), BG_NW * 32, s) !=
        cudaSuccess)
      return 0;
    nb = nb < nq ? nb : nq;
  }
  return nb;
}

}  // namespace

int plane_bg_group(int n) {
  switch (n) {
#define C_(N) case N: return bg_of<N>();
    FFTB_BG_SIZES(C_)
#undef C_
  }
  return 0;
}

size_t plane_bg_smem(int n0, int n1, int xmax, int bg) {
  if (n0 != n1 || bg != plane_bg_group(n0)) return 0;
  switch (n0) {
#define C_(N) case N: return bg_smem<N, bg_of<N>()>(xmax);
    FFTB_BG_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t prepare_plane_bg(int n, int xmax) {
  switch (n) {
#define C_(N) case N: return prep_bg<N>(xmax);
    FFTB_BG_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

int plane_bg_occupancy(int mode, int n, int xmax) {
  switch (n) {
#define C_(N) case N: return occ_bg<N>(mode, xmax);
    FFTB_BG_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t launch_plane_bg(int mode, const Launch& L) {
  if (mode != M_G2R && mode != M_R2G) return cudaErrorInvalidValue;
  switch (L.g.n0) {
#define C_(N) case N: return go_bg<N, bg_of<N>()>(mode, L);
    FFTB_BG_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
