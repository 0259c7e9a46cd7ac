// k_cluster.cu -- FP32 y and x stages of 256-point planes with the slab plane
// split across a cluster of two CTAs (distributed shared memory).
//
// A 256 x X slab plane (X up to about 150 occupied x-slabs) does not fit in
// one CTA's shared memory; the single-CTA kernels then keep it in a per-CTA
// block of global memory, whose L2 misses add DRAM traffic beyond the cube.
// Here the CTAs of a cluster (two, on two SMs) work on the same (band, z)
// plane and each holds part of its rows: rank r holds y in [r H, r H + H),
// H = N / (CTAs per cluster).
//   y phase: the y lines (occupied columns) are dealt over the warps of both
//            CTAs; a line's outputs go to the rank that holds their row, into
//            the partner's shared memory for the other half (st.shared::cluster).
//   x phase: each CTA transforms its own rows from its own half.
// r -> G splits the plane by columns instead: rank r holds every row of its
// half of the occupied columns (the y lines it transforms); the x phase
// sends each row's outputs to the rank that owns their column. Every remote
// access is then a store, which the issuing warp does not wait for (the
// fused apply, whose x phase needs whole rows and whose y phase whole
// columns, keeps the row split and reads the other half by remote loads).
// Cluster barriers (barrier.cluster arrive/wait) order the phases: after the
// y writes (before the x phase reads rows), after the x writes of r -> G and
// apply (before the y phase reads columns), and, split in an arrive after a
// CTA's last slab-plane read of a plane and a wait before its first write of
// the next, around the reuse of the halves. Every thread runs the same
// sequence of arrivals and waits, in the same plane loop (both ranks of a
// cluster walk the same planes), and the kernel ends with a wait, so no CTA
// leaves while its partner may still write into its shared memory.
#include <algorithm>

#include "kernels.cuh"

namespace fftb {
namespace {

// CTAs per cluster and warps per CTA (16 warps: one CTA per SM). Clusters
// of four CTAs of 8 warps (two CTAs per SM, a quarter plane each) measured
// slower in every direction; both build with -DFFTB_CL_CS / -DFFTB_CL_NW.
#ifndef FFTB_CL_CS
#define FFTB_CL_CS 2
#endif
#ifndef FFTB_CL_NW
#define FFTB_CL_NW 16
#endif
constexpr int CL_CS = FFTB_CL_CS, CL_NW = FFTB_CL_NW;
static_assert(CL_CS == 2 || CL_CS == 4, "clusters of two or four CTAs");

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_count() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}
// shared-memory address of the same location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float2 cl_ld(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
// cluster barrier halves (per thread: every thread of both CTAs arrives once per phase)
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

template <int N> __host__ __device__ constexpr int cl_scratch() { return (32 / Line<N>::G) * Line<N>::PITCH; }
// r -> G: the columns of each rank (rank q takes y tasks [q t, q t + t),
// t = the y tasks of x occupied columns over the ranks, rounded up)
template <int N> __host__ __device__ constexpr int cl_col_split(int x) {
  return (((x + 32 / Line<N>::G - 1) / (32 / Line<N>::G) + CL_CS - 1) / CL_CS) * (32 / Line<N>::G);
}
// elements of one CTA's part of the plane: rows [r N/CS, (r + 1) N/CS) of
// every column, or (r -> G) every row of its columns
template <int N> __host__ __device__ constexpr int cl_half(int mode, int xmax) {
  return mode == M_R2G ? N * a_pitch(cl_col_split<N>(xmax)) : (N / CL_CS) * a_pitch(xmax);
}
// shared memory: half slab plane, warp scratch rows, twiddles
template <int N> size_t cl_smem_c(int mode, int xmax) {
  return sizeof(float2) * ((size_t)cl_half<N>(mode, xmax) + (size_t)CL_NW * cl_scratch<N>() + N);
}

template <int N, int MODE>
__global__ void __launch_bounds__(CL_NW * 32, 16 / CL_NW) k_plane_cl(const Launch L) {
  using C = float2;
  using LN = Line<N>;
  constexpr int NW = CL_NW, NT = NW * 32, CS = CL_CS, H = N / CS;
  constexpr int W = 32 / LN::G, E = LN::E, SCR = cl_scratch<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int n2 = L.g.n2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane % LN::G, li = lane / LN::G;
  const uint32_t rank = cl_rank();
  const int abuf = cl_half<N>(MODE, L.g.xmax);
  C* A = reinterpret_cast<C*>(smem_raw);  // rows [rank H, rank H + H) of the plane
  C* scr = A + abuf + warp * SCR;
  C* tw = A + abuf + NW * SCR;
  C* row = scr + li * LN::PITCH;
  const uint32_t a_own = smem_u32(A);
  const uint32_t a_pair = cl_map(a_own, rank ^ 1u);  // the partner's (clusters of two)
  // shared::cluster address of element o of rank own's part
  auto a_addr = [&](uint32_t own, int o) {
    return (CS == 2 ? a_pair : cl_map(a_own, own)) + (uint32_t)o * (uint32_t)sizeof(C);
  };
  {
    const C* t0 = static_cast<const C*>(L.g.tw0);  // N0 == N1: one table serves y and x
    for (int m = threadIdx.x; m < N; m += NT) tw[m] = t0[m];
  }
  pdl_launch_dependents();
  __syncthreads();
  // the partner has started (its shared memory exists) before any remote access
  cl_arrive();
  cl_wait();
  pdl_wait();
  typename LN::template TwCache<C> tc;
  tc.load(g, tw);
  auto ysigned = [](int y) { return y < N - N / 2 ? y : y - N; };

  // element (y, c) of the plane: in this CTA's rows, or in those of rank y / H
  auto a_put = [&](int y, int c, int XP, C v) {
    const uint32_t own = (uint32_t)(y / H);
    const int o = (y - (int)own * H) * XP + c;
    if (!FFTB_IN(o, abuf, L.status)) return;
    if (own == rank) A[o] = v;
    else cl_st(a_addr(own, o), v);
  };
  auto a_get = [&](int y, int c, int XP) -> C {
    const uint32_t own = (uint32_t)(y / H);
    const int o = (y - (int)own * H) * XP + c;
    if (!FFTB_IN(o, abuf, L.status)) return czero<C>();
    return own == rank ? A[o] : cl_ld(a_addr(own, o));
  };

  const int nplanes = L.nb * n2;
  const int cw = (int)rank * NW + warp;  // this warp among the cluster's CS NW
  bool pending = false;                   // arrived for the halves' release, not yet waited
  auto a_acquire = [&]() {                // before this thread's first slab-plane write of a plane
    if (pending) {
      cl_wait();
      pending = false;
    }
  };
  int cur_k = -1;
  XiPack<E> xin, xout;
#pragma unroll 1
  for (int p = (int)cl_id(); p < nplanes; p += (int)cl_count()) {
    const int bl = p / n2;
    const int z = p - bl * n2;
    const BandInfo bi = L.g.band[L.band0 + bl];
    const KInfo ki = bi.ki;
    const int X = ki.X;
    const int cst = ki.bstride;
    const int cs = cl_col_split<N>(X);  // r -> G: columns of each rank
    const int XP = MODE == M_R2G ? a_pitch(cs) : a_pitch(X);
    const bool allx = X >= N;
    if (ki.xmap_base != cur_k) {
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
    const size_t tz = ((size_t)bl * n2 + z) * L.g.smax;
    C* Tz = static_cast<C*>(L.T) + tz;
    const size_t plane = (size_t)bi.cube + (size_t)z * (size_t)(N * N) * (size_t)cst;
    const int ty = (X + W - 1) / W;  // y tasks (over the cluster)
    constexpr int TX = H / W;        // x tasks of this CTA's rows

    if constexpr (MODE == M_G2R || MODE == M_APPLY) {
#pragma unroll 1
      for (int t = cw; t < ty; t += CS * NW) {
        const int c0 = t * W, nl = min(W, X - c0);
        C v[E];
        const int col = c0 + (li < nl ? li : 0);
        const int4 ci = cinfo[col];
        if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j = 0; j < LN::R0; ++j) {
              const int d = ysigned(LN::first_pos(g, m, j)) - ylo;
              v[m * LN::R0 + j] =
                  (unsigned)d < (unsigned)len && FFTB_IN(tz + sa + d, L.lim_T, L.status) ? Tz[sa + d] : czero<C>();
            }
        } else {
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LN::G);
          for (int q = lane; q < SCR; q += 32) scr[q] = czero<C>();
          __syncwarp();
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            if (FFTB_IN(tz + s, L.lim_T, L.status)) scr[((xy >> 16) - c0) * LN::PITCH + wpad(xy & 0xFFFF)] = Tz[s];
          }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j = 0; j < LN::R0; ++j) v[m * LN::R0 + j] = row[wpad(LN::first_pos(g, m, j))];
          __syncwarp();
        }
        LN::template run<+1>(v, g, row, tw, tc);
        a_acquire();
        if (li < nl) {
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j = 0; j < LN::RL; ++j) a_put(LN::last_pos(g, m, j), c0 + li, XP, v[m * LN::RL + j]);
        }
      }
      // every y output written (both halves) before the rows are read
      a_acquire();
      cl_arrive();
      cl_wait();
#pragma unroll 1
      for (int t = warp; t < TX; t += NW) {
        const int lr = t * W + li;           // row within this CTA's half
        const int y = H * (int)rank + lr;    // row of the plane
        C v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int xi = xin.get(q);
          v[q] = ((allx || xi != 255) && FFTB_IN(lr * XP + xi, abuf, L.status)) ? A[lr * XP + xi] : czero<C>();
        }
        LN::template run<+1>(v, g, row, tw, tc);
        if constexpr (MODE == M_G2R) {
          C* out = static_cast<C*>(L.cube_out) + plane + (size_t)y * N * cst;
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j = 0; j < LN::RL; ++j)
              if (FFTB_IN(plane + ((size_t)y * N + LN::last_pos(g, m, j)) * cst, L.lim_cube, L.status))
                out[(size_t)LN::last_pos(g, m, j) * cst] = v[m * LN::RL + j];
        } else {
          const float* vr = static_cast<const float*>(L.V) + (size_t)z * (N * N) + (size_t)y * N;
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j = 0; j < LN::RL; ++j) {
              const int x = LN::last_pos(g, m, j);
              const bool vin = FFTB_IN((size_t)z * (N * N) + (size_t)y * N + x, L.lim_V, L.status);
              row[wpad(x)] = scale(v[m * LN::RL + j], vin ? __ldg(vr + x) : 0.f);
            }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j = 0; j < LN::R0; ++j) v[m * LN::R0 + j] = row[wpad(LN::first_pos(g, m, j))];
          __syncwarp();
          LN::template run<-1>(v, g, row, tw, tc);
#pragma unroll
          for (int q = 0; q < E; ++q) {
            const int xi = xout.get(q);
            if ((allx || xi != 255) && FFTB_IN(lr * XP + xi, abuf, L.status)) A[lr * XP + xi] = v[q];
          }
        }
      }
    }
    if constexpr (MODE == M_R2G) {
#pragma unroll 1
      for (int t = warp; t < TX; t += NW) {
        const int lr = t * W + li;
        const int y = H * (int)rank + lr;
        const C* in = static_cast<const C*>(L.cube_in) + plane + (size_t)y * N * cst;
        C v[E];
#pragma unroll
        for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
          for (int j = 0; j < LN::R0; ++j)
            v[m * LN::R0 + j] = FFTB_IN(plane + ((size_t)y * N + LN::first_pos(g, m, j)) * cst, L.lim_cube, L.status)
                                    ? in[(size_t)LN::first_pos(g, m, j) * cst]
                                    : czero<C>();
        LN::template run<-1>(v, g, row, tw, tc);
        a_acquire();
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int xi = xout.get(q);
          if (allx || xi != 255) {
            uint32_t own = 0;  // the rank that holds column xi
#pragma unroll
            for (int k = 1; k < CS; ++k) own += xi >= k * cs ? 1u : 0u;
            const int o = y * XP + xi - (int)own * cs;
            if (FFTB_IN(o, abuf, L.status)) {
              if (own == rank) A[o] = v[q];
              else cl_st(a_addr(own, o), v[q]);
            }
          }
        }
      }
      a_acquire();
    }
    if constexpr (MODE == M_R2G || MODE == M_APPLY) {
      // every row written (both halves) before the columns are read
      cl_arrive();
      cl_wait();
      // r -> G: this rank's y tasks, its own columns; apply: tasks over the cluster
      const int th = cs / W;  // y tasks of each rank (r -> G)
      const int t_first = MODE == M_R2G ? (int)rank * th + warp : cw;
      const int t_end = MODE == M_R2G ? min((int)rank * th + th, ty) : ty;
      const int t_step = MODE == M_R2G ? NW : CS * NW;
#pragma unroll 1
      for (int t = t_first; t < t_end; t += t_step) {
        const int c0 = t * W, nl = min(W, X - c0);
        const int col = c0 + (li < nl ? li : 0);
        const int4 ci = cinfo[col];
        C v[E];
        if constexpr (MODE == M_R2G) {
          const int lc = col - (int)rank * cs;
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j = 0; j < LN::R0; ++j) {
              const int o = LN::first_pos(g, m, j) * XP + lc;
              v[m * LN::R0 + j] = FFTB_IN(o, abuf, L.status) ? A[o] : czero<C>();
            }
        } else {
#pragma unroll
          for (int m = 0; m < E / LN::R0; ++m)
#pragma unroll
            for (int j = 0; j < LN::R0; ++j) v[m * LN::R0 + j] = a_get(LN::first_pos(g, m, j), col, XP);
        }
        LN::template run<-1>(v, g, row, tw, tc);
        if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          if (li < nl) {
            const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
            for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
              for (int j = 0; j < LN::RL; ++j) {
                const int d = ysigned(LN::last_pos(g, m, j)) - ylo;
                if ((unsigned)d < (unsigned)len && FFTB_IN(tz + sa + d, L.lim_T, L.status)) Tz[sa + d] = v[m * LN::RL + j];
              }
          }
        } else {
#pragma unroll
          for (int m = 0; m < E / LN::RL; ++m)
#pragma unroll
            for (int j = 0; j < LN::RL; ++j) row[wpad(LN::last_pos(g, m, j))] = v[m * LN::RL + j];
          __syncwarp();
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LN::G);
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            if (FFTB_IN(tz + s, L.lim_T, L.status)) Tz[s] = scr[((xy >> 16) - c0) * LN::PITCH + wpad(xy & 0xFFFF)];
          }
          __syncwarp();
        }
      }
    }
    // this thread's last slab-plane read of the plane is done: release the halves
    cl_arrive();
    pending = true;
  }
  // no CTA leaves while its partner may still access its shared memory
  if (pending) cl_wait();
}

template <int MODE> const void* cl_fn(int n) {
  switch (n) {
    case 256: return (const void*)k_plane_cl<256, MODE>;
  }
  return nullptr;
}

}  // namespace

// largest over the three modes (mode 0), or of one mode
size_t plane_cluster_smem(int n0, int n1, int xmax, int mode) {
  if (n0 != n1) return 0;
  switch (n0) {
    case 256:
      return mode ? cl_smem_c<256>(mode, xmax)
                  : std::max(cl_smem_c<256>(M_G2R, xmax), cl_smem_c<256>(M_R2G, xmax));
  }
  return 0;
}

cudaError_t prepare_plane_cluster(int n, int xmax) {
  for (int mode : {M_G2R, M_R2G, M_APPLY}) {
    const size_t s = plane_cluster_smem(n, n, xmax, mode);
    const void* fn = mode == M_G2R ? cl_fn<M_G2R>(n) : mode == M_R2G ? cl_fn<M_R2G>(n) : cl_fn<M_APPLY>(n);
    if (s == 0 || !fn) return cudaErrorInvalidValue;
    cudaError_t e = raise_smem_limit(fn, (int)s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// clusters that can be resident at once (0: none), and their CTAs
int plane_cluster_size() { return CL_CS; }
int plane_cluster_count(int mode, int n, int xmax) {
  const size_t s = plane_cluster_smem(n, n, xmax, mode);
  const void* fn = mode == M_G2R ? cl_fn<M_G2R>(n) : mode == M_R2G ? cl_fn<M_R2G>(n) : cl_fn<M_APPLY>(n);
  if (s == 0 || !fn) return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CL_CS, 1, 1);
  cfg.blockDim = dim3(CL_NW * 32, 1, 1);
  cfg.dynamicSmemBytes = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL_CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n_cl = 0;
  return cudaOccupancyMaxActiveClusters(&n_cl, fn, &cfg) == cudaSuccess ? n_cl : 0;
}

// L.plane_ctas: CTAs (two per cluster; 0: one cluster per plane)
cudaError_t launch_plane_cluster(int mode, const Launch& L) {
  const int n = L.g.n0;
  const size_t s = plane_cluster_smem(n, n, L.g.xmax, mode);
  if (s == 0 || L.g.n1 != n) return cudaErrorInvalidValue;
  const int nplanes = L.nb * L.g.n2;
  const int ncl = L.plane_ctas > 0 ? std::max(1, std::min(L.plane_ctas / CL_CS, nplanes)) : nplanes;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(CL_CS * ncl, 1, 1);
  cfg.blockDim = dim3(CL_NW * 32, 1, 1);
  cfg.dynamicSmemBytes = s;
  cfg.stream = L.stream;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL_CS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = L.pdl ? 2 : 1;
  switch (n) {
    case 256:
      if (mode == M_G2R) return cudaLaunchKernelEx(&cfg, k_plane_cl<256, M_G2R>, L);
      if (mode == M_R2G) return cudaLaunchKernelEx(&cfg, k_plane_cl<256, M_R2G>, L);
      return cudaLaunchKernelEx(&cfg, k_plane_cl<256, M_APPLY>, L);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
