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

#include <map>
#include <mutex>
#include <utility>

#include "async_copy.cuh"
#include "check.cuh"
#include "fft_core.cuh"
#include "fftb_internal.h"
#include "line_fft.cuh"

namespace fftb {

// Element q of a lane's first-pass (R = R0) or last-pass (R = RL) order of a
// length-N line held by G lanes lies, for every lane, strictly inside
// (N/4, N - N/4): where every occupied position of that axis is within
// [-N/4, N/4] it is a zero input (G -> r) or an unneeded output (r -> G).
template <int N, int G, int R> __host__ __device__ constexpr bool x_mid(int q) {
  return (q / R) * G + (q % R) * (N / R) > N / 4 && (q / R) * G + (q % R) * (N / R) + G - 1 < N - N / 4;
}

// the first-pass inputs of a length-N line (E per lane) that are zero when
// every occupied position is within [-N/4, N/4], as a bit mask for Line::run
template <int N, int G, int R, int E> __host__ __device__ constexpr unsigned long long mid_mask() {
  unsigned long long m = 0;
  if (E > 64) return 0;
  for (int q = 0; q < E; ++q)
    if (x_mid<N, G, R>(q)) m |= 1ull << q;
  return m;
}

// ------------------------------------------------------------------ z stage
// Each occupied (x,y) stick is one length-N2 line held in registers by
// Line<N2>::G lanes; a warp carries 32 / G consecutive sticks, a CTA 8 warps.
// No block barrier after the twiddle table load. For a sphere stored stick
// by stick with consecutive gz (the canonical order of a cutoff sphere) the
// lanes index the coefficient list directly; otherwise the warp scatters
// (gathers) its sticks' entries through zeroed scratch rows.
constexpr int STICK_NW = 8;
template <int N2, int V = 0> __host__ __device__ constexpr int stick_tile_c2() {
  return STICK_NW * (32 / Line<N2, V>::G);
}
template <typename T, int N2, int V = 0> constexpr size_t stick_smem_c() {
  using C = typename cplx<T>::type;
  return sizeof(C) * ((size_t)STICK_NW * (32 / Line<N2, V>::G) * Line<N2, V>::PITCH + N2);
}

// resident z-stage CTAs per SM the register allocation must allow (FP32: two,
// measured best; the 128-point z-stage ran one CTA per SM without the cap;
// the two-pass schedule V = 2 holds 40 elements a lane: one)
template <typename T, int V = 0> __host__ __device__ constexpr int stick_minb() {
#ifdef FFTB_STICK_MINB
  return FFTB_STICK_MINB;
#else
  return (sizeof(T) == 8 || V == 2) ? 1 : 2;
#endif
}

// QZ: every sphere entry of the launch has |z| <= N2/4 (KF_Z_QUARTER): the
// z lines' inputs (G -> r) and needed outputs (r -> G) avoid the middle half
// of the line, whose loads, stores and (r -> G) arithmetic are dropped at
// compile time.
template <typename T, int N2, int MODE, bool TC = false, int V = 0, bool QZ = false>
__global__ void __launch_bounds__(STICK_NW * 32, (stick_minb<T, V>())) k_stick(const Launch L) {
  using C = typename cplx<T>::type;
  using LZ = Line<N2, V>;
  constexpr int WZ = 32 / LZ::G, EZ = LZ::E, NT = STICK_NW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane % LZ::G, l = lane / LZ::G;
  C* scr = tw + N2 + warp * WZ * LZ::PITCH;
  C* row = scr + l * LZ::PITCH;
  {
    const C* tw_g = static_cast<const C*>(L.g.tw2);
    for (int m = threadIdx.x; m < N2; m += NT) tw[m] = tw_g[m];
  }
  pdl_launch_dependents();
  __syncthreads();
  pdl_wait();
  typename LZ::template TwCache<C> tc;
  tc.load(g, tw);
  typename LZ::template TcW<MODE == M_G2R ? +1 : -1> tcw;
  if constexpr (TC) tcw.load(tw);
  auto zsigned = [](int z) { return z < N2 - N2 / 2 ? z : z - N2; };
  const int smax = L.g.smax;

  // tasks = (band, group of WZ sticks), dealt to warps with a grid stride so
  // that the warps active at any moment work on neighbouring stick groups
  // (their stick-row stores meet in L2)
  const int gpb = (smax + WZ - 1) / WZ;
  const int ntask = L.nb * gpb;
  const int nwarps = gridDim.x * STICK_NW;
  const int t0 = blockIdx.x * STICK_NW + warp;
  const int t1 = ntask;
  int cur_bl = -1, S = 0, stick_base = 0, bst = 1;
  bool canon = false;
  int64_t sph = 0;
  auto band_of = [&](int bl) {
    if (bl != cur_bl) {
      cur_bl = bl;
      const BandInfo bi = L.g.band[L.band0 + bl];
      S = bi.ki.S;
      stick_base = bi.ki.stick_base;
      canon = bi.ki.flags & KF_CANONICAL_STICKS;
      bst = bi.ki.bstride;
      sph = bi.sph;
    }
  };
  struct Task {
    int bl, s0, nl;
    int4 si;  // first entry, end entry, list position, signed gz of this lane's stick
    int64_t sph;
    int st;  // sphere entry stride (1 band-major, B_k batch-fastest)
    bool live, canon;
  };
  auto meta = [&](int t) {
    Task k{};
    if (t >= ntask) return k;  // past the last task: dead, no table reads
    k.bl = t / gpb;
    k.s0 = (t - k.bl * gpb) * WZ;
    band_of(k.bl);
    k.live = k.s0 < S;
    k.canon = canon;
    k.sph = sph;
    k.st = bst;
    k.nl = k.live ? min(WZ, S - k.s0) : 0;
    const int s = k.s0 + (l < k.nl ? l : 0);
    k.si = k.live ? L.g.stick_info[stick_base + s] : make_int4(0, 0, 0, 0);
    return k;
  };
  // global loads of a task into registers (canonical G->r or any r->G)
  auto load = [&](const Task& k, C (&v)[EZ]) {
    if constexpr (MODE == M_G2R) {
      const C* in = static_cast<const C*>(L.sph_in) + k.sph;
      const int len = k.si.y - k.si.x;
      if (k.st == 1) {  // band-major: the stick's entries are adjacent
#pragma unroll
        for (int m = 0; m < EZ / LZ::R0; ++m)
#pragma unroll
          for (int j = 0; j < LZ::R0; ++j) {
            if (QZ && x_mid<N2, LZ::G, LZ::R0>(m * LZ::R0 + j)) {  // no entry there
              v[m * LZ::R0 + j] = czero<C>();
              continue;
            }
            const int d = zsigned(LZ::first_pos(g, m, j)) - k.si.w;
            v[m * LZ::R0 + j] = (unsigned)d < (unsigned)len && FFTB_IN(k.sph + k.si.z + d, L.lim_sph, L.status)
                                    ? in[k.si.z + d]
                                    : czero<C>();
          }
      } else {  // batch-fastest: B_k apart
#pragma unroll
        for (int m = 0; m < EZ / LZ::R0; ++m)
#pragma unroll
          for (int j = 0; j < LZ::R0; ++j) {
            if (QZ && x_mid<N2, LZ::G, LZ::R0>(m * LZ::R0 + j)) {  // no entry there
              v[m * LZ::R0 + j] = czero<C>();
              continue;
            }
            const int d = zsigned(LZ::first_pos(g, m, j)) - k.si.w;
            v[m * LZ::R0 + j] =
                (unsigned)d < (unsigned)len && FFTB_IN(k.sph + (int64_t)(k.si.z + d) * k.st, L.lim_sph, L.status)
                    ? in[(int64_t)(k.si.z + d) * k.st]
                    : czero<C>();
          }
      }
    } else {
      const size_t tb = (size_t)k.bl * N2 * smax + k.s0 + (l < k.nl ? l : 0);
      const C* Tb = static_cast<const C*>(L.T) + tb;
#pragma unroll
      for (int m = 0; m < EZ / LZ::R0; ++m)
#pragma unroll
        for (int j = 0; j < LZ::R0; ++j)
          v[m * LZ::R0 + j] = FFTB_IN(tb + (size_t)LZ::first_pos(g, m, j) * smax, L.lim_T, L.status)
                                  ? Tb[(size_t)LZ::first_pos(g, m, j) * smax]
                                  : czero<C>();
    }
  };
  // transform and write a task whose inputs are in v
  auto finish = [&](const Task& k, C (&v)[EZ]) {
    if constexpr (MODE == M_G2R) {
      if constexpr (TC) LZ::template run_tc<+1>(v, g, row, scr, tw, tc, tcw);
      else LZ::template run<+1, QZ ? mid_mask<N2, LZ::G, LZ::R0, EZ>() : 0ull>(v, g, row, tw, tc);
      if (l < k.nl) {
        const size_t tb = (size_t)k.bl * N2 * smax + k.s0 + l;
        C* Tb = static_cast<C*>(L.T) + tb;
#pragma unroll
        for (int m = 0; m < EZ / LZ::RL; ++m)
#pragma unroll
          for (int j = 0; j < LZ::RL; ++j)
            if (FFTB_IN(tb + (size_t)LZ::last_pos(g, m, j) * smax, L.lim_T, L.status))
              Tb[(size_t)LZ::last_pos(g, m, j) * smax] = v[m * LZ::RL + j];
      }
    } else {
      if constexpr (TC) LZ::template run_tc<-1>(v, g, row, scr, tw, tc, tcw);
      else LZ::template run<-1>(v, g, row, tw, tc);
      C* out = static_cast<C*>(L.sph_out) + k.sph;
      if (k.canon) {
        if (l < k.nl) {
          const int len = k.si.y - k.si.x;
          if (k.st == 1) {
#pragma unroll
            for (int m = 0; m < EZ / LZ::RL; ++m)
#pragma unroll
              for (int j = 0; j < LZ::RL; ++j) {
                if (QZ && x_mid<N2, LZ::G, LZ::RL>(m * LZ::RL + j)) continue;  // no entry there
                const int d = zsigned(LZ::last_pos(g, m, j)) - k.si.w;
                if ((unsigned)d < (unsigned)len && FFTB_IN(k.sph + k.si.z + d, L.lim_sph, L.status))
                  out[k.si.z + d] = v[m * LZ::RL + j];
              }
          } else {
#pragma unroll
            for (int m = 0; m < EZ / LZ::RL; ++m)
#pragma unroll
              for (int j = 0; j < LZ::RL; ++j) {
                if (QZ && x_mid<N2, LZ::G, LZ::RL>(m * LZ::RL + j)) continue;  // no entry there
                const int d = zsigned(LZ::last_pos(g, m, j)) - k.si.w;
                if ((unsigned)d < (unsigned)len &&
                    FFTB_IN(k.sph + (int64_t)(k.si.z + d) * k.st, L.lim_sph, L.status))
                  out[(int64_t)(k.si.z + d) * k.st] = v[m * LZ::RL + j];
              }
          }
        }
      } else {
        const int ea = __shfl_sync(0xffffffffu, k.si.x, 0);
        const int eb = __shfl_sync(0xffffffffu, k.si.y, (k.nl - 1) * LZ::G);
#pragma unroll
        for (int m = 0; m < EZ / LZ::RL; ++m)
#pragma unroll
          for (int j = 0; j < LZ::RL; ++j) {
            if (QZ && x_mid<N2, LZ::G, LZ::RL>(m * LZ::RL + j)) continue;  // no entry there
            row[wpad(LZ::last_pos(g, m, j))] = v[m * LZ::RL + j];
          }
        __syncwarp();
        for (int e = ea + lane; e < eb; e += 32) {
          const uint32_t zs = (uint32_t)L.g.ent_zs[e];
          if (FFTB_IN(k.sph + (int64_t)L.g.ent_pos[e] * k.st, L.lim_sph, L.status))
            out[(int64_t)L.g.ent_pos[e] * k.st] = scr[((int)(zs & 0xFFFFFFu) - k.s0) * LZ::PITCH + wpad((int)(zs >> 24))];
        }
        __syncwarp();
      }
    }
  };
  // a non-canonical G->r task gathers its entries through the warp scratch
  auto scatter_load = [&](const Task& k, C (&v)[EZ]) {
    const C* in = static_cast<const C*>(L.sph_in) + k.sph;
    const int ea = __shfl_sync(0xffffffffu, k.si.x, 0);
    const int eb = __shfl_sync(0xffffffffu, k.si.y, (k.nl - 1) * LZ::G);
    for (int q = lane; q < WZ * LZ::PITCH; q += 32) scr[q] = czero<C>();
    __syncwarp();
    for (int e = ea + lane; e < eb; e += 32) {
      const uint32_t zs = (uint32_t)L.g.ent_zs[e];
      if (FFTB_IN(k.sph + (int64_t)L.g.ent_pos[e] * k.st, L.lim_sph, L.status))
        scr[((int)(zs & 0xFFFFFFu) - k.s0) * LZ::PITCH + wpad((int)(zs >> 24))] = in[(int64_t)L.g.ent_pos[e] * k.st];
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < EZ / LZ::R0; ++m)
#pragma unroll
      for (int j = 0; j < LZ::R0; ++j) v[m * LZ::R0 + j] = row[wpad(LZ::first_pos(g, m, j))];
    __syncwarp();
  };

  if (t0 >= t1) return;
  if constexpr (V == 2) {
    // the two-pass schedule (40 elements a lane) leaves no registers for a
    // second task in flight: one task at a time, eight sticks a warp
#pragma unroll 1
    for (int t = t0; t < t1; t += nwarps) {
      const Task k = meta(t);
      if (!k.live) continue;
      C v[EZ];
      if (MODE == M_R2G || k.canon) load(k, v);
      else scatter_load(k, v);
      finish(k, v);
    }
    return;
  }
  // two-deep software pipeline: the next task's records and inputs are in
  // flight while the current task is transformed and written
  C va[EZ], vb[EZ];
  Task ka = meta(t0), kb{};
  if (ka.live && (MODE == M_R2G || ka.canon)) load(ka, va);
#pragma unroll 1
  for (int t = t0; t < t1; t += 2 * nwarps) {
    kb = meta(t + nwarps);
    if (kb.live && (MODE == M_R2G || kb.canon)) load(kb, vb);
    if (ka.live) {
      if (!(MODE == M_R2G || ka.canon)) scatter_load(ka, va);
      finish(ka, va);
    }
    ka = meta(t + 2 * nwarps);
    if (ka.live && (MODE == M_R2G || ka.canon)) load(ka, va);
    if (kb.live) {
      if (!(MODE == M_R2G || kb.canon)) scatter_load(kb, vb);
      finish(kb, vb);
    }
  }
}

// ------------------------------------------------------------- y, x stages
// Persistent CTAs walk the (band, z) planes with a grid stride. Every y- or
// x-line is transformed by a group of Line<N>::G lanes holding it in
// registers (line_fft.cuh); a warp carries 32 / G lines at a time and needs
// no block barrier inside a phase. The slab plane A[y][xi] (the plane
// restricted to the X occupied x-slabs) is double buffered when shared memory
// allows, so one block barrier per plane separates its y and x phases, and a
// warp that finishes plane p's x phase goes straight on to plane p+1's y
// phase (with one buffer a second barrier ends each plane). A's pitch is X
// rounded up to a residue mod 16 (a_res) chosen for the bank pattern of the
// y phase's column writes and the x phase's row reads. x-phase tasks are
// dealt out after the y-phase tasks, so the warps with fewer y lines get more
// x rows.
#ifndef FFTB_PLANE_NW
#define FFTB_PLANE_NW 8
#endif


template <typename T> struct PlaneCfg { static constexpr int NW = FFTB_PLANE_NW; };

// In the variant with slab planes in global memory (EF), data read or written
// once per plane (cube rows, the stick row) takes the evict-first cache
// policy (ld/st.global.cs), so that it does not push the slab planes out of
// L2. Elsewhere plain accesses keep the end of a written cube in L2 for the
// next stage of a round trip.
template <bool EF, typename C> __device__ __forceinline__ C ld_once(const C* p) {
  if constexpr (EF) return __ldcs(p);
  else return *p;
}
template <bool EF, typename C> __device__ __forceinline__ void st_once(C* p, C v) {
  if constexpr (EF) __stcs(p, v);
  else *p = v;
}
// two adjacent FP32 complex values as one 16-byte store (p on a 16-byte boundary)
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
// resident CTAs per SM the register allocation must allow (measured best)
template <typename T, int N0> __host__ __device__ constexpr int plane_minb() {
#ifdef FFTB_PLANE_MINB
  return FFTB_PLANE_MINB;
#else
  return sizeof(T) == 8 ? 1 : (N0 <= 64 ? 3 : N0 == 160 ? 1 : 2);
#endif
}

__host__ __device__ constexpr int a_pitch(int x, int r = 2) { return x + ((r - x % 16) + 16) % 16; }
// Residue of the slab-plane pitch. 8-byte elements with G = 4 lanes per y and
// x line: a warp's column store covers 4 rows x 8 columns and its row load 8
// rows x 4 columns (16 and 8 banks a row); a pitch of 4 (mod 16) puts
// successive rows 8 banks apart, so every bank is hit twice, the two
// wavefronts that 256 bytes need at least (a pitch of 2 (mod 16) hits some
// banks of a column store four times). Other shapes keep 2 (mod 16).
template <typename C, int N0, int N1, int V> __host__ __device__ constexpr int a_res() {
  return sizeof(C) == 8 && Line<N0, V>::G == 4 && Line<N1, V>::G == 4 ? 4 : 2;
}
template <int N0, int N1, int V = 0> __host__ __device__ constexpr int plane_scratch() {
  return (32 / Line<N1, V>::G) * Line<N1, V>::PITCH > (32 / Line<N0, V>::G) * Line<N0, V>::PITCH
             ? (32 / Line<N1, V>::G) * Line<N1, V>::PITCH
             : (32 / Line<N0, V>::G) * Line<N0, V>::PITCH;
}

// Row pitch (elements) of cube rows staged in shared memory by the r -> G
// prefetch: 64 bytes beyond a multiple of 128, so the rows a warp reads at
// once fall on both halves of the banks; even, so every row starts on a
// 16-byte boundary.
template <typename C> __host__ __device__ constexpr int stage_pitch(int n) {
  return n + ((int)(64 / sizeof(C)) - n % (int)(128 / sizeof(C)) + (int)(128 / sizeof(C))) % (int)(128 / sizeof(C));
}
// Pitch of the staged rows of an r -> G x task. For 64-point rows the task's
// rows arrive as one bulk copy, unpadded (measured faster: the copy-issue
// instructions it saves outweigh the two-way bank conflicts of reading two
// rows 512 bytes apart); longer rows are copied one by one at stage_pitch.
template <typename C, int N0> __host__ __device__ constexpr int pf_row_pitch() {
  return N0 == 64 ? N0 : stage_pitch<C>(N0);
}
// The r -> G prefetch hands every warp at least one x task per plane.
template <typename T, int N0, int N1> __host__ __device__ constexpr bool rows_prefetchable() {
  return (N1 + 32 / Line<N0>::G - 1) / (32 / Line<N0>::G) >= PlaneCfg<T>::NW;
}
// Shared memory the prefetch adds for `mode` (0: none): the next plane's
// stick row (tp elements, G -> r and apply) or each warp's next x-task rows
// (r -> G), plus their mbarriers.
template <typename T, int N0, int N1> size_t plane_pf_bytes(int mode, int tp) {
  using C = typename cplx<T>::type;
  constexpr int NW = PlaneCfg<T>::NW, WX = 32 / Line<N0>::G;
  if (mode == 0) return 0;
  if (mode == M_R2G) return sizeof(C) * (size_t)NW * WX * pf_row_pitch<C, N0>() + 8 * NW;
  return sizeof(C) * (size_t)tp + 16;
}
template <typename T, int N0, int N1, int V = 0>
size_t plane_smem_c(int xmax, int a_bufs, bool ag = false, int pf_mode = 0, int tp = 0) {
  using C = typename cplx<T>::type;
  return sizeof(C) * ((ag ? 0 : (size_t)a_bufs * N1 * a_pitch(xmax, a_res<C, N0, N1, V>())) +
                      (size_t)PlaneCfg<T>::NW * plane_scratch<N0, N1, V>() + N0 + N1) +
         plane_pf_bytes<T, N0, N1>(pf_mode, tp) + (V >= 2 ? sizeof(uint64_t) * PlaneCfg<T>::NW : 0) + 16;
}

// packed per-lane slab indices: byte q of w[q / 4] = xi of position q, 255 =
// empty (unless all N0 x values are occupied: then 255 is slab 255)
template <int E> struct XiPack {
  uint32_t w[(E + 3) / 4];
  __device__ __forceinline__ int get(int q) const { return (int)((w[q >> 2] >> (8 * (q & 3))) & 0xFFu); }
};

// PF: the plane's global inputs arrive by bulk asynchronous copies issued
// one step ahead (G -> r, apply: the next plane's stick row, whole, by thread
// 0 after the mid-plane barrier; r -> G: each warp's next x task's cube rows,
// by the warp itself once it has read the current ones), completed on
// mbarriers. A wait that runs out sets the plan's status word; the CTA then
// leaves at the next block barrier, after its copies in flight have landed.
template <typename T, int N0, int N1, int MODE, bool TC = false, bool AG = false, bool PF = false, int V = 0,
          bool QP = false>
__global__ void __launch_bounds__(PlaneCfg<T>::NW * 32, (plane_minb<T, N0>())) k_plane(const Launch L) {
  using C = typename cplx<T>::type;
  using LY = Line<N1, V>;
  // G -> r with the two-pass schedule (FP32): the x lines take the paired
  // variant, whose outputs leave as 16-byte pairs (measured: 14 % faster at
  // 160^3; the same variant for the y lines, whose outputs go to the slab
  // plane, measured 1.5 % slower)
  constexpr bool PAIRED = (V == 2 || V == 3) && MODE == M_G2R && sizeof(T) == 4 && !TC && !AG && !PF;
  using LX = Line<N0, (PAIRED && N0 == 160) ? 4 : V>;
  constexpr int NW = PlaneCfg<T>::NW, NT = NW * 32;
  constexpr int WY = 32 / LY::G, WX = 32 / LX::G;   // lines per warp
  constexpr int EY = LY::E, EX = LX::E;
  constexpr int SCR = plane_scratch<N0, N1, V>();
  static_assert(WX * LX::PITCH <= SCR && WY * LY::PITCH <= SCR, "lines' exchange rows fit the warp's scratch");
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const int n2 = L.g.n2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gy = lane % LY::G, ly = lane / LY::G;
  const int gx = lane % LX::G, lx = lane / LX::G;
  constexpr int AR = a_res<C, N0, N1, V>();
  static_assert(!LX::PAIR || (AR % 2 == 0 && SCR % 2 == 0 && LX::PITCH % 2 == 0),
                "paired exchange rows start on 16-byte boundaries");
  const int abuf = N1 * a_pitch(L.g.xmax, AR);
  const int nbuf = L.a_bufs;
  // slab planes: shared memory, or (AG) this CTA's block of a global buffer
  C* A0 = AG ? static_cast<C*>(L.a_glob) + (size_t)blockIdx.x * nbuf * abuf : reinterpret_cast<C*>(smem_raw);
  C* sbase = reinterpret_cast<C*>(smem_raw) + (AG ? 0 : nbuf * abuf);
  C* scr = sbase + warp * SCR;
  C* tw0 = sbase + NW * SCR;
  C* tw1 = tw0 + N0;
  // prefetch staging (PF): a stick row, or NW blocks of WX cube rows at pitch RP
  constexpr int RP = pf_row_pitch<C, N0>();
  C* stg = tw1 + N1;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + (MODE == M_R2G ? NW * WX * RP : L.g.smax));
  // XS (the two-pass x schedule, r -> G): the cube rows of a warp's next x
  // task arrive by bulk copies in the lines' exchange rows, completed on the
  // warp's mbarrier (measured: 14 % faster than loads by the lanes; staging
  // the G -> r rows for bulk stores the same way measured 8 % slower than
  // stores by the lanes). Used where the cube is band-major and 16-byte
  // aligned (L.pf).
  constexpr bool XS = V >= 2 && !AG && !PF && !TC;
  // YS (the same schedule, G -> r): where a column's sticks are consecutive
  // in the stick row (canonical spheres), the stick values of a warp's next y
  // task, one contiguous run of the row, arrive by one bulk copy in the
  // warp's exchange rows, completed on the warp's mbarrier. The copy is issued
  // as soon as the rows are free: after the exchange of the warp's current y
  // task, or after the exchange of its last x task of the previous plane.
  constexpr bool YS = XS && MODE == M_G2R;
  // V = 3 (the two-pass schedule) and QP (the other schedules) for plans whose
  // k-points all have every occupied stick within [-N0/4, N0/4] x
  // [-N1/4, N1/4] (KF_XY_QUARTER): the y and x lines drop the middle half of
  // the line at compile time, zero inputs (G -> r, apply) and unneeded outputs
  // (r -> G, apply), whose arithmetic the compiler removes
  constexpr bool XQ = (V == 3 || QP) && !TC;
  constexpr unsigned long long ZMX = XQ ? mid_mask<N0, LX::G, LX::R0, EX>() : 0ull;  // zero x inputs (G -> r)
  constexpr unsigned long long ZMY = XQ ? mid_mask<N1, LY::G, LY::R0, EY>() : 0ull;  // zero y inputs (G -> r)
  static_assert(!XS || (LX::PITCH * sizeof(C)) % 16 == 0, "staged rows start on 16-byte boundaries");
  uint64_t* xbar = reinterpret_cast<uint64_t*>(tw1 + N1);
  // end of the layout (8-byte aligned): the slab-plane barrier of single-buffer kernels
  uint64_t* afree = PF ? bars + (MODE == M_R2G ? NW : 1) : (XS ? xbar + NW : reinterpret_cast<uint64_t*>(tw1 + N1));
  C* wst = stg + warp * (WX * RP);
  {
    const C* t0 = static_cast<const C*>(L.g.tw0);
    const C* t1 = static_cast<const C*>(L.g.tw1);
    for (int m = threadIdx.x; m < N0; m += NT) tw0[m] = t0[m];
    for (int m = threadIdx.x; m < N1; m += NT) tw1[m] = t1[m];
  }
  if constexpr (PF) {
    if (threadIdx.x < (MODE == M_R2G ? NW : 1)) {
      mbar_init(bars + threadIdx.x, 1);
      mbar_init_fence();
    }
  }
  if constexpr (XS && (MODE == M_R2G || YS)) {
    if (threadIdx.x < NW) {
      mbar_init(xbar + threadIdx.x, 1);
      mbar_init_fence();
    }
  }
  if (threadIdx.x == 0 && nbuf == 1) {
    mbar_init(afree, NW);
    mbar_init_fence();
  }
  pdl_launch_dependents();
  __syncthreads();
  pdl_wait();
  C* rowy = scr + ly * LY::PITCH;
  C* rowx = scr + lx * LX::PITCH;
  typename LY::template TwCache<C> tcy;
  typename LX::template TwCache<C> tcx;
  tcy.load(gy, tw1);
  tcx.load(gx, tw0);
  // tensor-core DFT8 operands (MIXED_TC): forward sign for G->r, inverse for r->G
  typename LY::template TcW<+1> wy_p;
  typename LX::template TcW<+1> wx_p;
  typename LY::template TcW<-1> wy_m;
  typename LX::template TcW<-1> wx_m;
  if constexpr (TC) {
    if constexpr (MODE != M_R2G) { wy_p.load(tw1); wx_p.load(tw0); }
    if constexpr (MODE != M_G2R) { wy_m.load(tw1); wx_m.load(tw0); }
  }
  // the paired x schedule's 16-byte cube stores need a cube on 16-byte boundaries (uniform)
  const bool pair16 = LX::PAIR && (reinterpret_cast<uintptr_t>(L.cube_out) % 16) == 0;
  // signed y of this lane's first-pass / last-pass y positions (direct stick I/O)
  auto ysigned = [](int y) { return y < N1 - N1 / 2 ? y : y - N1; };

  const int nplanes = L.nb * n2;
  // ---- prefetch state (PF)
  bool bad = false;          // a wait ran out
  bool outstanding = false;  // a copy phase was issued (or withheld by injection) and not yet seen complete
  uint32_t ph = 0;           // parity of the next phase to complete
  // G -> r, apply (thread 0): the stick row of plane pp, rounded up to 16 bytes (within the even pitch)
  auto issue_trow = [&](int pp) {
    const int bl2 = pp / n2, z2 = pp - bl2 * n2;
    const int S2 = L.g.band[L.band0 + bl2].ki.S;
    uint32_t bytes = (uint32_t)((S2 * (int)sizeof(C) + 15) & ~15);
    if (bytes && !FFTB_IN(((size_t)bl2 * n2 + z2) * L.g.smax + bytes / sizeof(C) - 1, L.lim_T, L.status)) bytes = 0;
    fence_proxy_async_smem();
    mbar_arrive_expect(bars, bytes);
    if (bytes) bulk_g2s(stg, static_cast<const C*>(L.T) + ((size_t)bl2 * n2 + z2) * L.g.smax, bytes, bars);
  };
  // r -> G: this warp's first x task of plane pp (the x tasks follow the y tasks)
  auto x_start = [&](int pp) {
    const int Xn = L.g.band[L.band0 + pp / n2].ki.X;
    return (warp - ((Xn + WY - 1) / WY) % NW + NW) % NW;
  };
  // r -> G (lane 0): the WX cube rows of x task t of plane pp
  auto issue_rows = [&](int pp, int t) {
    const int bl2 = pp / n2, z2 = pp - bl2 * n2;
    const int r0 = t * WX, nr = min(WX, N1 - r0);
    const size_t first = ((size_t)(L.band0 + bl2) * n2 + z2) * (size_t)(N1 * N0) + (size_t)r0 * N0;
    const C* src = static_cast<const C*>(L.cube_in) + first;
    fence_proxy_async_smem();
    if (!FFTB_IN(first + (size_t)nr * N0 - 1, L.lim_cube, L.status)) {
      mbar_arrive_expect(bars + warp, 0);  // nothing copied: the phase completes at once
      return;
    }
    mbar_arrive_expect(bars + warp, (uint32_t)(nr * N0 * sizeof(C)));
    if constexpr (RP == N0) {
      bulk_g2s(wst, src, (uint32_t)(nr * N0 * sizeof(C)), bars + warp);
    } else {
      for (int r = 0; r < nr; ++r) bulk_g2s(wst + r * RP, src + (size_t)r * N0, (uint32_t)(N0 * sizeof(C)), bars + warp);
    }
  };
  // waits for the outstanding phase of barrier b; false if the limit ran out
  auto await = [&](uint64_t* b) {
    if (outstanding && !bad) {
      if (mbar_wait(b, ph, WAIT_LIMIT_NS)) {
        outstanding = false;
        ph ^= 1;
      } else {
        bad = true;
      }
    }
  };
  // leaving after a failed wait: let copies in flight land, report
  auto abort_plane = [&]() {
    if (outstanding) mbar_wait(bars + (MODE == M_R2G ? warp : 0), ph, WAIT_LIMIT_NS);
    if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(L.status) = STATUS_WAIT_TIMEOUT;
  };
  if constexpr (PF) {
    const bool withhold = (L.inject & INJECT_SKIP_FIRST_PREFETCH) && blockIdx.x == 0;
    if ((int)blockIdx.x < nplanes) {
      if constexpr (MODE == M_R2G) {
        if (lane == 0 && !(withhold && warp == 0)) issue_rows(blockIdx.x, x_start(blockIdx.x));
      } else {
        if (threadIdx.x == 0 && !withhold) issue_trow(blockIdx.x);
      }
      outstanding = true;
    }
  }
  // XS, r -> G (lane 0): the cube rows of x task t of plane pp into the
  // warp's exchange rows (row r of the task to line r's row)
  const bool xs_on = XS && L.pf != 0;  // uniform: band-major cube on 16-byte boundaries
  uint32_t xph = 0;                    // parity of the warp barrier's next phase
  bool xpend = false;                  // a row copy was issued (or withheld) and not yet waited for
  C* const xrows = scr;
  auto issue_xrows = [&](int pp, int t) {
    const int bl2 = pp / n2, z2 = pp - bl2 * n2;
    const int r0 = t * WX, nr = min(WX, N1 - r0);
    const size_t first = ((size_t)(L.band0 + bl2) * n2 + z2) * (size_t)(N1 * N0) + (size_t)r0 * N0;
    const C* src = static_cast<const C*>(L.cube_in) + first;
    fence_proxy_async_smem();
    if (!FFTB_IN(first + (size_t)nr * N0 - 1, L.lim_cube, L.status)) {
      mbar_arrive_expect(xbar + warp, 0);  // nothing copied: the phase completes at once
      return;
    }
    mbar_arrive_expect(xbar + warp, (uint32_t)(nr * N0 * sizeof(C)));
    for (int r = 0; r < nr; ++r)
      bulk_g2s(xrows + r * LX::PITCH, src + (size_t)r * N0, (uint32_t)(N0 * sizeof(C)), xbar + warp);
  };
  // YS (lane 0): the stick values of y task t of plane pp, from the even
  // stick position at or below its first column's first stick to the end of
  // its last column, rounded up to 16 bytes (inside the even-pitch row)
  static_assert(!YS || WY * LY::PITCH >= WY * N1 + 2, "a task's sticks fit the warp's exchange rows");
  static_assert(!YS || (N1 + WX - 1) / WX >= NW, "every warp has an x task in each plane");
  auto issue_ycols = [&](int pp, int t) {
    const int bl2 = pp / n2, z2 = pp - bl2 * n2;
    const KInfo k2 = L.g.band[L.band0 + bl2].ki;
    const int4* ci2 = L.g.col_info + k2.col_base;
    const int c0 = t * WY, cl = c0 + min(WY, k2.X - c0) - 1;
    const int s_lo = ci2[c0].x & ~1;
    const int4 cz = ci2[cl];
    const uint32_t bytes = (uint32_t)(((cz.x + cz.y - s_lo) * (int)sizeof(C) + 15) & ~15);
    const size_t first = ((size_t)bl2 * n2 + z2) * L.g.smax + s_lo;
    fence_proxy_async_smem();
    if (bytes == 0 || !FFTB_IN(first + bytes / sizeof(C) - 1, L.lim_T, L.status)) {
      mbar_arrive_expect(xbar + warp, 0);  // nothing copied: the phase completes at once
      return;
    }
    mbar_arrive_expect(xbar + warp, bytes);
    bulk_g2s(xrows, static_cast<const C*>(L.T) + first, bytes, xbar + warp);
  };
  // YS (warp-uniform): this warp's first y task of plane pn, if pn's columns
  // are staged and the warp has a y task there (withheld under test injection)
  auto ys_issue_first = [&](int pn, bool withhold) {
    if (!YS || bad || pn >= nplanes) return;
    const KInfo kn = L.g.band[L.band0 + pn / n2].ki;
    if (!(kn.flags & KF_CONTIGUOUS_COLUMNS) || warp >= (kn.X + WY - 1) / WY) return;
    __syncwarp();
    if (lane == 0 && !withhold) issue_ycols(pn, warp);
    xpend = true;
  };
  // waits for this warp's outstanding row copy (XS, YS); a wait that runs out marks the CTA bad
  auto xwait = [&]() {
    if (xpend && !bad) {
      const bool ok = mbar_wait(xbar + warp, xph, WAIT_LIMIT_NS);
      if (__any_sync(0xffffffffu, ok)) {
        xpend = false;
        xph ^= 1;
      } else {
        bad = true;
      }
    }
  };
  if constexpr (YS) ys_issue_first(blockIdx.x, (L.inject & INJECT_SKIP_FIRST_PREFETCH) && blockIdx.x == 0 && warp == 0);
  // One slab-plane buffer: instead of a block barrier at the end of every
  // plane, each warp arrives on afree after its last read of the plane's slab
  // plane, and waits for that phase before its first write of the next
  // plane's, so warps still finishing a plane overlap the others' start of
  // the next (one phase per plane, NW arrivals; at most one phase ahead).
  // (slab planes in shared memory only: with slab planes in global memory,
  // 256^3, the block barrier measured as fast or slightly faster)
  const bool a_single = nbuf == 1 && !AG;
  uint32_t a_phase = 0;     // this CTA's plane count: the phase of the current plane
  bool a_got = false;       // this warp has waited for the previous plane's phase
  bool a_rel = false;       // this warp has arrived for the current plane
  auto a_acquire = [&]() {  // warp-uniform, before a slab-plane write
    if (a_single && a_phase > 0 && !a_got) {
      if (!mbar_wait(afree, (a_phase - 1) & 1, WAIT_LIMIT_NS)) {
        bad = true;
        *reinterpret_cast<volatile int32_t*>(L.status) = STATUS_WAIT_TIMEOUT;
      }
      a_got = true;
    }
  };
  auto a_release = [&]() {  // warp-uniform, after the warp's last slab-plane read of the plane
    if (a_single && !a_rel) {
      __syncwarp();
      if (lane == 0) mbar_arrive(afree);
      a_rel = true;
    }
  };
  int cur_k = -1;
  XiPack<EX> xin, xout;  // slab index of this lane's first-pass / last-pass x positions
  int parity = 0;
#pragma unroll 1
  for (int p = blockIdx.x; p < nplanes; p += gridDim.x, parity ^= (nbuf - 1)) {
    const int bl = p / n2;
    const int z = p - bl * n2;
    const int gb = L.band0 + bl;
    const BandInfo bi = L.g.band[gb];
    const KInfo ki = bi.ki;
    const int X = ki.X;
    const int cst = ki.bstride;  // cube point stride: 1 band-major, B_k batch-fastest
    const int XP = a_pitch(X, AR);
    // every x occupied (a full frequency box): all 256 byte values of the
    // per-lane slab indices are slabs, none marks an empty x
    const bool allx = X >= N0;
    if (ki.xmap_base != cur_k) {  // a new k-point (uniform across the CTA)
      cur_k = ki.xmap_base;
      const int16_t* xm = L.g.xmap + ki.xmap_base;
#pragma unroll
      for (int q = 0; q < (EX + 3) / 4; ++q) { xin.w[q] = 0; xout.w[q] = 0; }
#pragma unroll
      for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
        for (int j = 0; j < LX::R0; ++j) {
          const int q = m * LX::R0 + j, xi = xm[LX::first_pos(gx, m, j)];
          xin.w[q >> 2] |= (uint32_t)(xi < 0 ? 255 : xi) << (8 * (q & 3));
        }
#pragma unroll
      for (int m = 0; m < EX / LX::RL; ++m)
#pragma unroll
        for (int j = 0; j < LX::RL; ++j) {
          const int q = m * LX::RL + j, xi = xm[LX::last_pos(gx, m, j)];
          xout.w[q >> 2] |= (uint32_t)(xi < 0 ? 255 : xi) << (8 * (q & 3));
        }
    }
    C* A = A0 + parity * abuf;
    const int4* __restrict__ cinfo = L.g.col_info + ki.col_base;
    const int32_t* sxy = L.g.stick_xy + ki.stick_base;
    const size_t tz = ((size_t)bl * n2 + z) * L.g.smax;  // first element of this plane's stick row
    C* Tz = static_cast<C*>(L.T) + tz;
    const size_t plane = (size_t)bi.cube + (size_t)z * (size_t)(N1 * N0) * (size_t)cst;
    const int ty = (X + WY - 1) / WY;       // y tasks of this plane
    const int tx = (N1 + WX - 1) / WX;      // x tasks
    const int x_first = ty % NW;            // x tasks start after the y tasks

    if constexpr (MODE == M_G2R || MODE == M_APPLY) {
      // y-DFT (+) of the occupied x-slab columns: scatter the sticks of this
      // warp's columns into zeroed scratch rows, transform, write A columns
      const C* Tr = Tz;
      if constexpr (PF) {
        await(bars);
        Tr = stg;
      }
#pragma unroll 1
      for (int t = warp; t < ty; t += NW) {
        const int c0 = t * WY, nl = min(WY, X - c0);
        C v[EY];
        const int col = c0 + (ly < nl ? ly : 0);
        const int4 ci = cinfo[col];  // first stick, sticks, signed gy of the first
        if (YS && (ki.flags & KF_CONTIGUOUS_COLUMNS)) {
          // the task's sticks, staged from the even position sb on
          xwait();
          const int sb = __shfl_sync(0xffffffffu, ci.x, 0) & ~1;
          const int sa = ci.x - sb, len = ci.y, ylo = ci.z;
#pragma unroll
          for (int m = 0; m < EY / LY::R0; ++m)
#pragma unroll
            for (int j = 0; j < LY::R0; ++j) {
              if (XQ && x_mid<N1, LY::G, LY::R0>(m * LY::R0 + j)) {  // no occupied y there
                v[m * LY::R0 + j] = czero<C>();
                continue;
              }
              const int d = ysigned(LY::first_pos(gy, m, j)) - ylo;
              v[m * LY::R0 + j] = (unsigned)d < (unsigned)len ? xrows[sa + d] : czero<C>();
            }
          __syncwarp();
        } else if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          // each column's sticks are consecutive in gy: index them directly
          const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
          for (int m = 0; m < EY / LY::R0; ++m)
#pragma unroll
            for (int j = 0; j < LY::R0; ++j) {
              if (XQ && x_mid<N1, LY::G, LY::R0>(m * LY::R0 + j)) {  // no occupied y there
                v[m * LY::R0 + j] = czero<C>();
                continue;
              }
              const int d = ysigned(LY::first_pos(gy, m, j)) - ylo;
              if constexpr (PF) v[m * LY::R0 + j] = (unsigned)d < (unsigned)len ? Tr[sa + d] : czero<C>();
              else
                v[m * LY::R0 + j] = (unsigned)d < (unsigned)len && FFTB_IN(tz + sa + d, L.lim_T, L.status)
                                        ? ld_once<AG>(Tr + sa + d)
                                        : czero<C>();
            }
        } else {
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LY::G);
          for (int q = lane; q < WY * LY::PITCH; q += 32) scr[q] = czero<C>();
          __syncwarp();
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            if constexpr (PF) scr[((xy >> 16) - c0) * LY::PITCH + LY::pad(xy & 0xFFFF)] = Tr[s];
            else if (FFTB_IN(tz + s, L.lim_T, L.status))
              scr[((xy >> 16) - c0) * LY::PITCH + LY::pad(xy & 0xFFFF)] = ld_once<AG>(Tr + s);
          }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < EY / LY::R0; ++m)
#pragma unroll
            for (int j = 0; j < LY::R0; ++j)
              v[m * LY::R0 + j] = XQ && x_mid<N1, LY::G, LY::R0>(m * LY::R0 + j) ? czero<C>()  // no stick there
                                                                                 : rowy[LY::pad(LY::first_pos(gy, m, j))];
          __syncwarp();
        }
        if constexpr (TC) LY::template run_tc<+1>(v, gy, rowy, scr, tw1, tcy, wy_p);
        else if constexpr (YS) {
          // once the exchange rows have been read back, fetch the next y task's sticks into them
          LY::template run2<+1, ZMY>(v, gy, rowy, tw1, tcy, [] {}, [&] {
            if ((ki.flags & KF_CONTIGUOUS_COLUMNS) && !bad && t + NW < ty) {
              if (lane == 0) issue_ycols(p, t + NW);
              xpend = true;
            }
          });
        } else LY::template run<+1, ZMY>(v, gy, rowy, tw1, tcy);
        a_acquire();
        if (ly < nl) {
#pragma unroll
          for (int m = 0; m < EY / LY::RL; ++m)
#pragma unroll
            for (int j = 0; j < LY::RL; ++j)
              if (FFTB_IN(LY::last_pos(gy, m, j) * XP + c0 + ly, abuf, L.status))
                A[LY::last_pos(gy, m, j) * XP + c0 + ly] = v[m * LY::RL + j];
        }
      }
      if constexpr (PF) {
        if (__syncthreads_or(bad)) {
          abort_plane();
          return;
        }
        // the stick row is consumed: fetch the next plane's during the x phase
        const int pn = p + gridDim.x;
        if (threadIdx.x == 0 && pn < nplanes) issue_trow(pn);
        outstanding = pn < nplanes;
      } else if constexpr (YS) {
        if (__syncthreads_or(bad)) {
          // leaving after a failed wait: let this warp's copies in flight land, report
          if (xpend) mbar_wait(xbar + warp, xph, WAIT_LIMIT_NS);
          if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(L.status) = STATUS_WAIT_TIMEOUT;
          return;
        }
      } else {
        __syncthreads();
      }
      // x-DFT (+) of every row, zero-extended from the X occupied columns
#pragma unroll 1
      for (int t = (warp - x_first + NW) % NW; t < tx; t += NW) {
        const int y0 = t * WX, row = y0 + lx;
        const bool live = row < N1;
        C v[EX];
#pragma unroll
        for (int q = 0; q < EX; ++q) {
          if (XQ && x_mid<N0, LX::G, LX::R0>(q)) {  // no occupied x there
            v[q] = czero<C>();
            continue;
          }
          const int xi = xin.get(q);
          v[q] = (live && (allx || xi != 255) && FFTB_IN(row * XP + xi, abuf, L.status)) ? A[row * XP + xi]
                                                                                          : czero<C>();
        }
        if (MODE == M_G2R && t + NW >= tx) a_release();
        if constexpr (TC) LX::template run_tc<+1>(v, gx, rowx, scr, tw0, tcx, wx_p);
        else if constexpr (YS) {
          // after the last exchange of this warp's x phase: the next plane's first y task
          LX::template run2<+1, ZMX>(v, gx, rowx, tw0, tcx, [] {}, [&] {
            if (t + NW >= tx) ys_issue_first(p + gridDim.x, false);
          });
        } else LX::template run<+1, ZMX>(v, gx, rowx, tw0, tcx);
        if constexpr (MODE == M_G2R) {
          if (live && cst == 1) {
            C* out = static_cast<C*>(L.cube_out) + plane + (size_t)row * N0;
            bool done = false;
            if constexpr (LX::PAIR) {
              if (pair16) {  // the paired schedule's (x, x + 1) as 16-byte stores
#pragma unroll
                for (int m = 0; m < EX / LX::RL; m += 2)
#pragma unroll
                  for (int j = 0; j < LX::RL; ++j)
                    if (FFTB_IN(plane + (size_t)row * N0 + LX::last_pos(gx, m, j) + 1, L.lim_cube, L.status))
                      st_pair(out + LX::last_pos(gx, m, j), v[m * LX::RL + j], v[(m + 1) * LX::RL + j]);
                done = true;
              }
            }
            if (!done) {
#pragma unroll
              for (int m = 0; m < EX / LX::RL; ++m)
#pragma unroll
                for (int j = 0; j < LX::RL; ++j)
                  if (FFTB_IN(plane + (size_t)row * N0 + LX::last_pos(gx, m, j), L.lim_cube, L.status))
                    st_once<AG>(out + LX::last_pos(gx, m, j), v[m * LX::RL + j]);
            }
          } else if (live) {  // batch-fastest cube: points B_k apart
            C* out = static_cast<C*>(L.cube_out) + plane + (size_t)row * N0 * cst;
#pragma unroll
            for (int m = 0; m < EX / LX::RL; ++m)
#pragma unroll
              for (int j = 0; j < LX::RL; ++j)
                if (FFTB_IN(plane + (size_t)row * N0 * cst + (size_t)LX::last_pos(gx, m, j) * cst, L.lim_cube, L.status))
                  st_once<AG>(out + (size_t)LX::last_pos(gx, m, j) * cst, v[m * LX::RL + j]);
          }
        } else {
          // V(r) * psi(r), then back to first-pass order and x-DFT (-)
          const T* vr = static_cast<const T*>(L.V) + (size_t)z * (N1 * N0) + (size_t)(live ? row : 0) * N0;
#pragma unroll
          for (int m = 0; m < EX / LX::RL; ++m)
#pragma unroll
            for (int j = 0; j < LX::RL; ++j) {
              const int x = LX::last_pos(gx, m, j);
              const bool vin = FFTB_IN((size_t)z * (N1 * N0) + (size_t)(live ? row : 0) * N0 + x, L.lim_V, L.status);
              rowx[LX::pad(x)] = scale(v[m * LX::RL + j], vin ? __ldg(vr + x) : T(0));
            }
          __syncwarp();
#pragma unroll
          for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
            for (int j = 0; j < LX::R0; ++j) v[m * LX::R0 + j] = rowx[LX::pad(LX::first_pos(gx, m, j))];
          __syncwarp();
          if constexpr (TC) LX::template run_tc<-1>(v, gx, rowx, scr, tw0, tcx, wx_m);
          else LX::template run<-1>(v, gx, rowx, tw0, tcx);
          if (live) {
#pragma unroll
            for (int q = 0; q < EX; ++q) {
              if (XQ && x_mid<N0, LX::G, LX::RL>(q)) continue;  // no occupied x there
              const int xi = xout.get(q);
              if ((allx || xi != 255) && FFTB_IN(row * XP + xi, abuf, L.status)) A[row * XP + xi] = v[q];
            }
          }
        }
      }
    }
    if constexpr (MODE == M_R2G) {
      const bool xs_rows = XS && xs_on && cst == 1;  // uniform
      if (xs_rows) {
        const int t0 = (warp - x_first + NW) % NW;
        if (t0 < tx) {
          // withheld under test injection: the wait below runs out
          const bool withhold = (L.inject & INJECT_SKIP_FIRST_PREFETCH) && blockIdx.x == 0 && warp == 0 &&
                                p == (int)blockIdx.x;
          __syncwarp();
          if (lane == 0 && !withhold) issue_xrows(p, t0);
          xpend = true;
        }
      }
#pragma unroll 1
      for (int t = (warp - x_first + NW) % NW; t < tx; t += NW) {
        const int y0 = t * WX, row = y0 + lx;
        const bool live = row < N1;
        C v[EX];
        if (xs_rows) {
          if (xpend && !bad) {
            const bool ok = mbar_wait(xbar + warp, xph, WAIT_LIMIT_NS);
            if (__any_sync(0xffffffffu, ok)) {
              xpend = false;
              xph ^= 1;
            } else {
              bad = true;
            }
          }
          const C* in = xrows + lx * LX::PITCH;
#pragma unroll
          for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
            for (int j = 0; j < LX::R0; ++j)
              v[m * LX::R0 + j] = live ? in[LX::first_pos(gx, m, j)] : czero<C>();
          __syncwarp();
        } else if constexpr (PF) {
          if (__any_sync(0xffffffffu, outstanding && !bad)) {
            const bool ok = mbar_wait(bars + warp, ph, WAIT_LIMIT_NS);
            if (__any_sync(0xffffffffu, ok)) {
              outstanding = false;
              ph ^= 1;
            } else {
              bad = true;
            }
          }
          const C* in = wst + lx * RP;
#pragma unroll
          for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
            for (int j = 0; j < LX::R0; ++j)
              v[m * LX::R0 + j] = live ? in[LX::first_pos(gx, m, j)] : czero<C>();
          __syncwarp();
          // the rows are in registers: fetch this warp's next x task
          int pn = p, tn = t + NW;
          if (tn >= tx) {
            pn = p + gridDim.x;
            tn = pn < nplanes ? x_start(pn) : 0;
          }
          if (!bad && pn < nplanes) {
            if (lane == 0) issue_rows(pn, tn);
            outstanding = true;
          }
        } else if (cst == 1) {
          const C* in = static_cast<const C*>(L.cube_in) + plane + (size_t)(live ? row : 0) * N0;
#pragma unroll
          for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
            for (int j = 0; j < LX::R0; ++j)
              v[m * LX::R0 + j] =
                  live && FFTB_IN(plane + (size_t)row * N0 + LX::first_pos(gx, m, j), L.lim_cube, L.status)
                      ? ld_once<AG>(in + LX::first_pos(gx, m, j))
                      : czero<C>();
        } else {  // batch-fastest cube: points B_k apart
          const C* in = static_cast<const C*>(L.cube_in) + plane + (size_t)(live ? row : 0) * N0 * cst;
#pragma unroll
          for (int m = 0; m < EX / LX::R0; ++m)
#pragma unroll
            for (int j = 0; j < LX::R0; ++j)
              v[m * LX::R0 + j] =
                  live && FFTB_IN(plane + (size_t)row * N0 * cst + (size_t)LX::first_pos(gx, m, j) * cst, L.lim_cube,
                                  L.status)
                      ? ld_once<AG>(in + (size_t)LX::first_pos(gx, m, j) * cst)
                      : czero<C>();
        }
        if constexpr (TC) LX::template run_tc<-1>(v, gx, rowx, scr, tw0, tcx, wx_m);
        else if constexpr (XS) {
          // once the exchange rows have been read back, fetch this warp's next
          // x task of the plane into them (overlapping the second pass)
          LX::template run2<-1>(v, gx, rowx, tw0, tcx, [] {}, [&] {
            if (xs_rows && !bad && t + NW < tx) {
              if (lane == 0) issue_xrows(p, t + NW);
              xpend = true;
            }
          });
        } else LX::template run<-1>(v, gx, rowx, tw0, tcx);
        a_acquire();
        if (live) {
#pragma unroll
          for (int q = 0; q < EX; ++q) {
            if (XQ && x_mid<N0, LX::G, LX::RL>(q)) continue;  // no occupied x there
            const int xi = xout.get(q);
            if ((allx || xi != 255) && FFTB_IN(row * XP + xi, abuf, L.status)) A[row * XP + xi] = v[q];
          }
        }
      }
    }
    if constexpr (MODE == M_R2G || MODE == M_APPLY) {
      if constexpr (PF && MODE == M_R2G) {
        if (__syncthreads_or(bad)) {
          abort_plane();
          return;
        }
      } else if constexpr (XS && MODE == M_R2G) {
        if (__syncthreads_or(bad)) {
          // leaving after a failed wait: let this warp's copies in flight land, report
          if (xpend) mbar_wait(xbar + warp, xph, WAIT_LIMIT_NS);
          if (threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(L.status) = STATUS_WAIT_TIMEOUT;
          return;
        }
      } else {
        __syncthreads();
      }
      // y-DFT (-) of each occupied column; keep the occupied sticks
#pragma unroll 1
      for (int t = warp; t < ty; t += NW) {
        const int c0 = t * WY, nl = min(WY, X - c0);
        const int col = c0 + (ly < nl ? ly : 0);
        const int4 ci = cinfo[col];
        C v[EY];
#pragma unroll
        for (int m = 0; m < EY / LY::R0; ++m)
#pragma unroll
          for (int j = 0; j < LY::R0; ++j)
            v[m * LY::R0 + j] = FFTB_IN(LY::first_pos(gy, m, j) * XP + col, abuf, L.status)
                                    ? A[LY::first_pos(gy, m, j) * XP + col]
                                    : czero<C>();
        if (t + NW >= ty) a_release();
        if constexpr (TC) LY::template run_tc<-1>(v, gy, rowy, scr, tw1, tcy, wy_m);
        else LY::template run<-1>(v, gy, rowy, tw1, tcy);
        if (ki.flags & KF_CONTIGUOUS_COLUMNS) {
          if (ly < nl) {
            const int sa = ci.x, len = ci.y, ylo = ci.z;
#pragma unroll
            for (int m = 0; m < EY / LY::RL; ++m)
#pragma unroll
              for (int j = 0; j < LY::RL; ++j) {
                if (XQ && x_mid<N1, LY::G, LY::RL>(m * LY::RL + j)) continue;  // no occupied y there
                const int d = ysigned(LY::last_pos(gy, m, j)) - ylo;
                if ((unsigned)d < (unsigned)len && FFTB_IN(tz + sa + d, L.lim_T, L.status)) Tz[sa + d] = v[m * LY::RL + j];
              }
          }
        } else {
#pragma unroll
          for (int m = 0; m < EY / LY::RL; ++m)
#pragma unroll
            for (int j = 0; j < LY::RL; ++j) {
              if (XQ && x_mid<N1, LY::G, LY::RL>(m * LY::RL + j)) continue;  // no stick there
              rowy[LY::pad(LY::last_pos(gy, m, j))] = v[m * LY::RL + j];
            }
          __syncwarp();
          const int sbeg = __shfl_sync(0xffffffffu, ci.x, 0);
          const int send = __shfl_sync(0xffffffffu, ci.x + ci.y, (nl - 1) * LY::G);
          for (int s = sbeg + lane; s < send; s += 32) {
            const int xy = sxy[s];
            if (FFTB_IN(tz + s, L.lim_T, L.status)) Tz[s] = scr[((xy >> 16) - c0) * LY::PITCH + LY::pad(xy & 0xFFFF)];
          }
          __syncwarp();
        }
      }
    }
    if (AG && nbuf == 1) __syncthreads();
    // the end of this plane: warps without a slab-plane read arrive now
    a_release();
    ++a_phase;
    a_got = false;
    a_rel = false;
  }
}

// ---------------------------------------------------------------- dispatch
// lengths whose default FP32 plane kernels have the line-pruned variant (QP)
template <typename T, bool TC, int N> constexpr bool qp_variant() {
  return sizeof(T) == 4 && !TC && (N == 64 || N == 96 || N == 128 || N == 256);
}

// Launches a stage kernel; with L.pdl the launch allows programmatic
// dependent launch (every stage kernel starts with pdl_launch_dependents and
// calls pdl_wait before touching stage data, so neighbours only overlap their
// launch latency and prologues).
template <typename... A, typename... B>
cudaError_t launch_k(void (*kernel)(A...), dim3 grid, dim3 block, size_t smem, const Launch& L, B&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = L.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<B>(args)...);
}

// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes`, never lowering it: plans of one grid size but different
// spheres or buffers share the kernel, and a lower limit set by one plan
// would make another plan's launches fail.
inline cudaError_t raise_smem_limit(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> have;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int& h = have[{dev, fn}];
  if (bytes <= h) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) h = bytes;
  return e;
}

#define FFTB_SIZES(X) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(96) X(128) X(160) X(256)

template <typename T, bool TC> size_t stick_smem_t(int n2) {
  switch (n2) {
#define C_(N) case N: return stick_smem_c<T, N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}
template <typename T, bool TC> size_t plane_smem_t(int n0, int n1, int xmax, int a_bufs, bool ag) {
  if (n0 != n1) return 0;
  switch (n0) {
#define C_(N) case N: return plane_smem_c<T, N, N>(xmax, a_bufs, ag);
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}
// schedule of the default z-stage kernels: FP32 160-point lines on the
// two-pass 40 x 4 schedule (as the pruned ones), the rest their default
template <typename T, bool TC, int N2> constexpr int stick_v() {
  return (sizeof(T) == 4 && !TC && N2 == 160) ? 2 : 0;
}
template <typename T, bool TC> int stick_tile_t(int n2) {
  switch (n2) {
#define C_(N) case N: return stick_tile_c2<N, stick_v<T, TC, N>()>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}

template <typename T, bool TC, int N2> cudaError_t go_stick(int mode, const Launch& L, int ctas) {
  constexpr int V = stick_v<T, TC, N2>();
  const size_t smem = stick_smem_c<T, N2, V>();
  const int gpb = (L.g.smax + (32 / Line<N2, V>::G) - 1) / (32 / Line<N2, V>::G);
  const int need = (L.nb * gpb + STICK_NW - 1) / STICK_NW;  // one task per warp
  const dim3 grid(ctas > 0 ? min(ctas, need) : need);
  if (mode == M_G2R) return launch_k(k_stick<T, N2, M_G2R, TC, V>, grid, STICK_NW * 32, smem, L, L);
  return launch_k(k_stick<T, N2, M_R2G, TC, V>, grid, STICK_NW * 32, smem, L, L);
}
template <typename T, bool TC, int N, bool QP = false> cudaError_t go_plane(int mode, const Launch& L) {
  if constexpr (!QP && qp_variant<T, TC, N>()) {
    if (L.xq) return go_plane<T, TC, N, true>(mode, L);
  }
  if constexpr (N >= 128) {
    if (L.a_glob) {  // slab planes too large for shared memory: per-CTA blocks of a global buffer
      const size_t smem = plane_smem_c<T, N, N>(L.g.xmax, L.a_bufs, true);
      const int nplanes = L.nb * L.g.n2;
      const int ctas = min(min(L.plane_ctas, nplanes), L.a_blocks);  // never more CTAs than slab-plane blocks
      if (ctas < 1) return cudaErrorInvalidValue;
      const dim3 grid(ctas);
      constexpr int NT = PlaneCfg<T>::NW * 32;
      if (mode == M_G2R) return launch_k(k_plane<T, N, N, M_G2R, TC, true, false, 0, QP>, grid, NT, smem, L, L);
      if (mode == M_R2G) return launch_k(k_plane<T, N, N, M_R2G, TC, true, false, 0, QP>, grid, NT, smem, L, L);
      return launch_k(k_plane<T, N, N, M_APPLY, TC, true, false, 0, QP>, grid, NT, smem, L, L);
    }
  }
  if (L.a_glob) return cudaErrorInvalidValue;
  const size_t smem = plane_smem_c<T, N, N>(L.g.xmax, L.a_bufs);
  const int nplanes = L.nb * L.g.n2;
  const dim3 grid(L.plane_ctas > 0 ? min(L.plane_ctas, nplanes) : nplanes);
  constexpr int NT = PlaneCfg<T>::NW * 32;
  if (mode == M_G2R) return launch_k(k_plane<T, N, N, M_G2R, TC, false, false, 0, QP>, grid, NT, smem, L, L);
  if (mode == M_R2G) return launch_k(k_plane<T, N, N, M_R2G, TC, false, false, 0, QP>, grid, NT, smem, L, L);
  return launch_k(k_plane<T, N, N, M_APPLY, TC, false, false, 0, QP>, grid, NT, smem, L, L);
}
template <typename T, bool TC, int N2> cudaError_t prep_stick() {
  constexpr int V = stick_v<T, TC, N2>();
  const int s = (int)stick_smem_c<T, N2, V>();
  cudaError_t e = raise_smem_limit((const void*)k_stick<T, N2, M_G2R, TC, V>, s);
  if (e == cudaSuccess)
    e = raise_smem_limit((const void*)k_stick<T, N2, M_R2G, TC, V>, s);
  return e;
}
template <typename T, bool TC, int N, bool QP = false> cudaError_t prep_plane(int xmax, int a_bufs, bool ag) {
  if constexpr (!QP && qp_variant<T, TC, N>()) {
    cudaError_t e = prep_plane<T, TC, N, true>(xmax, a_bufs, ag);
    if (e != cudaSuccess) return e;
  }
  if constexpr (N >= 128) {
    if (ag) {
      const int s = (int)plane_smem_c<T, N, N>(xmax, a_bufs, true);
      cudaError_t e = raise_smem_limit((const void*)k_plane<T, N, N, M_G2R, TC, true, false, 0, QP>, s);
      if (e == cudaSuccess)
        e = raise_smem_limit((const void*)k_plane<T, N, N, M_R2G, TC, true, false, 0, QP>, s);
      if (e == cudaSuccess)
        e = raise_smem_limit((const void*)k_plane<T, N, N, M_APPLY, TC, true, false, 0, QP>, s);
      return e;
    }
  }
  if (ag) return cudaErrorInvalidValue;
  const int s = (int)plane_smem_c<T, N, N>(xmax, a_bufs);
  cudaError_t e = raise_smem_limit((const void*)k_plane<T, N, N, M_G2R, TC, false, false, 0, QP>, s);
  if (e == cudaSuccess)
    e = raise_smem_limit((const void*)k_plane<T, N, N, M_R2G, TC, false, false, 0, QP>, s);
  if (e == cudaSuccess)
    e = raise_smem_limit((const void*)k_plane<T, N, N, M_APPLY, TC, false, false, 0, QP>, s);
  return e;
}

template <typename T, bool TC, int N, bool QP = false> int occ_plane(int mode, int xmax, int a_bufs, bool ag) {
  constexpr int NT = PlaneCfg<T>::NW * 32;
  int nb = 0;
  cudaError_t e;
  // the line-pruned variant must be resident the same way (the plan sizes one grid for both)
  int nq = 1 << 30;
  if constexpr (!QP && qp_variant<T, TC, N>()) nq = occ_plane<T, TC, N, true>(mode, xmax, a_bufs, ag);
  if constexpr (N >= 128) {
    if (ag) {
      const size_t sm = plane_smem_c<T, N, N>(xmax, a_bufs, true);
      if (mode == M_G2R)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_G2R, TC, true, false, 0, QP>, NT, sm);
      else if (mode == M_R2G)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_R2G, TC, true, false, 0, QP>, NT, sm);
      else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_APPLY, TC, true, false, 0, QP>, NT, sm);
      return e == cudaSuccess ? min(nb, nq) : 0;
    }
  }
  if (ag) return 0;
  const size_t smem = plane_smem_c<T, N, N>(xmax, a_bufs);
  if (mode == M_G2R)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_G2R, TC, false, false, 0, QP>, NT, smem);
  else if (mode == M_R2G)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_R2G, TC, false, false, 0, QP>, NT, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_plane<T, N, N, M_APPLY, TC, false, false, 0, QP>, NT, smem);
  return e == cudaSuccess ? min(nb, nq) : 0;
}
template <typename T, bool TC, int N2> int occ_stick() {
  constexpr int V = stick_v<T, TC, N2>();
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stick<T, N2, M_G2R, TC, V>, STICK_NW * 32,
                                                    stick_smem_c<T, N2, V>()) != cudaSuccess)
    return 0;
  return nb;
}
template <typename T, bool TC> int stick_occupancy_t(int n2) {
  switch (n2) {
#define C_(N) case N: return occ_stick<T, TC, N>();
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}
template <typename T, bool TC> int plane_occupancy_t(int mode, int n0, int n1, int xmax, int a_bufs, bool ag) {
  if (n0 != n1) return 0;
  switch (n0) {
#define C_(N) case N: return occ_plane<T, TC, N>(mode, xmax, a_bufs, ag);
    FFTB_SIZES(C_)
#undef C_
  }
  return 0;
}

template <typename T, bool TC> cudaError_t launch_stick_t(int mode, const Launch& L, int tiles) {
  switch (L.g.n2) {
#define C_(N) case N: return go_stick<T, TC, N>(mode, L, tiles);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}
template <typename T, bool TC> cudaError_t launch_plane_t(int mode, const Launch& L) {
  if (L.g.n0 != L.g.n1) return cudaErrorInvalidValue;
  switch (L.g.n0) {
#define C_(N) case N: return go_plane<T, TC, N>(mode, L);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}
template <typename T, bool TC> cudaError_t prepare_t(int n0, int n1, int n2, int xmax, int a_bufs, bool ag) {
  cudaError_t e = cudaErrorInvalidValue;
  switch (n2) {
#define C_(N) case N: e = prep_stick<T, TC, N>(); break;
    FFTB_SIZES(C_)
#undef C_
  }
  if (e != cudaSuccess || n0 != n1) return e == cudaSuccess ? cudaErrorInvalidValue : e;
  switch (n0) {
#define C_(N) case N: return prep_plane<T, TC, N>(xmax, a_bufs, ag);
    FFTB_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

#define FFTB_INSTANTIATE(T, TC)                                                    \
  template size_t stick_smem_t<T, TC>(int);                                        \
  template size_t plane_smem_t<T, TC>(int, int, int, int, bool);                   \
  template int stick_tile_t<T, TC>(int);                                           \
  template cudaError_t launch_stick_t<T, TC>(int, const Launch&, int);             \
  template cudaError_t launch_plane_t<T, TC>(int, const Launch&);                  \
  template cudaError_t prepare_t<T, TC>(int, int, int, int, int, bool);            \
  template int plane_occupancy_t<T, TC>(int, int, int, int, int, bool);            \
  template int stick_occupancy_t<T, TC>(int);

}  // namespace fftb
