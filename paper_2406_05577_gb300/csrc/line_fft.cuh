// line_fft.cuh -- register-resident 1D DFTs of whole lines, G lanes per line.
//
// A length-N line is held by G = N / E lanes, E elements each. The DFT is
// factored Cooley-Tukey style (Sec. 2.1) into Stockham passes whose radices
// all divide E, so in every pass each lane owns E / R whole butterflies:
// butterfly m of lane g is i = g + m G; its inputs sit at i + j N/R. The
// lane->butterfly map is fixed, so every address below is a per-lane base plus
// a compile-time offset. Between passes the lanes of a line exchange values
// through a private shared-memory row of the warp (one pad element after
// every 8, so stride-R stores fall on distinct banks); a line held by a single
// lane (G = 1) exchanges by register renaming only.
#pragma once

#include "fft_core.cuh"

namespace fftb {

// E and the radix schedule of each supported length.
template <int N> struct LP;
#define FFTB_LP(N_, E_, R0, R1, R2, R3)                 \
  template <> struct LP<N_> {                           \
    static constexpr int E = E_;                        \
    static constexpr int R[4] = {R0, R1, R2, R3};       \
  }
FFTB_LP(12, 12, 4, 3, 0, 0);
FFTB_LP(16, 16, 16, 0, 0, 0);
FFTB_LP(20, 20, 4, 5, 0, 0);
FFTB_LP(24, 12, 6, 4, 0, 0);
FFTB_LP(32, 16, 16, 2, 0, 0);
FFTB_LP(40, 20, 4, 5, 2, 0);
FFTB_LP(48, 12, 6, 4, 2, 0);
FFTB_LP(64, 8, 8, 8, 0, 0);
FFTB_LP(96, 12, 6, 4, 4, 0);
FFTB_LP(128, 16, 16, 8, 0, 0);
FFTB_LP(160, 20, 4, 4, 2, 5);
#undef FFTB_LP

template <int N> struct Line {
  static constexpr int E = LP<N>::E;
  static constexpr int G = N / E;
  static constexpr int NP = LP<N>::R[1] == 0 ? 1 : LP<N>::R[2] == 0 ? 2 : LP<N>::R[3] == 0 ? 3 : 4;
  static constexpr int R0 = LP<N>::R[0];
  static constexpr int RL = LP<N>::R[NP - 1];
  static constexpr int PITCH = wpitch(N);
  static_assert(32 % G == 0, "lanes per line must divide the warp");
  static_assert(R0 * (NP > 1 ? LP<N>::R[1] : 1) * (NP > 2 ? LP<N>::R[2] : 1) * (NP > 3 ? LP<N>::R[3] : 1) == N,
                "radix schedule must multiply to N");

  // position of v[m * R0 + j] before run(), and of v[m * RL + j] after it
  __device__ __forceinline__ static int first_pos(int g, int m, int j) { return g + m * G + j * (N / R0); }
  __device__ __forceinline__ static int last_pos(int g, int m, int j) { return g + m * G + j * (N / RL); }

  template <int p> __host__ __device__ static constexpr int radix() { return LP<N>::R[p]; }
  template <int p> __host__ __device__ static constexpr int span() {  // product of radices before p
    int s = 1;
    for (int q = 0; q < p; ++q) s *= LP<N>::R[q];
    return s;
  }

  // Pass 1's twiddles depend only on the lane when G is a multiple of its
  // span (k = g mod P for every butterfly of the lane): TwCache keeps those
  // R - 1 values in registers for the whole kernel.
  static constexpr bool CACHE1 = NP > 1 && (G % span<1>() == 0);
  template <typename C> struct TwCache {
    C w[CACHE1 ? LP<N>::R[1] - 1 : 1];
    __device__ __forceinline__ void load(int g, const C* __restrict__ tw) {
      if constexpr (CACHE1) {
        constexpr int R = radix<1>(), P = span<1>(), STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) w[j - 1] = tw[j * (g % P) * STEP];
      }
    }
  };

  // twiddle + radix-R butterflies of pass p on the lane's registers
  template <int p, int S, typename C>
  __device__ __forceinline__ static void compute(C (&v)[E], int g, const C* __restrict__ tw,
                                                 const TwCache<C>& tc) {
    constexpr int R = radix<p>(), P = span<p>();
#pragma unroll
    for (int m = 0; m < E / R; ++m) {
      if constexpr (P > 1) {
        const int k = (g + m * G) % P;
        constexpr int STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) {
          C w;
          if constexpr (p == 1 && CACHE1) w = tc.w[j - 1];
          else w = tw[j * k * STEP];
          v[m * R + j] = (S > 0) ? cmul(v[m * R + j], w) : cmulc(v[m * R + j], w);
        }
      }
      dft<R, S>(&v[m * R]);
    }
  }

  // move pass p's outputs into pass p+1's input order
  template <int p, typename C>
  __device__ __forceinline__ static void exchange(C (&v)[E], int g, C* __restrict__ row) {
    constexpr int R = radix<p>(), P = span<p>(), R2 = radix<p + 1>(), NB2 = N / R2;
    if constexpr (G == 1) {
      C t[E];
#pragma unroll
      for (int m = 0; m < E / R; ++m) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int i = m, k = i % P;
          t[(i - k) * R + k + j * P] = v[m * R + j];
        }
      }
#pragma unroll
      for (int m = 0; m < E / R2; ++m)
#pragma unroll
        for (int j = 0; j < R2; ++j) v[m * R2 + j] = t[m + j * NB2];
    } else {
#pragma unroll
      for (int m = 0; m < E / R; ++m) {
        const int i = g + m * G, k = i % P;
#pragma unroll
        for (int j = 0; j < R; ++j) row[wpad((i - k) * R + k + j * P)] = v[m * R + j];
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < E / R2; ++m)
#pragma unroll
        for (int j = 0; j < R2; ++j) v[m * R2 + j] = row[wpad(g + m * G + j * NB2)];
      __syncwarp();
    }
  }

  template <int p, int S, typename C>
  __device__ __forceinline__ static void passes(C (&v)[E], int g, C* __restrict__ row, const C* __restrict__ tw,
                                                const TwCache<C>& tc) {
    compute<p, S>(v, g, tw, tc);
    if constexpr (p + 1 < NP) {
      exchange<p>(v, g, row);
      passes<p + 1, S>(v, g, row, tw, tc);
    }
  }

  // v in first_pos order -> DFT (sign S) in last_pos order. All lanes of the
  // warp must call it (it synchronises the warp when G > 1). tc holds this
  // lane's pass-1 twiddles (TwCache::load with the same g and table).
  template <int S, typename C>
  __device__ __forceinline__ static void run(C (&v)[E], int g, C* __restrict__ row, const C* __restrict__ tw,
                                             const TwCache<C>& tc) {
    passes<0, S>(v, g, row, tw, tc);
  }
};

}  // namespace fftb
