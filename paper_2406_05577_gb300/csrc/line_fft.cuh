// line_fft.cuh -- register-resident 1D DFTs of whole lines, G lanes per line.
//
// A length-N line is held by G = N / E lanes, E elements each. The DFT is
// factored Cooley-Tukey style (Sec. 2.1) into Stockham passes whose radices
// all divide E, so in every pass each lane owns E / R whole butterflies:
// butterfly m of lane g is i = g + m G (the paired variant's last pass:
// i = 2 G (m / 2) + 2 g + m mod 2); its inputs sit at i + j N/R. The
// lane->butterfly map is fixed, so every address below is a per-lane base plus
// a compile-time offset. Between passes the lanes of a line exchange values
// through a private shared-memory row of the warp (one pad element after
// every 8, so stride-R stores fall on distinct banks; the paired variant two
// after every R0); a line held by a single lane (G = 1) exchanges by register
// renaming only.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "fft_core.cuh"

namespace fftb {

// smallest row pitch >= n that is 8 (mod 16) elements (paired exchange rows)
__host__ __device__ constexpr int pair_pitch(int n) { return n + ((8 - n % 16) + 16) % 16; }

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
FFTB_LP(64, 8, 8, 8, 0, 0);  // measured best of 8x8, 16x4 (E=16) and 4x16 (E=16)
FFTB_LP(96, 12, 6, 4, 4, 0);
FFTB_LP(128, 16, 16, 8, 0, 0);
FFTB_LP(160, 20, 4, 4, 2, 5);
FFTB_LP(256, 16, 16, 16, 0, 0);
#undef FFTB_LP

// Schedule variants the autotuner may pick instead (V = 1): a different
// radix order or element count per lane for the same length.
template <int N, int V> struct LPV : LP<N> {};
template <int N> struct has_alt_schedule { static constexpr bool value = false; };
#define FFTB_LPV(N_, E_, R0, R1, R2, R3)                                      \
  template <> struct LPV<N_, 1> {                                           \
    static constexpr int E = E_;                                            \
    static constexpr int R[4] = {R0, R1, R2, R3};                           \
  };                                                                        \
  template <> struct has_alt_schedule<N_> { static constexpr bool value = true; }
FFTB_LPV(64, 16, 16, 4, 0, 0);
FFTB_LPV(96, 24, 12, 8, 0, 0);
FFTB_LPV(128, 16, 8, 16, 0, 0);
FFTB_LPV(160, 20, 10, 4, 4, 0);
#undef FFTB_LPV
// Two-pass schedules for the plane stages: a composite DFT of the whole E in
// registers, one exchange, then radix-G butterflies on G = N / E lanes.
template <> struct LPV<160, 2> {
  static constexpr int E = 40;
  static constexpr int R[4] = {40, 4, 0, 0};
};
// the same schedule for the plane kernels that drop the middle half of each
// x line (every occupied x within [-N/4, N/4])
template <> struct LPV<160, 3> : LPV<160, 2> {};
// V = 4: the 40 x 4 schedule with paired ownership for lines whose outputs
// leave in 16-byte pairs (FP32): after the exchange each lane holds the
// radix-4 butterflies of two adjacent positions (k1 = 2 G q + 2 g + b), so
// every output pair (x, x + 1) is in one lane. The exchange rows put two pad
// elements after every 40 (pitch 8 (mod 16)), so that the pass-0 stores
// (pairs of consecutive outputs of a lane) and the pass-1 loads (a lane's two
// positions) are 16-byte accesses that hit every bank of a quarter warp once.
template <> struct LPV<160, 4> : LPV<160, 2> {
  static constexpr bool PAIR = true;
};
template <typename P, typename = void> struct lpv_pair { static constexpr bool value = false; };
template <typename P> struct lpv_pair<P, std::void_t<decltype(P::PAIR)>> { static constexpr bool value = P::PAIR; };

// ----------------------------------------------------------- tensor cores
// A radix-8 pass as a dense product on the tensor cores (split precision):
// 16 butterflies (rows) x 8 complex inputs = a 16 x 16 real matrix A, the
// DFT8 matrix as a 16 x 16 real matrix W (real index 2 j + re/im), one
// mma.sync.m16n8k16 per 8 output columns. A and W are split into FP16 hi + lo
// parts (x = hi + lo + O(2^-22 x)); D = A_hi W_hi + A_hi W_lo + A_lo W_hi is
// accumulated in FP32. Each row is scaled by a power of two first so that its
// largest component lies in [2^13, 2^14) (inside FP16 range, lo parts normal),
// and unscaled exactly afterwards.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
// split (x, y) into packed FP16 hi and lo
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x, y);
  const float2 hf = __half22float2(h);
  hi = h2u(h);
  lo = h2u(__floats2half2_rn(x - hf.x, y - hf.y));
}
// 2^e such that m * 2^e < 2^15 (m >= 0), and its inverse
__device__ __forceinline__ void row_scale(float m, float& s, float& inv) {
  int ex = (__float_as_int(m) >> 23) & 0xFF;      // biased exponent of m
  int es = 141 - ex + 127;                        // 2^(14 - (ex - 127)), biased
  es = es < 1 ? 1 : (es > 254 ? 254 : es);
  s = __int_as_float(es << 23);
  inv = __int_as_float((254 - es) << 23);         // 2^-(es - 127)
}

template <int N, int V = 0> struct Line {
  using LPN = LPV<N, V>;
  static constexpr int E = LPN::E;
  static constexpr int G = N / E;
  static constexpr int NP = LPN::R[1] == 0 ? 1 : LPN::R[2] == 0 ? 2 : LPN::R[3] == 0 ? 3 : 4;
  static constexpr int R0 = LPN::R[0];
  static constexpr int RL = LPN::R[NP - 1];
  // paired ownership (two passes, one first-pass butterfly a lane, FP32 rows)
  static constexpr bool PAIR = lpv_pair<LPN>::value;
  static_assert(!PAIR || (NP == 2 && E == R0 && (E / LPN::R[1]) % 2 == 0 && (N / LPN::R[1]) % (2 * G) == 0),
                "paired ownership: two passes, one first-pass butterfly, pairs of second-pass butterflies");
  // exchange-row pad: one element after every 8, or (PAIR) two after every R0
  __host__ __device__ static constexpr int pad(int e) { return PAIR ? e + 2 * (e / R0) : e + (e >> 3); }
  static constexpr int PITCH = PAIR ? pair_pitch(N + 2 * (N / R0)) : wpitch(N, G);
  static_assert(32 % G == 0, "lanes per line must divide the warp");
  static_assert(R0 * (NP > 1 ? LPN::R[1] : 1) * (NP > 2 ? LPN::R[2] : 1) * (NP > 3 ? LPN::R[3] : 1) == N,
                "radix schedule must multiply to N");

  // the index of butterfly m of lane g in the last pass (PAIR: pairs of adjacent indices)
  __host__ __device__ static constexpr int bfly(int g, int m) {
    return PAIR ? 2 * G * (m >> 1) + 2 * g + (m & 1) : g + m * G;
  }
  // position of v[m * R0 + j] before run(), and of v[m * RL + j] after it
  __device__ __forceinline__ static int first_pos(int g, int m, int j) { return g + m * G + j * (N / R0); }
  __device__ __forceinline__ static int last_pos(int g, int m, int j) {
    return (NP == 1 ? g + m * G : bfly(g, m)) + j * (N / RL);
  }

  template <int p> __host__ __device__ static constexpr int radix() { return LPN::R[p]; }
  template <int p> __host__ __device__ static constexpr int span() {  // product of radices before p
    int s = 1;
    for (int q = 0; q < p; ++q) s *= LPN::R[q];
    return s;
  }

  // Pass 1's twiddles depend only on the lane when G is a multiple of its
  // span (k = g mod P for every butterfly of the lane): TwCache keeps those
  // R - 1 values in registers for the whole kernel.
  static constexpr bool CACHE1 = NP > 1 && (G % span<1>() == 0);
  template <typename C> struct TwCache {
    C w[CACHE1 ? LPN::R[1] - 1 : 1];
    __device__ __forceinline__ void load(int g, const C* __restrict__ tw) {
      if constexpr (CACHE1) {
        constexpr int R = radix<1>(), P = span<1>(), STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) w[j - 1] = tw[j * (g % P) * STEP];
      }
    }
  };

  // twiddle + radix-R butterflies of pass p on the lane's registers (ZM: the
  // inputs of pass 0 known to be zero, bit q for v[q])
  template <int p, int S, unsigned long long ZM = 0, typename C>
  __device__ __forceinline__ static void compute(C (&v)[E], int g, const C* __restrict__ tw,
                                                 const TwCache<C>& tc) {
    constexpr int R = radix<p>(), P = span<p>();
#pragma unroll
    for (int m = 0; m < E / R; ++m) {
      if constexpr (P > 1) {
        const int k = (p == NP - 1 ? bfly(g, m) : g + m * G) % P;
        constexpr int STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) {
          C w;
          if constexpr (p == 1 && CACHE1) w = tc.w[j - 1];
          else w = tw[j * k * STEP];
          v[m * R + j] = (S > 0) ? cmul(v[m * R + j], w) : cmulc(v[m * R + j], w);
        }
      }
      if constexpr (!(p == 0 && ZM != 0)) dft<R, S>(&v[m * R]);
    }
    if constexpr (p == 0 && ZM != 0) first_z<S, ZM, 0>(v);
  }
  // pass 0 with the inputs of ZM known to be zero: butterfly M takes bits
  // M R .. M R + R - 1 (no twiddles before the first pass)
  template <int S, unsigned long long ZM, int M, typename C> __device__ __forceinline__ static void first_z(C (&v)[E]) {
    constexpr int R = radix<0>();
    if constexpr (M < E / R) {
      dft_z<R, S, (ZM >> (M * R)) & (R >= 64 ? ~0ull : (1ull << R) - 1)>(&v[M * R]);
      first_z<S, ZM, M + 1>(v);
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
    } else if constexpr (PAIR) {
      // lane g's outputs (positions g R + j) in 16-byte pairs, then its two
      // butterflies' inputs (positions 2 G q + 2 g + {0, 1} + j N / R2) likewise
      static_assert(sizeof(C) == 8 && p == 0, "paired exchange: FP32, the one exchange");
#pragma unroll
      for (int j = 0; j < R; j += 2)
        *reinterpret_cast<float4*>(row + pad(g * R + j)) = make_float4(v[j].x, v[j].y, v[j + 1].x, v[j + 1].y);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < E / R2; m += 2)
#pragma unroll
        for (int j = 0; j < R2; ++j) {
          const float4 t = *reinterpret_cast<const float4*>(row + pad(bfly(g, m) + j * NB2));
          v[m * R2 + j] = mk(t.x, t.y);
          v[(m + 1) * R2 + j] = mk(t.z, t.w);
        }
      __syncwarp();
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

  template <int p, int S, unsigned long long ZM = 0, typename C>
  __device__ __forceinline__ static void passes(C (&v)[E], int g, C* __restrict__ row, const C* __restrict__ tw,
                                                const TwCache<C>& tc) {
    compute<p, S, ZM>(v, g, tw, tc);
    if constexpr (p + 1 < NP) {
      exchange<p>(v, g, row);
      passes<p + 1, S>(v, g, row, tw, tc);
    }
  }

  // ---- tensor-core radix-8 pass (MIXED_TC precision)
  // W fragments of this lane (B operand, col layout): n-tile nt covers output
  // columns 2 k' + c' for k' in [4 nt, 4 nt + 4); lane holds rows k = 2 t, 2 t + 1,
  // 2 t + 8, 2 t + 9 (t = lane & 3) of column n = lane >> 2.
  template <int S> struct TcW {
    uint32_t hi[2][2], lo[2][2];
    __device__ __forceinline__ void load(const float2* __restrict__ tw) {
      const int lane = threadIdx.x & 31, t = lane & 3, gq = lane >> 2;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int kp = 4 * nt + (gq >> 1), cp = gq & 1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = t + 4 * h;
          const float2 w = tw[((j * kp) & 7) * (N / 8)];   // e^{+2 pi i j k'/8}
          const float wr = w.x, wi = float(S) * w.y;
          // rows k = 2 j (re input), 2 j + 1 (im input) of column (k', c')
          const float e0 = cp == 0 ? wr : wi;        // re input -> re out: wr ; -> im out: wi
          const float e1 = cp == 0 ? -wi : wr;       // im input -> re out: -wi; -> im out: wr
          split2(e0, e1, hi[nt][h], lo[nt][h]);
        }
      }
    }
  };

  // Pass p (radix 8) for all WL = 32 / G lines of the warp, in place in the
  // warp's scratch rows (base = first row). Inputs and outputs stay where the
  // Stockham pass would read and write them.
  template <int p, int S>
  __device__ __forceinline__ static void tc_pass(float2* base, const float2* __restrict__ tw, const TcW<S>& W) {
    static_assert(radix<p>() == 8, "tensor-core pass is radix 8");
    constexpr int P = span<p>(), NB = N / 8, WL = 32 / G, TILES = WL * NB / 16, STEP = N / (P * 8);
    static_assert((WL * NB) % 16 == 0, "butterflies per warp must fill 16-row tiles");
    const int lane = threadIdx.x & 31, t = lane & 3, gq = lane >> 2;
    float2 x[TILES][2][2];  // [tile][row half][input j = t + 4 h]
#pragma unroll
    for (int ti = 0; ti < TILES; ++ti)
#pragma unroll
      for (int rh = 0; rh < 2; ++rh) {
        const int b = 16 * ti + gq + 8 * rh, line = b / NB, i = b - line * NB;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = t + 4 * h;
          float2 val = base[line * PITCH + wpad(i + j * NB)];
          if constexpr (P > 1) {
            const float2 w = tw[j * (i % P) * STEP];
            val = (S > 0) ? cmul(val, w) : cmulc(val, w);
          }
          x[ti][rh][h] = val;
        }
      }
    __syncwarp();
#pragma unroll
    for (int ti = 0; ti < TILES; ++ti) {
      float s[2], inv[2];
#pragma unroll
      for (int rh = 0; rh < 2; ++rh) {
        float m = fmaxf(fmaxf(fabsf(x[ti][rh][0].x), fabsf(x[ti][rh][0].y)),
                        fmaxf(fabsf(x[ti][rh][1].x), fabsf(x[ti][rh][1].y)));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        row_scale(m, s[rh], inv[rh]);
      }
      uint32_t ah[4], al[4];
      split2(x[ti][0][0].x * s[0], x[ti][0][0].y * s[0], ah[0], al[0]);   // row gq,     j = t
      split2(x[ti][1][0].x * s[1], x[ti][1][0].y * s[1], ah[1], al[1]);   // row gq + 8, j = t
      split2(x[ti][0][1].x * s[0], x[ti][0][1].y * s[0], ah[2], al[2]);   // row gq,     j = t + 4
      split2(x[ti][1][1].x * s[1], x[ti][1][1].y * s[1], ah[3], al[3]);   // row gq + 8, j = t + 4
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(d, ah, W.hi[nt][0], W.hi[nt][1]);
        mma16816(d, ah, W.lo[nt][0], W.lo[nt][1]);
        mma16816(d, al, W.hi[nt][0], W.hi[nt][1]);
        const int kp = 4 * nt + t;  // output complex index held by this lane
#pragma unroll
        for (int rh = 0; rh < 2; ++rh) {
          const int b = 16 * ti + gq + 8 * rh, line = b / NB, i = b - line * NB, k = i % P;
          base[line * PITCH + wpad((i - k) * 8 + k + kp * P)] = make_float2(d[2 * rh] * inv[rh], d[2 * rh + 1] * inv[rh]);
        }
      }
    }
  }

  // positions the lane loads for pass q (q = NP means the final last_pos order)
  template <int q, typename C>
  __device__ __forceinline__ static void load_for(C (&v)[E], int g, const C* row) {
    if constexpr (q < NP) {
      constexpr int Rq = radix<q>(), NBq = N / Rq;
#pragma unroll
      for (int m = 0; m < E / Rq; ++m)
#pragma unroll
        for (int j = 0; j < Rq; ++j) v[m * Rq + j] = row[wpad(g + m * G + j * NBq)];
    } else {
#pragma unroll
      for (int m = 0; m < E / RL; ++m)
#pragma unroll
        for (int j = 0; j < RL; ++j) v[m * RL + j] = row[wpad(last_pos(g, m, j))];
    }
  }
  // store pass p's outputs (lane layout) where the Stockham pass puts them
  template <int p, typename C>
  __device__ __forceinline__ static void store_out(const C (&v)[E], int g, C* row) {
    constexpr int R = radix<p>(), P = span<p>();
#pragma unroll
    for (int m = 0; m < E / R; ++m) {
      const int i = g + m * G, k = i % P;
#pragma unroll
      for (int j = 0; j < R; ++j) row[wpad((i - k) * R + k + j * P)] = v[m * R + j];
    }
  }

  // row (the lane's line) lies inside the warp's scratch that starts at base:
  // the two alias, so neither is __restrict__.
  template <int p, int S>
  __device__ __forceinline__ static void tc_passes(float2 (&v)[E], int g, float2* row, float2* base,
                                                   const float2* __restrict__ tw, const TwCache<float2>& tc,
                                                   const TcW<S>& W) {
    if constexpr (radix<p>() == 8 && G > 1) {
      if constexpr (p == 0) {
#pragma unroll
        for (int m = 0; m < E / R0; ++m)
#pragma unroll
          for (int j = 0; j < R0; ++j) row[wpad(first_pos(g, m, j))] = v[m * R0 + j];
        __syncwarp();
      }
      tc_pass<p, S>(base, tw, W);
      __syncwarp();
      load_for<p + 1>(v, g, row);
      __syncwarp();
      if constexpr (p + 1 < NP) tc_passes<p + 1, S>(v, g, row, base, tw, tc, W);
    } else {
      compute<p, S>(v, g, tw, tc);
      if constexpr (p + 1 < NP) {
        store_out<p>(v, g, row);
        __syncwarp();
        if constexpr (!(radix<p + 1>() == 8 && G > 1)) {
          load_for<p + 1>(v, g, row);
          __syncwarp();
        }
        tc_passes<p + 1, S>(v, g, row, base, tw, tc, W);
      }
    }
  }

  // As run(), with every radix-8 pass on the tensor cores (MIXED_TC).
  // base = the warp's first scratch row; W = TcW<S>::load for this table.
  template <int S>
  __device__ __forceinline__ static void run_tc(float2 (&v)[E], int g, float2* row, float2* base,
                                                const float2* __restrict__ tw, const TwCache<float2>& tc,
                                                const TcW<S>& W) {
    tc_passes<0, S>(v, g, row, base, tw, tc, W);
  }

  // v in first_pos order -> DFT (sign S) in last_pos order. All lanes of the
  // warp must call it (it synchronises the warp when G > 1). tc holds this
  // lane's pass-1 twiddles (TwCache::load with the same g and table).
  // ZM: inputs known to be zero (bit q: v[q] of the first-pass order)
  template <int S, unsigned long long ZM = 0, typename C>
  __device__ __forceinline__ static void run(C (&v)[E], int g, C* __restrict__ row, const C* __restrict__ tw,
                                             const TwCache<C>& tc) {
    passes<0, S, ZM>(v, g, row, tw, tc);
  }

  // As run() for a two-pass schedule, with two hooks around its one exchange:
  // before() runs (on every lane) before the exchange rows are written,
  // after() once every lane has read them back (the rows are free again).
  template <int S, unsigned long long ZM = 0, typename C, typename B, typename A>
  __device__ __forceinline__ static void run2(C (&v)[E], int g, C* __restrict__ row, const C* __restrict__ tw,
                                              const TwCache<C>& tc, B&& before, A&& after) {
    static_assert(NP == 2 && G > 1, "one exchange between two passes");
    compute<0, S, ZM>(v, g, tw, tc);
    before();
    exchange<0>(v, g, row);
    after();
    compute<1, S>(v, g, tw, tc);
  }
};

}  // namespace fftb
