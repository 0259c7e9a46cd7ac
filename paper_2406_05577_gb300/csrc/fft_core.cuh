// fft_core.cuh -- register codelets and shared-memory Stockham passes for the
// batched 1D DFTs of the staged sphere <-> cube transform.
//
// A 1D DFT of length N (Sec. 2.1: y = DFT_n x, omega_n = e^{-j 2 pi/n}; the
// G -> r direction uses the conjugate root, Sec. 2.2) is factored
// Cooley-Tukey style (N = R_0 R_1 ... R_{P-1}, Sec. 2.1) into Stockham
// autosort passes. Pass p with radix R reads R inputs spaced N/R apart,
// twiddles them by w^{j k} (k = butterfly index mod L, L = R_0...R_{p-1},
// w = e^{s 2 pi j/(L R)}), runs a radix-R DFT in registers and writes the R
// outputs spaced L apart at (i - k) R + k. After the last pass the data are
// in natural order.
//
// Many independent lines run together. Every thread of the CTA takes
// (line, butterfly) work items; a pass first loads all of its items into
// registers, synchronises, then computes and stores, so a pass may work in
// place on a shared-memory buffer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftb {

// ------------------------------------------------------------ complex math
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// a * (S j), S = +1 or -1
template <int S, typename C> __device__ __forceinline__ C mulj(C a) {
  return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}
template <typename C, typename T> __device__ __forceinline__ C scale(C a, T s) {
  return mk(a.x * s, a.y * s);
}
template <typename C> __device__ __forceinline__ C czero() { return mk(decltype(C::x)(0), decltype(C::x)(0)); }

// ------------------------------------------------------------- codelets
// In-place radix-R DFT y_k = sum_j x_j e^{S 2 pi j jk / R}, natural order.
// The constants are cos/sin of 2 pi m / R written out from their closed forms.
template <int S, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a - b;
  a = a + b;
  b = t;
}

template <int S, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C t0 = x0 + x2, t1 = x0 - x2, t2 = x1 + x3, t3 = mulj<S>(x1 - x3);
  x0 = t0 + t2;
  x2 = t0 - t2;
  x1 = t1 + t3;
  x3 = t1 - t3;
}

template <int S, typename C> __device__ __forceinline__ void dft3(C& x0, C& x1, C& x2) {
  using T = decltype(C::x);
  const T c1 = T(-0.5);                                   // cos(2 pi/3)
  const T s1 = T(S) * T(0.86602540378443864676372317);   // S sin(2 pi/3) = S sqrt(3)/2
  C t1 = x1 + x2, t2 = x1 - x2;
  C a = x0 + scale(t1, c1);
  C b = mulj<1>(scale(t2, s1));
  x0 = x0 + t1;
  x1 = a + b;
  x2 = a - b;
}

template <int S, typename C> __device__ __forceinline__ void dft5(C& x0, C& x1, C& x2, C& x3, C& x4) {
  using T = decltype(C::x);
  const T c1 = T(0.30901699437494742410229342);          // cos(2 pi/5) = (sqrt5 - 1)/4
  const T c2 = T(-0.80901699437494742410229342);         // cos(4 pi/5) = -(sqrt5 + 1)/4
  const T s1 = T(S) * T(0.95105651629515357211643933);   // sin(2 pi/5)
  const T s2 = T(S) * T(0.58778525229247312916870595);   // sin(4 pi/5)
  C t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3;
  C a1 = x0 + scale(t1, c1) + scale(t2, c2);
  C a2 = x0 + scale(t1, c2) + scale(t2, c1);
  C b1 = mulj<1>(scale(t3, s1) + scale(t4, s2));
  C b2 = mulj<1>(scale(t3, s2) - scale(t4, s1));
  x0 = x0 + t1 + t2;
  x1 = a1 + b1;
  x4 = a1 - b1;
  x2 = a2 + b2;
  x3 = a2 - b2;
}

template <int S, typename C> __device__ __forceinline__ void dft8(C* v) {
  using T = decltype(C::x);
  const T h = T(0.70710678118654752440084436);           // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  // o1 *= (1 + S j)/sqrt2, o2 *= S j, o3 *= (-1 + S j)/sqrt2
  o1 = scale(o1 + mulj<S>(o1), h);
  o2 = mulj<S>(o2);
  o3 = scale(mulj<S>(o3) - o3, h);
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}

// radix 6 = 3 x 2 (Cooley-Tukey): DFT3 of the even and odd inputs, twiddle
// the odd outputs by W6^k1, then radix-2 butterflies.
template <int S, typename C> __device__ __forceinline__ void dft6(C* v) {
  using T = decltype(C::x);
  const T h = T(0.5), r = T(S) * T(0.86602540378443864676372317);  // W6 = 1/2 + S j sqrt3/2
  C a0 = v[0], a1 = v[2], a2 = v[4], b0 = v[1], b1 = v[3], b2 = v[5];
  dft3<S>(a0, a1, a2);
  dft3<S>(b0, b1, b2);
  b1 = mk(b1.x * h - b1.y * r, b1.x * r + b1.y * h);   // * W6^1
  b2 = mk(-b2.x * h - b2.y * r, b2.x * r - b2.y * h);  // * W6^2 = -1/2 + S j sqrt3/2
  v[0] = a0 + b0; v[3] = a0 - b0;
  v[1] = a1 + b1; v[4] = a1 - b1;
  v[2] = a2 + b2; v[5] = a2 - b2;
}

// radix 16 = 4 x 4: DFT4 over n1 for each n2 (inputs 4 n1 + n2), twiddle by
// W16^(n2 k1), DFT4 over n2, outputs k1 + 4 k2.
template <int S, typename C> __device__ __forceinline__ void dft16(C* v) {
  using T = decltype(C::x);
  const T c1 = T(0.92387953251128675612818319);  // cos(pi/8)
  const T s1 = T(0.38268343236508977172845998);  // sin(pi/8)
  const T h = T(0.70710678118654752440084436);   // cos(pi/4)
  C y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C a = v[n2], b = v[4 + n2], c = v[8 + n2], d = v[12 + n2];
    dft4<S>(a, b, c, d);
    y[n2][0] = a; y[n2][1] = b; y[n2][2] = c; y[n2][3] = d;
  }
  // W16^m = cos(2 pi m/16) + S j sin(2 pi m/16)
  auto w = [&](C a, T cr, T si) { return mk(a.x * cr - a.y * (T(S) * si), a.x * (T(S) * si) + a.y * cr); };
  y[1][1] = w(y[1][1], c1, s1);  y[1][2] = w(y[1][2], h, h);   y[1][3] = w(y[1][3], s1, c1);
  y[2][1] = w(y[2][1], h, h);    y[2][2] = mulj<S>(y[2][2]);   y[2][3] = w(y[2][3], -h, h);
  y[3][1] = w(y[3][1], s1, c1);  y[3][2] = w(y[3][2], -h, h);  y[3][3] = w(y[3][3], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = y[0][k1], b = y[1][k1], c = y[2][k1], d = y[3][k1];
    dft4<S>(a, b, c, d);
    v[k1] = a; v[k1 + 4] = b; v[k1 + 8] = c; v[k1 + 12] = d;
  }
}

// radix 10 = 2 x 5 (Cooley-Tukey): DFT5 of the even and of the odd inputs,
// twiddle the odd outputs by W10^k, then radix-2 butterflies (W10^(k+5) = -W10^k).
template <int S, typename C> __device__ __forceinline__ void dft10(C* v) {
  using T = decltype(C::x);
  const T c1 = T(0.80901699437494742410229342), s1 = T(0.58778525229247312916870595);  // 36 degrees
  const T c2 = T(0.30901699437494742410229342), s2 = T(0.95105651629515357211643933);  // 72 degrees
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], e4 = v[8];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7], o4 = v[9];
  dft5<S>(e0, e1, e2, e3, e4);
  dft5<S>(o0, o1, o2, o3, o4);
  // W10^k = cos + S j sin of 2 pi k / 10
  auto w = [&](C a, T cr, T si) { return mk(a.x * cr - a.y * (T(S) * si), a.x * (T(S) * si) + a.y * cr); };
  o1 = w(o1, c1, s1);
  o2 = w(o2, c2, s2);
  o3 = w(o3, -c2, s2);
  o4 = w(o4, -c1, s1);
  v[0] = e0 + o0; v[5] = e0 - o0;
  v[1] = e1 + o1; v[6] = e1 - o1;
  v[2] = e2 + o2; v[7] = e2 - o2;
  v[3] = e3 + o3; v[8] = e3 - o3;
  v[4] = e4 + o4; v[9] = e4 - o4;
}

// radix 12 = 4 x 3: DFT4 over n1 for each n2 (inputs 3 n1 + n2), twiddle by
// W12^(n2 k1), DFT3 over n2, outputs k1 + 4 k2.
template <int S, typename C> __device__ __forceinline__ void dft12(C* v) {
  using T = decltype(C::x);
  const T r3 = T(0.86602540378443864676372317), h = T(0.5);
  C y[3][4];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    C a = v[n2], b = v[3 + n2], c = v[6 + n2], d = v[9 + n2];
    dft4<S>(a, b, c, d);
    y[n2][0] = a; y[n2][1] = b; y[n2][2] = c; y[n2][3] = d;
  }
  auto w = [&](C a, T cr, T si) { return mk(a.x * cr - a.y * (T(S) * si), a.x * (T(S) * si) + a.y * cr); };
  y[1][1] = w(y[1][1], r3, h);    // W12^1
  y[1][2] = w(y[1][2], h, r3);    // W12^2
  y[1][3] = mulj<S>(y[1][3]);     // W12^3
  y[2][1] = w(y[2][1], h, r3);    // W12^2
  y[2][2] = w(y[2][2], -h, r3);   // W12^4
  y[2][3] = mk(-y[2][3].x, -y[2][3].y);  // W12^6
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = y[0][k1], b = y[1][k1], c = y[2][k1];
    dft3<S>(a, b, c);
    v[k1] = a; v[k1 + 4] = b; v[k1 + 8] = c;
  }
}

template <int R, int S, typename C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2<S>(v[0], v[1]);
  else if constexpr (R == 3) dft3<S>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<S>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 5) dft5<S>(v[0], v[1], v[2], v[3], v[4]);
  else if constexpr (R == 6) dft6<S>(v);
  else if constexpr (R == 8) dft8<S>(v);
  else if constexpr (R == 10) dft10<S>(v);
  else if constexpr (R == 12) dft12<S>(v);
  else if constexpr (R == 16) dft16<S>(v);
  else static_assert(R == 2, "unsupported radix");
}

// ------------------------------------------------------------ radix plan
// Radices taken in this order: 8 while 8 | N, then 4, 2, 3, 5.
template <int N> struct first_radix {
  static constexpr int value = (N % 8 == 0) ? 8 : (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2
                               : (N % 3 == 0) ? 3 : (N % 5 == 0) ? 5 : 0;
};
template <int N> struct min_radix {
  static constexpr int R = first_radix<N>::value;
  static constexpr int rest = (R == 0 || R == N) ? 0 : min_radix<N / R>::value;
  static constexpr int value = (rest == 0 || R < rest) ? R : rest;
};
template <> struct min_radix<1> { static constexpr int value = 0; };

// ------------------------------------------------------------ fast division
// q = n / d for n, d < 2^16 via one multiply-high (m = ceil(2^32 / d)).
struct FastDiv {
  uint32_t d, m;
  __device__ __forceinline__ FastDiv(uint32_t dd) : d(dd), m(dd ? (uint32_t)((0x100000000ull + dd - 1) / dd) : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return d == 1 ? n : __umulhi(n, m); }
};

// --------------------------------------------------------------- one pass
// MAP_ELEM: consecutive threads take consecutive butterflies of one line
// (coalesced along the transformed dimension); otherwise consecutive
// threads take consecutive lines.
template <int N, int R, int P, int S, int NT, int MAXIT, bool MAP_ELEM, typename C,
          typename Src, typename Dst>
__device__ __forceinline__ void stockham_pass(int nl, const C* __restrict__ tw, Src&& src, Dst&& dst) {
  constexpr int NB = N / R;
  const int total = nl * NB;
  const FastDiv fd(nl > 0 ? nl : 1);
  C v[MAXIT][R];
#pragma unroll
  for (int it = 0; it < MAXIT; ++it) {
    const int w = threadIdx.x + it * NT;
    if (w < total) {
      int line, i;
      if constexpr (MAP_ELEM) { line = w / NB; i = w - line * NB; }
      else { i = (int)fd.div((uint32_t)w); line = w - i * nl; }
#pragma unroll
      for (int j = 0; j < R; ++j) v[it][j] = src(line, i + j * NB);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXIT; ++it) {
    const int w = threadIdx.x + it * NT;
    if (w < total) {
      int line, i;
      if constexpr (MAP_ELEM) { line = w / NB; i = w - line * NB; }
      else { i = (int)fd.div((uint32_t)w); line = w - i * nl; }
      const int k = i % P;
      if constexpr (P > 1) {
        constexpr int STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) {
          const C w_ = tw[j * k * STEP];
          v[it][j] = (S > 0) ? cmul(v[it][j], w_) : cmulc(v[it][j], w_);
        }
      }
      dft<R, S>(v[it]);
      const int base = (i - k) * R + k;
#pragma unroll
      for (int j = 0; j < R; ++j) dst(line, base + j * P, v[it][j]);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------- whole line FFT
// Runs every pass of a length-N DFT on nl lines (nl * N <= NT * EPT).
// first(line, e) reads the input, mid_ld / mid_st address the in-place
// shared buffer used between passes, last(line, e, v) receives the output.
template <int N, int REM, int P, int S, int NT, int EPT, bool MAP_ELEM, bool FIRST, typename C,
          typename First, typename MidLd, typename MidSt, typename Last>
__device__ __forceinline__ void fft_passes(int nl, const C* __restrict__ tw, First&& first,
                                           MidLd&& mid_ld, MidSt&& mid_st, Last&& last) {
  constexpr int R = first_radix<REM>::value;
  static_assert(R != 0, "length must be 2^a 3^b 5^c");
  constexpr int MAXIT = (EPT * NT / N * (N / R) + NT - 1) / NT;  // ceil(lines_max * N/R / NT)
  constexpr bool LAST = (REM == R);
  if constexpr (FIRST && LAST) {
    stockham_pass<N, R, P, S, NT, MAXIT, MAP_ELEM, C>(nl, tw, first, last);
  } else if constexpr (FIRST) {
    stockham_pass<N, R, P, S, NT, MAXIT, MAP_ELEM, C>(nl, tw, first, mid_st);
  } else if constexpr (LAST) {
    stockham_pass<N, R, P, S, NT, MAXIT, MAP_ELEM, C>(nl, tw, mid_ld, last);
  } else {
    stockham_pass<N, R, P, S, NT, MAXIT, MAP_ELEM, C>(nl, tw, mid_ld, mid_st);
  }
  if constexpr (!LAST)
    fft_passes<N, REM / R, P * R, S, NT, EPT, MAP_ELEM, false, C>(nl, tw, first, mid_ld, mid_st, last);
}

template <int N, int S, int NT, int EPT, bool MAP_ELEM, typename C, typename First, typename MidLd,
          typename MidSt, typename Last>
__device__ __forceinline__ void fft_lines(int nl, const C* __restrict__ tw, First&& first, MidLd&& mid_ld,
                                          MidSt&& mid_st, Last&& last) {
  fft_passes<N, N, 1, S, NT, EPT, MAP_ELEM, true, C>(nl, tw, first, mid_ld, mid_st, last);
}

// Lines of length N one pass-set can hold with NT threads and EPT elements each.
template <int N, int NT, int EPT> struct lines_per_chunk {
  static constexpr int value = (NT * EPT) / N;
};

__host__ __device__ constexpr int odd_pitch(int n) { return (n & 1) ? n : n + 1; }

// ------------------------------------------------------- warp-level passes
// A warp owns a few whole lines and runs all passes of their DFTs alone,
// synchronising with __syncwarp only. Between passes the lines sit in the
// warp's private shared-memory scratch, row-major with one pad element after
// every 8 (wpad): stride-R butterfly stores then fall on distinct banks.
// The row pitch is = 8 (mod 16) complex elements, so the two lines a
// half-warp touches use opposite bank halves.
__host__ __device__ constexpr int wpitch(int n) {
  return (n + n / 8) + ((8 - (n + n / 8) % 16) + 16) % 16;
}
__device__ __forceinline__ int wpad(int e) { return e + (e >> 3); }

template <int N, int R, int P, int S, int MAXIT, typename C, typename Src, typename Dst>
__device__ __forceinline__ void wpass(int nl, const C* __restrict__ tw, Src&& src, Dst&& dst) {
  constexpr int NB = N / R;
  const int lane = threadIdx.x & 31;
  const int total = nl * NB;
  C v[MAXIT][R];
#pragma unroll
  for (int it = 0; it < MAXIT; ++it) {
    const int w = lane + 32 * it;
    if (w < total) {
      const int line = w / NB, i = w - line * NB;
#pragma unroll
      for (int j = 0; j < R; ++j) v[it][j] = src(line, i + j * NB);
    }
  }
  __syncwarp();
#pragma unroll
  for (int it = 0; it < MAXIT; ++it) {
    const int w = lane + 32 * it;
    if (w < total) {
      const int line = w / NB, i = w - line * NB;
      const int k = i % P;
      if constexpr (P > 1) {
        constexpr int STEP = N / (P * R);
#pragma unroll
        for (int j = 1; j < R; ++j) {
          const C w_ = tw[j * k * STEP];
          v[it][j] = (S > 0) ? cmul(v[it][j], w_) : cmulc(v[it][j], w_);
        }
      }
      dft<R, S>(v[it]);
      const int base = (i - k) * R + k;
#pragma unroll
      for (int j = 0; j < R; ++j) dst(line, base + j * P, v[it][j]);
    }
  }
  __syncwarp();
}

// All passes of a length-N DFT on nl <= LMAX lines owned by one warp.
template <int N, int REM, int P, int S, int LMAX, bool FIRST, typename C, typename First,
          typename MidLd, typename MidSt, typename Last>
__device__ __forceinline__ void wfft_passes(int nl, const C* __restrict__ tw, First&& first,
                                            MidLd&& mid_ld, MidSt&& mid_st, Last&& last) {
  constexpr int R = first_radix<REM>::value;
  static_assert(R != 0, "length must be 2^a 3^b 5^c");
  constexpr int MAXIT = (LMAX * (N / R) + 31) / 32;
  constexpr bool LAST = (REM == R);
  if constexpr (FIRST && LAST) {
    wpass<N, R, P, S, MAXIT, C>(nl, tw, first, last);
  } else if constexpr (FIRST) {
    wpass<N, R, P, S, MAXIT, C>(nl, tw, first, mid_st);
  } else if constexpr (LAST) {
    wpass<N, R, P, S, MAXIT, C>(nl, tw, mid_ld, last);
  } else {
    wpass<N, R, P, S, MAXIT, C>(nl, tw, mid_ld, mid_st);
  }
  if constexpr (!LAST)
    wfft_passes<N, REM / R, P * R, S, LMAX, false, C>(nl, tw, first, mid_ld, mid_st, last);
}

template <int N, int S, int LMAX, typename C, typename First, typename MidLd, typename MidSt, typename Last>
__device__ __forceinline__ void wfft(int nl, const C* __restrict__ tw, First&& first, MidLd&& mid_ld,
                                     MidSt&& mid_st, Last&& last) {
  wfft_passes<N, N, 1, S, LMAX, true, C>(nl, tw, first, mid_ld, mid_st, last);
}

}  // namespace fftb
