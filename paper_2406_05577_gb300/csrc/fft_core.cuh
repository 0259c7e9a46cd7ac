// fft_core.cuh -- complex arithmetic, register codelets and the exchange-row
// layout of the batched 1D DFTs of the staged sphere <-> cube transform.
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

// ------------------------------------------------- compile-time twiddles
// cos and sin of 2 pi m / L for integers m and L, evaluated by the compiler
// in double precision: the angle is reduced exactly (integer arithmetic in
// units of a turn / (8 L)) to an octant, folded to [0, pi/4] by the
// symmetries of the circle, and the Taylor series of cos and sin about 0 is
// summed to 30 terms (the terms at pi/4 fall below 1e-17 after 11).
namespace ctw {
constexpr double kPi = 3.141592653589793238462643383279502884;
__host__ __device__ constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / double((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 30; ++k) {
    term *= -x * x / double((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
// (cos, sin)(2 pi m / L) as c (sel = 0) or s (sel = 1)
__host__ __device__ constexpr double cs(int m, int L, int sel) {
  const long q = ((long)m % L + L) % L;     // turn fraction q / L in [0, 1)
  const long t = 8 * q;                     // in units of a turn / (8 L)
  const int oct = (int)(t / L);             // octant 0..7
  const long r = t - (long)oct * L;         // angle inside the octant: (pi/4) r / L
  double c = 0, s = 0;
  if (oct % 2 == 0) {                       // alpha = (pi/4) r / L in [0, pi/4)
    const double a = (kPi / 4) * (double(r) / double(L));
    c = taylor_cos(a);
    s = taylor_sin(a);
  } else {                                  // alpha = pi/4 + (pi/4) r / L: use pi/2 - alpha in (0, pi/4]
    const double b = (kPi / 4) * (double(L - r) / double(L));
    c = taylor_sin(b);
    s = taylor_cos(b);
  }
  const int quad = oct / 2;                 // rotate by quad quarter turns
  const double cc = quad == 0 ? c : quad == 1 ? -s : quad == 2 ? -c : s;
  const double ss = quad == 0 ? s : quad == 1 ? c : quad == 2 ? -s : -c;
  return sel == 0 ? cc : ss;
}
}  // namespace ctw

// v * e^{S 2 pi j m / L} with the constant evaluated by the compiler; quarter
// turns become sign changes and swaps.
template <int M, int L, int S, typename C> __device__ __forceinline__ C wconst(C a) {
  using T = decltype(C::x);
  constexpr int q = ((M % L) + L) % L;
  if constexpr (q == 0) return a;
  else if constexpr (4 * q == L) return mulj<S>(a);
  else if constexpr (2 * q == L) return mk(-a.x, -a.y);
  else if constexpr (4 * q == 3 * L) return mulj<-S>(a);
  else {
    constexpr T c = T(ctw::cs(q, L, 0));
    constexpr T sn = T(S) * T(ctw::cs(q, L, 1));
    return mk(a.x * c - a.y * sn, a.x * sn + a.y * c);
  }
}

template <int R, int S, typename C> __device__ __forceinline__ void dft(C* v);

// y[n2][k1] *= W^(n2 k1) for every element, index I = n2 A + k1
template <int A, int B, int S, int I, typename C> __device__ __forceinline__ void ct_twiddle(C (&y)[B][A]) {
  if constexpr (I < A * B) {
    y[I / A][I % A] = wconst<(I / A) * (I % A), A * B, S>(y[I / A][I % A]);
    ct_twiddle<A, B, S, I + 1>(y);
  }
}

// Composite radix A * B in registers (Cooley-Tukey, Sec. 2.1): input index
// n = B n1 + n2, output index k = k1 + A k2; a DFT-A over n1 for each n2,
// the twiddles W^(n2 k1) (W = e^{S 2 pi j / (A B)}, compile-time constants),
// then a DFT-B over n2 for each k1.
template <int A, int B, int S, typename C> __device__ __forceinline__ void dft_ct(C* v) {
  C y[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) y[n2][n1] = v[B * n1 + n2];
    dft<A, S>(y[n2]);
  }
  ct_twiddle<A, B, S, 0>(y);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2][k1];
    dft<B, S>(t);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
  }
}

// ----------------------------------------------- inputs known to be zero
// The same transforms when some inputs are zero at compile time (bit i of Z:
// input i is zero), for lines that carry fewer values than their length: a
// sum or difference with a known zero is not computed. The results equal the
// general codelets' (up to the sign of zero results).
template <bool ZA, bool ZB, typename C> __device__ __forceinline__ C zadd(C a, C b) {
  if constexpr (ZA && ZB) return czero<C>();
  else if constexpr (ZA) return b;
  else if constexpr (ZB) return a;
  else return a + b;
}
template <bool ZA, bool ZB, typename C> __device__ __forceinline__ C zsub(C a, C b) {
  if constexpr (ZA && ZB) return czero<C>();
  else if constexpr (ZA) return mk(-b.x, -b.y);
  else if constexpr (ZB) return a;
  else return a - b;
}
template <int S, unsigned Z, typename C> __device__ __forceinline__ void dft4_z(C& x0, C& x1, C& x2, C& x3) {
  constexpr bool Z0 = Z & 1, Z1 = (Z >> 1) & 1, Z2 = (Z >> 2) & 1, Z3 = (Z >> 3) & 1;
  constexpr bool T02 = Z0 && Z2, T13 = Z1 && Z3;
  const C t0 = zadd<Z0, Z2>(x0, x2), t1 = zsub<Z0, Z2>(x0, x2);
  const C t2 = zadd<Z1, Z3>(x1, x3), t3 = mulj<S>(zsub<Z1, Z3>(x1, x3));
  x0 = zadd<T02, T13>(t0, t2);
  x2 = zsub<T02, T13>(t0, t2);
  x1 = zadd<T02, T13>(t1, t3);
  x3 = zsub<T02, T13>(t1, t3);
}
// radix 8 as dft8: DFT4 of the even and of the odd inputs, twiddles, radix 2
template <int S, unsigned Z, typename C> __device__ __forceinline__ void dft8_z(C* v) {
  using T = decltype(C::x);
  constexpr unsigned ZE = (Z & 1) | ((Z >> 1) & 2) | ((Z >> 2) & 4) | ((Z >> 3) & 8);           // inputs 0 2 4 6
  constexpr unsigned ZO = ((Z >> 1) & 1) | ((Z >> 2) & 2) | ((Z >> 3) & 4) | ((Z >> 4) & 8);    // inputs 1 3 5 7
  constexpr bool EZ = ZE == 15, OZ = ZO == 15;
  const T h = T(0.70710678118654752440084436);  // 1/sqrt(2)
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4_z<S, ZE>(e0, e1, e2, e3);
  dft4_z<S, ZO>(o0, o1, o2, o3);
  if constexpr (!OZ) {
    o1 = scale(o1 + mulj<S>(o1), h);
    o2 = mulj<S>(o2);
    o3 = scale(mulj<S>(o3) - o3, h);
  }
  v[0] = zadd<EZ, OZ>(e0, o0); v[4] = zsub<EZ, OZ>(e0, o0);
  v[1] = zadd<EZ, OZ>(e1, o1); v[5] = zsub<EZ, OZ>(e1, o1);
  v[2] = zadd<EZ, OZ>(e2, o2); v[6] = zsub<EZ, OZ>(e2, o2);
  v[3] = zadd<EZ, OZ>(e3, o3); v[7] = zsub<EZ, OZ>(e3, o3);
}
// bits of Z at the inputs B n1 + n2 of the DFT-A over n1 (the composite's first stage)
template <int A, int B> __host__ __device__ constexpr unsigned ct_sub_mask(unsigned long long Z, int n2) {
  unsigned m = 0;
  for (int n1 = 0; n1 < A; ++n1) m |= (unsigned)((Z >> (B * n1 + n2)) & 1ull) << n1;
  return m;
}
template <int A, int B, int S, unsigned long long Z, int N2I, typename C>
__device__ __forceinline__ void ct_stage1_z(C (&y)[B][A], const C* v) {
  if constexpr (N2I < B) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) y[N2I][n1] = v[B * n1 + N2I];
    constexpr unsigned m = ct_sub_mask<A, B>(Z, N2I);
    static_assert(A == 8, "zero-aware first stage of radix 8");
    dft8_z<S, m>(y[N2I]);
    ct_stage1_z<A, B, S, Z, N2I + 1>(y, v);
  }
}
// composite radix A * B (dft_ct) with the inputs of Z known to be zero
template <int A, int B, int S, unsigned long long Z, typename C> __device__ __forceinline__ void dft_ct_z(C* v) {
  C y[B][A];
  ct_stage1_z<A, B, S, Z, 0>(y, v);
  ct_twiddle<A, B, S, 0>(y);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    C t[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2][k1];
    dft<B, S>(t);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k1 + A * k2] = t[k2];
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
  else if constexpr (R == 20) dft_ct<4, 5, S>(v);
  else if constexpr (R == 24) dft_ct<8, 3, S>(v);
  else if constexpr (R == 32) dft_ct<8, 4, S>(v);
  else if constexpr (R == 40) dft_ct<8, 5, S>(v);
  else static_assert(R == 2, "unsupported radix");
}
// radix R with the inputs of Z zero at compile time (zero-aware for 4, 8 and 40 = 8 x 5)
template <int R, int S, unsigned long long Z, typename C> __device__ __forceinline__ void dft_z(C* v) {
  if constexpr (Z == 0) dft<R, S>(v);
  else if constexpr (R == 4) dft4_z<S, (unsigned)Z>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8_z<S, (unsigned)Z>(v);
  else if constexpr (R == 40) dft_ct_z<8, 5, S, Z>(v);
  else dft<R, S>(v);
}

// ------------------------------------------------------- exchange rows
// Between passes the lines of a warp sit in the warp's private shared-memory
// scratch, row-major with one pad element after every 8 (wpad): stride-R
// butterfly stores then fall on distinct banks. The G lanes of one line touch
// a window of about G consecutive elements (2 G words) at a time, so the row
// pitch is chosen = G (mod 2 G) complex elements for G = 2, 4, 8: the windows
// of the 32 / G lines of a warp then start 2 G words apart modulo an odd
// multiple, and together tile the 32 banks.
__host__ __device__ constexpr int wpitch(int n, int g = 8) {
  const int base = n + n / 8;
  const int m = (g >= 2 && g <= 8) ? 2 * g : 16;
  const int r = (g >= 2 && g <= 8) ? g : 8;
  return base + ((r - base % m) % m + m) % m;
}
__device__ __forceinline__ int wpad(int e) { return e + (e >> 3); }

}  // namespace fftb
