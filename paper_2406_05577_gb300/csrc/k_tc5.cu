// k_tc5.cu -- MIXED_TC plane stage on the 5th-generation tensor cores.
//
// The y- and x-DFTs of one (band, z) plane (Fig. 3, second and third
// stage) are written as dense products with the DFT matrix, in the real form
// of a complex product,
//   [Re D]   [ C  -S ] [Re B]        C = cos(theta), S = sin(theta),
//   [Im D] = [ S   C ] [Im B],       theta = +-2 pi j m / N,
// pruned to the rows and columns the sphere occupies. Operands are split
// into FP16 high and low parts, v = hi + lo, and each product is the sum
// Wh Bh + Wh Bl + Wl Bh accumulated in FP32 in tensor memory (TMEM); the
// dropped Wl Bl term is 2^-22 of the result. Data are scaled per plane by a
// power of two so the FP16 operands neither overflow nor lose the low
// part.
//
//   G -> r: stick row -> B1[xu][(part, y)]; D1 = W1 B1^T (rows (y', part));
//           D1 -> B2[y'][(part, xu)];  D2 = W0 B2^T (rows (x', part));
//           D2 -> cube rows (y', x').
//   r -> G: cube plane -> B1[y][(part, x)]; D1 = W0 B1^T (rows (xu, part));
//           D1 -> B2[xu][(part, y)];  D2 = W1 B2^T (rows (yu, part));
//           D2 -> the sticks of the stick row.
// xu / yu index the union over k-points of the occupied x values and stick
// y values (the pruned dimensions); W matrices are built once per CTA.
//
// A CTA runs PL independent pipelines of one warpgroup (128 threads) each,
// sharing the W matrices; a pipeline walks its planes with a grid stride,
// its inputs arriving by bulk asynchronous copies one plane ahead. One thread
// of the pipeline issues the MMAs and commits them to an mbarrier; every
// wait is bounded and a failed wait sets the plan's status word.
#include <cuda_fp16.h>

#include "kernels.cuh"
#include "umma.cuh"

namespace fftb {
namespace {

constexpr int TC5_PL = 2;                 // pipelines (warpgroups) per CTA
constexpr int TC5_NT = 160 * TC5_PL;      // per pipeline: 4 SIMT warps and 1 MMA warp

__device__ __forceinline__ void named_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// barrier of one pipeline that also ORs a predicate over its threads
__device__ __forceinline__ bool named_sync_or(int id, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id)
      : "memory");
  return r != 0;
}

// v[0..7] -> FP16 high and low parts, 8 halves each (one core-matrix row)
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 a = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    const float2 af = __half22float2(a);
    const __half2 b = __floats2half2_rn(v[2 * i] - af.x, v[2 * i + 1] - af.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&a);
    l[i] = *reinterpret_cast<const uint32_t*>(&b);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ void st16(unsigned char* base, uint32_t off, const uint4& v) {
  *reinterpret_cast<uint4*>(base + off) = v;
}

// largest power-of-two exponent e with 2 * count * 2^e <= 65504: the bound on
// one complex output of a length-count product with |W| <= 1 and inputs <= 2^e
__device__ __forceinline__ int fp16_headroom(int count) {
  int e = 0;
  while (2.0f * (float)count * ldexpf(1.f, e + 1) <= 65504.f) ++e;
  return e;
}

struct Row {  // union row xu of the current k-point
  int xi, sa, len, ylo;
};

}  // namespace

// Per-pipeline and per-CTA shared memory of the tensor-core plane kernel.
template <int N> struct Tc5Layout {
  static constexpr int NR = (N + 15) / 16 * 16;
  static constexpr int KF = (N + 7) / 8 * 8;
  int kh1, kh2, ny, k1, k2, kr;
  size_t w_a, w_b;       // bytes of one W matrix (hi and lo), first and second
  size_t stage, opb1, opb2, per_pl, total;
  __host__ __device__ Tc5Layout(int mode, const Tc5Geo& P, int smax, bool shared_w) {
    kh1 = (P.yu + 7) & ~7;
    kh2 = (P.xu + 7) & ~7;
    ny = (P.xu + 15) & ~15;
    k1 = 2 * kh1;
    k2 = 2 * kh2;
    kr = 2 * KF;
    const size_t sp = (size_t)N * 8 + 16;  // staged cube row pitch (r -> G)
    if (mode == M_G2R) {
      w_a = 2 * (size_t)128 * k1 * 2;
      w_b = shared_w ? 0 : 2 * (size_t)128 * k2 * 2;
      stage = ((size_t)smax * 8 + 127) / 128 * 128;
      opb1 = 2 * (size_t)ny * k1 * 2;
      opb2 = 2 * (size_t)NR * k2 * 2;
    } else {
      w_a = 2 * (size_t)128 * kr * 2;
      w_b = shared_w ? 0 : w_a;
      const size_t rop = 2 * (size_t)NR * kr * 2, raw = (size_t)N * sp;
      stage = ((rop > raw ? rop : raw) + 127) / 128 * 128;
      opb1 = 0;  // the first operand is built in place of the staged plane
      opb2 = 2 * (size_t)ny * kr * 2;
    }
    per_pl = stage + opb1 + opb2 + 64 * sizeof(Row) + 64;
    total = w_a + w_b + TC5_PL * per_pl + (5 * TC5_PL + 1) * 8 + 16 * TC5_PL + 16;
  }
};

// Row m of a product result <-> (index, part). r -> G, whose results keep
// only the pruned rows, deals them to the four lane quarters (the warps that
// can read them) in whole 8-row groups: group g goes to quarter g % 4.
__host__ __device__ inline void tc5_row(int mode, int m, int& idx, int& part) {
  part = m & 1;
  if (mode == M_G2R) {
    idx = m >> 1;
  } else {
    const int q = m >> 5, j = (m & 31) >> 1;
    idx = 8 * (q + 4 * (j >> 3)) + (j & 7);
  }
}

// The W matrices of one direction, rows (out, part), K blocks (part, in), as
// the shared-memory image the kernel copies in: [first hi | first lo |
// second hi | second lo] (the second pair absent when both are the same).
template <int N, int MODE>
__global__ void k_tc5_weights(const float2* __restrict__ tw, const Tc5Geo P, unsigned char* __restrict__ img) {
  using LY = Tc5Layout<N>;
  const bool shared_w = P.xlo == P.ylo && P.xu == P.yu;
  const LY lay(MODE, P, 0, shared_w);
  const int KA = MODE == M_G2R ? lay.k1 : lay.kr;
  const int KB = MODE == M_G2R ? lay.k2 : lay.kr;
  const int nW = shared_w ? 1 : 2;
  for (int w = 0; w < nW; ++w) {
    unsigned char* W = img + (w == 0 ? 0 : lay.w_a);
    const int K = w == 0 ? KA : KB;
    const int kh = K / 2;
    const size_t half_bytes = (size_t)128 * K * 2;
    // G -> r: the first maps y (union) -> y' (all), the second x (union) -> x' (all)
    // r -> G: the first maps x (all) -> xu (union), the second y (all) -> yu (union)
    const bool first = w == 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 128 * K; i += gridDim.x * blockDim.x) {
      const int m = i / K, k = i - m * K;
      int out, pm;
      tc5_row(MODE, m, out, pm);
      const int pk = k >= kh, j = k - pk * kh;
      int o = -1, in = -1;
      if (MODE == M_G2R) {
        const int lo = first ? P.ylo : P.xlo, cnt = first ? P.yu : P.xu;
        if (out < N && j < cnt) {
          o = out;
          in = ((lo + j) % N + N) % N;
        }
      } else {
        const int lo = first ? P.xlo : P.ylo, cnt = first ? P.xu : P.yu;
        if (out < cnt && j < N) {
          o = ((lo + out) % N + N) % N;
          in = j;
        }
      }
      float v = 0.f;
      if (o >= 0) {
        const float2 e = tw[(o * in) % N];                    // e^{+2 pi i o in / N}
        const float c = e.x, sn = MODE == M_G2R ? e.y : -e.y;  // sine of the signed angle
        v = pm == 0 ? (pk == 0 ? c : -sn) : (pk == 0 ? sn : c);
      }
      const __half h = __float2half_rn(v);
      const __half l = __float2half_rn(v - __half2float(h));
      const uint32_t off = umma::kmajor_off(m, k, K);
      *reinterpret_cast<__half*>(W + off) = h;
      *reinterpret_cast<__half*>(W + half_bytes + off) = l;
    }
  }
}

// waits for the phase of `b` with parity ph; false when the pipeline's abort
// flag is raised or the time limit runs out (which raises the flag)
__device__ __forceinline__ bool wait_or_abort(uint64_t* b, uint32_t ph, volatile int* abort_flag) {
  if (mbar_try_wait(b, ph)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(b, ph)) {
    if (*abort_flag) return false;
    if (global_ns() - t0 > WAIT_LIMIT_NS) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

template <int N, int MODE>
__global__ void __launch_bounds__(TC5_NT, 1) k_plane_tc5(const Launch L, const Tc5Geo P) {
  using LY = Tc5Layout<N>;
  constexpr int NR = LY::NR, KF = LY::KF;
  extern __shared__ __align__(1024) unsigned char sm[];
  const bool shared_w = P.xlo == P.ylo && P.xu == P.yu;
  const LY lay(MODE, P, L.g.smax, shared_w);
  // threads [0, 128 PL): four SIMT warps per pipeline; then one MMA warp per pipeline
  const bool mma_role = threadIdx.x >= 128 * TC5_PL;
  const int pl = mma_role ? (threadIdx.x - 128 * TC5_PL) >> 5 : threadIdx.x >> 7;
  const int t = threadIdx.x & 127, warp = t >> 5, lane = threadIdx.x & 31;
  const int bar_id = 1 + pl;

  unsigned char* Wa = sm;  // hi, then lo
  unsigned char* Wb = shared_w ? sm : sm + lay.w_a;
  unsigned char* base = sm + lay.w_a + lay.w_b + pl * lay.per_pl;
  unsigned char* stage = base;
  unsigned char* ob1 = MODE == M_G2R ? base + lay.stage : stage;  // first B operand (hi, lo)
  unsigned char* ob2 = base + lay.stage + lay.opb1;               // second B operand (hi, lo)
  Row* rinfo = reinterpret_cast<Row*>(ob2 + lay.opb2);
  float* red = reinterpret_cast<float*>(rinfo + 64);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + lay.w_a + lay.w_b + TC5_PL * lay.per_pl);
  uint64_t* bar_in = bars + 5 * pl;      // input copies
  uint64_t* bar_m1 = bars + 5 * pl + 1;  // first products done
  uint64_t* bar_m2 = bars + 5 * pl + 2;  // second products done
  uint64_t* bar_o1 = bars + 5 * pl + 3;  // first operand written (128 arrivals)
  uint64_t* bar_o2 = bars + 5 * pl + 4;  // second operand written (128 arrivals)
  uint64_t* bar_w = bars + 5 * TC5_PL;   // the W image
  int* ctl = reinterpret_cast<int*>(bar_w + 1);  // per pipeline: copies, first, second products issued; abort
  volatile int* issued = ctl + 4 * pl;
  volatile int* abort_flag = ctl + 4 * pl + 3;
  uint32_t* slot = reinterpret_cast<uint32_t*>(ctl + 4 * TC5_PL);

  const int KA = MODE == M_G2R ? lay.k1 : lay.kr;  // K of the first product
  const int KB = MODE == M_G2R ? lay.k2 : lay.kr;  // K of the second
  const uint32_t ob1_half = MODE == M_G2R ? (uint32_t)lay.ny * lay.k1 * 2 : (uint32_t)NR * lay.kr * 2;
  const uint32_t ob2_half = MODE == M_G2R ? (uint32_t)NR * lay.k2 * 2 : (uint32_t)lay.ny * lay.kr * 2;
  const int n1_mma = MODE == M_G2R ? lay.ny : NR;  // N of the first product

  // ---- W image (bulk copy), zeroed B operands, barriers, tensor memory
  if (threadIdx.x == 0) {
    for (int i = 0; i < TC5_PL; ++i) {
      mbar_init(bars + 5 * i, 1);
      mbar_init(bars + 5 * i + 1, 1);
      mbar_init(bars + 5 * i + 2, 1);
      mbar_init(bars + 5 * i + 3, 128);
      mbar_init(bars + 5 * i + 4, 128);
    }
    mbar_init(bar_w, 1);
    for (int i = 0; i < 4 * TC5_PL; ++i) ctl[i] = 0;
    mbar_init_fence();
    const uint32_t wbytes = (uint32_t)(lay.w_a + lay.w_b);
    mbar_arrive_expect(bar_w, wbytes);
    bulk_g2s(sm, P.w, wbytes, bar_w);
  }
  if (!mma_role) {
    for (size_t i = t; i < (lay.opb1 + lay.opb2) / 16; i += 128)
      reinterpret_cast<uint4*>(base + lay.stage)[i] = make_uint4(0, 0, 0, 0);
    if (MODE != M_G2R)
      for (size_t i = t; i < lay.stage / 16; i += 128) reinterpret_cast<uint4*>(stage)[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x < 32) {
    umma::tmem_alloc(slot, 256 * TC5_PL);
    umma::tmem_relinquish();
  }
  fence_proxy_async_smem();
  umma::fence_before_sync();
  pdl_launch_dependents();
  __syncthreads();
  umma::fence_after_sync();
  pdl_wait();
  const bool w_bad = __syncthreads_or(!mbar_wait(bar_w, 0, WAIT_LIMIT_NS)) != 0;
  const uint32_t tmem = *slot + 256 * pl;
  const uint32_t t_d1 = tmem;  // first product; second products alternate at +64 and +128
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;

  const int n2 = L.g.n2;
  const int nplanes = L.nb * n2;
  const int stride = gridDim.x * TC5_PL;
  const size_t plane_elems = (size_t)N * N;
  const size_t sp = (size_t)N * 8 + 16;
  const int first = blockIdx.x * TC5_PL + pl;
  const bool withhold = (L.inject & INJECT_SKIP_FIRST_PREFETCH) && blockIdx.x == 0 && pl == 0;

  // the input of plane pp: its stick row of S2 sticks (G -> r: the MMA
  // thread) or its cube rows (r -> G: SIMT warp 0, a row per lane at a time)
  auto issue_input = [&](int pp, int S2) {
    const int bl2 = pp / n2, z2 = pp - bl2 * n2;
    fence_proxy_async_smem();
    if (MODE == M_G2R) {
      const uint32_t bytes = (uint32_t)((S2 * 8 + 15) & ~15);
      mbar_arrive_expect(bar_in, bytes);
      if (bytes) bulk_g2s(stage, static_cast<const float2*>(L.T) + ((size_t)bl2 * n2 + z2) * L.g.smax, bytes, bar_in);
      issued[0] = issued[0] + 1;
    } else {
      const float2* src = static_cast<const float2*>(L.cube_in) + ((size_t)(L.band0 + bl2) * n2 + z2) * plane_elems;
      if (lane == 0) mbar_arrive_expect(bar_in, (uint32_t)(N * N * 8));
      __syncwarp();
      for (int y = lane; y < N; y += 32) bulk_g2s(stage + y * sp, src + (size_t)y * N, (uint32_t)(N * 8), bar_in);
      __syncwarp();
      if (lane == 0) issued[0] = issued[0] + 1;
    }
  };

  int c_in = 0, c_m1 = 0, c_m2 = 0;  // waits completed by the SIMT warps
  if (mma_role) {
    // ================= MMA thread: issues both products of every plane
    if (lane == 0 && !w_bad) {
      // D (=) Ah Bh + Ah Bl + Al Bh, committed to `bar`
      auto issue_mma = [&](uint32_t d, const unsigned char* A, uint32_t a_half, const unsigned char* B,
                           uint32_t b_half, int K, uint32_t id, uint64_t* bar) {
        umma::fence_after_sync();
        const uint64_t ah = umma::sdesc(smem_u32(A), K), al = umma::sdesc(smem_u32(A) + a_half, K);
        const uint64_t bh = umma::sdesc(smem_u32(B), K), bl = umma::sdesc(smem_u32(B) + b_half, K);
        const int ns = K / 16;  // one K step advances the start address by 256 bytes (16 in the field)
#pragma unroll 1
        for (int s = 0; s < ns; ++s) umma::mma_f16(d, ah + 16 * s, bh + 16 * s, id, s != 0);
#pragma unroll 1
        for (int s = 0; s < ns; ++s) umma::mma_f16(d, ah + 16 * s, bl + 16 * s, id, 1u);
#pragma unroll 1
        for (int s = 0; s < ns; ++s) umma::mma_f16(d, al + 16 * s, bh + 16 * s, id, 1u);
        umma::commit(bar);
      };
      const uint32_t id1 = umma::idesc_f16(128, MODE == M_G2R ? lay.ny : NR);
      const uint32_t id2 = umma::idesc_f16(128, MODE == M_G2R ? NR : lay.ny);
      if (MODE == M_G2R && first < nplanes && !withhold) issue_input(first, L.g.band[L.band0 + first / n2].ki.S);
#pragma unroll 1
      for (int it = 0;; ++it) {
        const int p = first + it * stride;
        if (p >= nplanes) break;
        int S_nx = 0;
        if (MODE == M_G2R && p + stride < nplanes) S_nx = L.g.band[L.band0 + (p + stride) / n2].ki.S;
        if (!wait_or_abort(bar_o1, it & 1, abort_flag)) break;
        issue_mma(t_d1, Wa, (uint32_t)(128 * KA * 2), ob1, ob1_half, KA, id1, bar_m1);
        issued[1] = issued[1] + 1;
        if (MODE == M_G2R && p + stride < nplanes) issue_input(p + stride, S_nx);  // the stick row is consumed
        if (!wait_or_abort(bar_o2, it & 1, abort_flag)) break;
        issue_mma(tmem + 64 + 64 * (it & 1), Wb, (uint32_t)(128 * KB * 2), ob2, ob2_half, KB, id2, bar_m2);
        issued[2] = issued[2] + 1;
      }
    }
  } else if (!w_bad) {
    // ================= SIMT warps: operands in, results out
    // bounded wait agreed on by the pipeline's 128 threads
    auto await = [&](uint64_t* b, int& consumed) {
      const bool ok = wait_or_abort(b, consumed & 1, abort_flag);
      if (named_sync_or(bar_id, !ok)) {
        if (t == 0) *abort_flag = 1;
        return false;
      }
      ++consumed;
      umma::fence_after_sync();
      return true;
    };
    KInfo ki_cur{};  // band record of the current plane, loaded one plane ahead
    if (first < nplanes) {
      ki_cur = L.g.band[L.band0 + first / n2].ki;
      if (MODE != M_G2R && t < 32 && !withhold) issue_input(first, 0);
    }
    int cur_k = -1, pprev = -1;
    float inv_prev = 1.f;
    // software pipeline: A(p) first operand, C(p - stride) output of the
    // previous plane, D(p) second operand; the MMA thread runs the products
    // in between, so they overlap the neighbouring plane's SIMT work
#pragma unroll 1
    for (int it = 0;; ++it) {
      const int p = first + it * stride;
      const bool have = p < nplanes;
      if (!have && pprev < 0) break;
      const KInfo ki = ki_cur;
      KInfo ki_nx{};
      if (p + stride < nplanes) ki_nx = L.g.band[L.band0 + (p + stride) / n2].ki;
      float inv_scale = 1.f;
      if (have) {
        // ---- A: input and first operand
        if (!await(bar_in, c_in)) break;
        if (MODE == M_G2R && ki.xmap_base != cur_k) {  // rows of the union x range for this k-point
          cur_k = ki.xmap_base;
          if (t < 64) {
            Row r{-1, 0, 0, 0};
            if (t < P.xu) {
              const int x = ((P.xlo + t) % N + N) % N;
              const int xi = L.g.xmap[ki.xmap_base + x];
              if (xi >= 0) {
                const int4 c = L.g.col_info[ki.col_base + xi];
                r = Row{xi, c.x, c.y, c.z};
              }
            }
            rinfo[t] = r;
          }
          named_sync(bar_id);
        }
        if constexpr (MODE == M_G2R) {
          // plane scale from the stick row
          const float2* st = reinterpret_cast<const float2*>(stage);
          float mx = 0.f;
          for (int i = t; i < ki.S; i += 128) mx = fmaxf(mx, fmaxf(fabsf(st[i].x), fabsf(st[i].y)));
#pragma unroll
          for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (lane == 0) red[warp] = mx;
          named_sync(bar_id);
          mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
          const int e = fp16_headroom(P.yu) - (mx > 0.f ? ilogbf(mx) + 1 : 0);
          const float scale = ldexpf(1.f, e);
          inv_scale = ldexpf(1.f, -e);
          // B1[xu][(part, y)]: lanes 8 rows of one K chunk (conflict-free stores)
          const int nc = lay.kh1 / 8, rg = (P.xu + 7) / 8;
          for (int i2 = t; i2 < rg * nc * 8; i2 += 128) {
            const int r = i2 & 7, c = (i2 >> 3) % nc, g = (i2 >> 3) / nc;
            const int xu = g * 8 + r;
            if (xu >= P.xu) continue;
            const Row ri = rinfo[xu];
            float re[8], im[8];
#pragma unroll
            for (int e2 = 0; e2 < 8; ++e2) {
              const int d = P.ylo + c * 8 + e2 - ri.ylo;
              float2 v = make_float2(0.f, 0.f);
              if (ri.xi >= 0 && (unsigned)d < (unsigned)ri.len) v = st[ri.sa + d];
              re[e2] = v.x * scale;
              im[e2] = v.y * scale;
            }
            uint4 h, l;
            split8(re, h, l);
            st16(ob1, umma::kmajor_off(xu, c * 8, lay.k1), h);
            st16(ob1 + ob1_half, umma::kmajor_off(xu, c * 8, lay.k1), l);
            split8(im, h, l);
            st16(ob1, umma::kmajor_off(xu, lay.kh1 + c * 8, lay.k1), h);
            st16(ob1 + ob1_half, umma::kmajor_off(xu, lay.kh1 + c * 8, lay.k1), l);
          }
        } else {
          // the staged plane -> registers, plane scale, then B1[y][(part, x)] in place
          constexpr int QC = N / 8;                    // 8-element chunks per row
          constexpr int ITEMS = (N * QC + 127) / 128;  // per thread
          float2 v[ITEMS][8];
          float mx = 0.f;
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const int i2 = t + 128 * i;
            if (i2 < N * QC) {
              const int r = i2 & 7, q = (i2 >> 3) % QC, g = (i2 >> 3) / QC;
              const float4* src = reinterpret_cast<const float4*>(stage + (g * 8 + r) * sp + q * 64);
#pragma unroll
              for (int e2 = 0; e2 < 4; ++e2) {
                const float4 a = src[e2];
                v[i][2 * e2] = make_float2(a.x, a.y);
                v[i][2 * e2 + 1] = make_float2(a.z, a.w);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
              }
            }
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (lane == 0) red[warp] = mx;
          named_sync(bar_id);  // also: every read of the staged plane is done
          mx = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
          const int e = fp16_headroom(N) - (mx > 0.f ? ilogbf(mx) + 1 : 0);
          const float scale = ldexpf(1.f, e);
          inv_scale = ldexpf(1.f, -e);
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const int i2 = t + 128 * i;
            if (i2 < N * QC) {
              const int r = i2 & 7, q = (i2 >> 3) % QC, g = (i2 >> 3) / QC;
              const int y = g * 8 + r;
              float re[8], im[8];
#pragma unroll
              for (int e2 = 0; e2 < 8; ++e2) {
                re[e2] = v[i][e2].x * scale;
                im[e2] = v[i][e2].y * scale;
              }
              uint4 h, l;
              split8(re, h, l);
              st16(ob1, umma::kmajor_off(y, q * 8, lay.kr), h);
              st16(ob1 + ob1_half, umma::kmajor_off(y, q * 8, lay.kr), l);
              split8(im, h, l);
              st16(ob1, umma::kmajor_off(y, KF + q * 8, lay.kr), h);
              st16(ob1 + ob1_half, umma::kmajor_off(y, KF + q * 8, lay.kr), l);
            }
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(bar_o1);
      }
      // ---- C: output of the previous plane
      if (pprev >= 0) {
        if (!await(bar_m2, c_m2)) break;
        const uint32_t t_d2 = tmem + 64 + 64 * ((it - 1) & 1);
        const int blp = pprev / n2, zp = pprev - blp * n2;
        int o, pm;  // this lane is row (o, part); lanes t, t ^ 1 pair up
        tc5_row(MODE, t, o, pm);
        float v[64];
        if constexpr (MODE == M_G2R) {
          float2* out = static_cast<float2*>(L.cube_out) + ((size_t)(L.band0 + blp) * n2 + zp) * plane_elems;
          const bool live = o < N;
          umma::ld64(t_d2 + lane_off, NR / 16, v);
          umma::ld_wait();
#pragma unroll
          for (int j = 0; j < NR; j += 2) {
            const float a = v[j] * inv_prev, b = v[j + 1] * inv_prev;
            const float recv = __shfl_xor_sync(0xffffffffu, pm ? a : b, 1);
            const int y = j + pm;  // even lane: column j, odd lane: column j + 1
            if (live && y < N) out[(size_t)y * N + o] = pm ? make_float2(recv, b) : make_float2(a, recv);
          }
        } else {
          float2* Tz = static_cast<float2*>(L.T) + ((size_t)blp * n2 + zp) * L.g.smax;
          const bool live = o < P.yu;
          const int y = P.ylo + o;
          umma::ld64(t_d2 + lane_off, lay.ny / 16, v);
          umma::ld_wait();
#pragma unroll
          for (int j = 0; j < 64; j += 2) {
            if (j < lay.ny) {
              const float a = v[j] * inv_prev, b = v[j + 1] * inv_prev;
              const float recv = __shfl_xor_sync(0xffffffffu, pm ? a : b, 1);
              const int xu = j + pm;
              if (live && xu < P.xu) {
                const Row ri = rinfo[xu];
                const int d = y - ri.ylo;
                if (ri.xi >= 0 && (unsigned)d < (unsigned)ri.len)
                  Tz[ri.sa + d] = pm ? make_float2(recv, b) : make_float2(a, recv);
              }
            }
          }
        }
        umma::fence_before_sync();
        pprev = -1;
      }
      if (!have) break;
      // ---- D: first product -> second operand
      if (!await(bar_m1, c_m1)) break;
      if (MODE != M_G2R) {
        if (t < 32 && p + stride < nplanes) issue_input(p + stride, 0);  // B1 is consumed
        if (ki.xmap_base != cur_k) {  // rows for this plane's output (read after later barriers)
          cur_k = ki.xmap_base;
          if (t < 64) {
            Row r{-1, 0, 0, 0};
            if (t < P.xu) {
              const int x = ((P.xlo + t) % N + N) % N;
              const int xi = L.g.xmap[ki.xmap_base + x];
              if (xi >= 0) {
                const int4 c = L.g.col_info[ki.col_base + xi];
                r = Row{xi, c.x, c.y, c.z};
              }
            }
            rinfo[t] = r;
          }
        }
      }
      {
        int o, pm;  // this lane is row (o, part) of D1
        tc5_row(MODE, t, o, pm);
        const int orows = MODE == M_G2R ? N : P.xu;   // valid rows of D1
        const int kh = MODE == M_G2R ? lay.kh2 : KF;  // K per part of the second product
        const int kk = MODE == M_G2R ? lay.k2 : lay.kr;
        const bool live = o < orows;
        float v[64];
        umma::ld64(t_d1 + lane_off, n1_mma / 16, v);
        umma::ld_wait();
        if (live) {
#pragma unroll
          for (int c0 = 0; c0 < 64; c0 += 8) {
            if (c0 < kh && c0 < n1_mma) {
              float w8[8];
#pragma unroll
              for (int e2 = 0; e2 < 8; ++e2) w8[e2] = v[c0 + e2];
              uint4 h, l;
              split8(w8, h, l);
              st16(ob2, umma::kmajor_off(o, pm * kh + c0, kk), h);
              st16(ob2 + ob2_half, umma::kmajor_off(o, pm * kh + c0, kk), l);
            }
          }
        }
      }
      umma::fence_before_sync();
      fence_proxy_async_smem();
      mbar_arrive(bar_o2);
      inv_prev = inv_scale;
      pprev = p;
      ki_cur = ki_nx;
    }
  }
  __syncthreads();  // nothing is issued after this point
  if (!mma_role && t == 0 && (*abort_flag || w_bad)) {
    *reinterpret_cast<volatile int32_t*>(L.status) = STATUS_WAIT_TIMEOUT;
    // copies and products issued (counted by their issuers) but not seen
    // complete (counted by the SIMT waits) land before the memory is released
    if (issued[0] > c_in) mbar_wait(bar_in, c_in & 1, WAIT_LIMIT_NS);
    if (issued[1] > c_m1) mbar_wait(bar_m1, c_m1 & 1, WAIT_LIMIT_NS);
    if (issued[2] > c_m2) mbar_wait(bar_m2, c_m2 & 1, WAIT_LIMIT_NS);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  if (threadIdx.x < 32) umma::tmem_dealloc(*slot, 256 * TC5_PL);
}

// ------------------------------------------------------------------ host side
namespace {
template <int N> size_t smem_of(int mode, const Tc5Geo& P, int smax) {
  const bool shared_w = P.xlo == P.ylo && P.xu == P.yu;
  const size_t s = Tc5Layout<N>(mode, P, smax, shared_w).total;
  // at most 512 / (128 * TC5_PL) resident CTAs per SM, so TMEM never runs out
  const size_t floor_bytes = (size_t)(228 * 1024) / (512 / (256 * TC5_PL) + 1) + 1024;
  return s > floor_bytes ? s : floor_bytes;
}
template <int N> const void* kernel_of(int mode) {
  return mode == M_G2R ? (const void*)k_plane_tc5<N, M_G2R> : (const void*)k_plane_tc5<N, M_R2G>;
}
#define TC5_SIZES(X) X(16) X(32) X(48) X(64)
}  // namespace

bool tc5_supported(int n0, int n1) {
  if (n0 != n1) return false;
  switch (n0) {
#define C_(N) case N: return true;
    TC5_SIZES(C_)
#undef C_
  }
  return false;
}

size_t tc5_smem(int mode, int n, const Tc5Geo& P, int smax) {
  switch (n) {
#define C_(N) case N: return smem_of<N>(mode, P, smax);
    TC5_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t tc5_prepare(int mode, int n, const Tc5Geo& P, int smax, int* occupancy) {
  const void* fn = nullptr;
  switch (n) {
#define C_(N) case N: fn = kernel_of<N>(mode); break;
    TC5_SIZES(C_)
#undef C_
  }
  if (!fn) return cudaErrorInvalidValue;
  const size_t s = tc5_smem(mode, n, P, smax);
  cudaError_t e = raise_smem_limit(fn, (int)s);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, fn, TC5_NT, s);
}

size_t tc5_weight_bytes(int mode, int n, const Tc5Geo& P) {
  const bool shared_w = P.xlo == P.ylo && P.xu == P.yu;
  switch (n) {
#define C_(N) \
  case N: { const Tc5Layout<N> l(mode, P, 0, shared_w); return l.w_a + l.w_b; }
    TC5_SIZES(C_)
#undef C_
  }
  return 0;
}

cudaError_t tc5_build_weights(int mode, int n, const Tc5Geo& P, const void* tw, void* img) {
  const float2* t = static_cast<const float2*>(tw);
  unsigned char* o = static_cast<unsigned char*>(img);
  switch (n) {
#define C_(N)                                                                  \
  case N:                                                                      \
    if (mode == M_G2R) k_tc5_weights<N, M_G2R><<<64, 256>>>(t, P, o);          \
    else k_tc5_weights<N, M_R2G><<<64, 256>>>(t, P, o);                        \
    return cudaGetLastError();
    TC5_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc5_launch(int mode, const Launch& L, const Tc5Geo& P, int ctas) {
  const int n = L.g.n0;
  const size_t s = tc5_smem(mode, n, P, L.g.smax);
  const int nplanes = L.nb * L.g.n2;
  const int need = (nplanes + TC5_PL - 1) / TC5_PL;
  const dim3 grid(ctas > 0 && ctas < need ? ctas : need);
  switch (n) {
#define C_(N)                                                                                  \
  case N:                                                                                      \
    if (mode == M_G2R) return launch_k(k_plane_tc5<N, M_G2R>, grid, TC5_NT, s, L, L, P);    \
    return launch_k(k_plane_tc5<N, M_R2G>, grid, TC5_NT, s, L, L, P);
    TC5_SIZES(C_)
#undef C_
  }
  return cudaErrorInvalidValue;
}

}  // namespace fftb
