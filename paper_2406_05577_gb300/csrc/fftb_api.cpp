// fftb_api.cpp -- the C ABI: plans (geometry, twiddles, device tables,
// scratch) and the launch schedule of each direction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/fftb.h"
#include "fftb_internal.h"
#include "geometry.h"
#include "tables.h"

// NVTX ranges (header-only; a no-op unless a profiler is attached): one per
// execute, per host-buffer execute, per autotune and per stage launch.
#include <nvtx3/nvToolsExt.h>

#define FFTB_EXPORT extern "C" __attribute__((visibility("default")))

namespace fftb {

template <typename T, bool TC> size_t stick_smem_t(int);
template <typename T, bool TC> size_t plane_smem_t(int, int, int, int, bool);
template <typename T, bool TC> int stick_tile_t(int);
template <typename T, bool TC> cudaError_t launch_stick_t(int, const Launch&, int);
template <typename T, bool TC> cudaError_t launch_plane_t(int, const Launch&);
template <typename T, bool TC> cudaError_t prepare_t(int, int, int, int, int, bool);
template <typename T, bool TC> int plane_occupancy_t(int, int, int, int, int, bool);
template <typename T, bool TC> int stick_occupancy_t(int);

// P_F64 -> double, P_F32 -> float, P_TC -> float with tensor-core radix-8 passes
#define FFTB_BY_PREC(prec, call)                                                           \
  ((prec) == P_F64 ? call<double, false> : (prec) == P_TC ? call<float, true> : call<float, false>)

static const int kSizes[] = {12, 16, 20, 24, 32, 40, 48, 64, 96, 128, 160, 256};

bool grid_size_supported(int n) {
  for (int s : kSizes)
    if (s == n) return true;
  return false;
}
bool plane_size_supported(int n0, int n1) { return n0 == n1 && grid_size_supported(n0); }
size_t stick_smem(int prec, int n2) { return FFTB_BY_PREC(prec, stick_smem_t)(n2); }
size_t plane_smem(int prec, int n0, int n1, int xmax, int a_bufs, bool a_glob) {
  return FFTB_BY_PREC(prec, plane_smem_t)(n0, n1, xmax, a_bufs, a_glob);
}
int stick_tile(int prec, int n2) { return FFTB_BY_PREC(prec, stick_tile_t)(n2); }
cudaError_t prepare_kernels(int prec, int n0, int n1, int n2, int xmax, int a_bufs, bool a_glob) {
  return FFTB_BY_PREC(prec, prepare_t)(n0, n1, n2, xmax, a_bufs, a_glob);
}
int stick_occupancy(int prec, int n2) { return FFTB_BY_PREC(prec, stick_occupancy_t)(n2); }
int plane_occupancy(int prec, int mode, int n0, int n1, int xmax, int a_bufs, bool a_glob) {
  return FFTB_BY_PREC(prec, plane_occupancy_t)(mode, n0, n1, xmax, a_bufs, a_glob);
}
cudaError_t launch_stick(int prec, int mode, const Launch& L, int tiles) {
  return FFTB_BY_PREC(prec, launch_stick_t)(mode, L, tiles);
}
cudaError_t launch_plane(int prec, int mode, const Launch& L) { return FFTB_BY_PREC(prec, launch_plane_t)(mode, L); }

static thread_local std::string g_last_error;

static fftb_status fail(fftb_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
void set_last_error(const std::string& msg) { g_last_error = msg; }

static fftb_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FFTB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace fftb

using namespace fftb;

struct fftb_plan_s {
  int32_t n[3];
  int32_t nk;
  fftb_direction dir;
  fftb_precision prec;
  int prec_kernel;  // P_F32 or P_F64
  int32_t csize;    // bytes per complex element
  std::vector<KGeom> geo;
  std::vector<int32_t> bands;
  int32_t total_bands = 0;
  int64_t sphere_elems = 0, cube_elems = 0;
  int32_t smax = 0, xmax = 0, tiles = 0, chunk = 1;
  int32_t tpitch = 2;  // stick-row pitch of T: smax rounded up to even
  int32_t layout = 0;  // 0 band-major, 1 batch-fastest (band index fastest)
  // batch-fastest FP32 plans: plane stages over groups of bands of one k-point
  int bg = 0;                      // group size in use (0: one band per plane)
  int bg_size = 0;                 // the grid's group size where the grouped kernels fit, else 0
  int bg_occ[2] = {0, 0};          // their resident CTAs per SM: G->r, r->G
  std::vector<int2> groups;        // (first band, bands) of every group, k-point by k-point
  std::vector<int32_t> band_grp;   // group of a band that starts one, else -1
  void* d_groups = nullptr;
  cudaStream_t cap_stream = nullptr;  // graph capture for executes on the legacy default stream
  int64_t graph_launches = 0;         // executes that replayed (or first launched) a recorded graph
  double scale_g2r = 1.0, scale_r2g = 1.0;  // output normalisation (fftb_plan_set_scale)
  int device = 0;
  int32_t plane_ctas[3] = {0, 0, 0};  // persistent CTAs: G->r, r->G, apply
  int32_t a_bufs = 2;                 // slab-plane buffers of the plane stage
  bool a_glob = false;                // slab planes in global memory (FP64, large planes)
  void* d_A = nullptr;                // those slab planes, one block per persistent CTA
  size_t A_bytes = 0;
  int32_t a_blocks = 0;               // CTA blocks d_A holds
  // device memory
  void* d_tables = nullptr;
  size_t tables_bytes = 0;
  void* d_T = nullptr;
  size_t T_bytes = 0;
  Geo g{};
  const void* d_V = nullptr;
  // sphere offset of every band (complex elements; total_bands + 1 values)
  std::vector<int64_t> band_sph;
  // host-buffer path: copy-in, compute and copy-out streams and their events
  cudaStream_t hs[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> hev;
  // host-buffer path staging (allocated on first use)
  void* d_stage_in = nullptr;
  void* d_stage_out = nullptr;
  void* d_stage_cube = nullptr;
  size_t stage_in_bytes = 0, stage_out_bytes = 0, stage_cube_bytes = 0;
  int64_t launches = 0;
  // CUDA-graph execution (fftb_plan_set_graph)
  bool use_graph = false;
  cudaGraphExec_t gexec = nullptr;
  const void* g_in = nullptr;
  void* g_out = nullptr;
  void* g_cube = nullptr;
  const void* g_V = nullptr;
  int sms = 0;
  int plane_occ[3] = {0, 0, 0};  // resident plane CTAs per SM: G->r, r->G, apply
  int stick_occ = 1;             // resident z-stage CTAs per SM
  // bulk-copy prefetch in the plane stage (FP32), per mode: kernels exist and
  // fit in shared memory (pf_fit), their resident CTAs per SM (pf_occ), and
  // the level asked for (fftb_plan_set_prefetch: 0 off, 1 where no resident
  // CTA is lost, 2 wherever it fits)
  bool pf_fit[3] = {false, false, false};
  int pf_occ[3] = {0, 0, 0};
  int pf_level = 1;
  // alternative radix schedules (FP32): available, resident CTAs, in use
  bool alt_plane_ok = false, alt_stick_ok = false;
  int alt_plane_occ[3] = {0, 0, 0};
  int alt_stick_occ = 0;
  int sched_plane = 0, sched_stick = 0;  // plane: bit i for mode index i (G->r, r->G, apply)
  bool pdl = true;                       // programmatic dependent launch between stage kernels
  // MIXED_TC plane stages on the 5th-generation tensor cores (grids up to
  // 64): G->r and r->G use them, the z stage then runs in FP32
  bool tc5 = false;
  Tc5Geo tc5g[2] = {};  // G->r, r->G (each with its DFT-matrix image)
  void* d_tc5w = nullptr;
  int tc5_ctas = 0;
  int stick_prec = P_F32;
  // MIXED_TC: the tensor-core kernels the plan was built with (tc5, plane
  // kernel precision, z-stage precision), and whether they are in use; off,
  // the plan runs the FP32 kernels (fftb_plan_set_tensor_cores, autotuner)
  bool tc_avail = false, tc_on = false, tc5_ok = false;
  int plane_tc = P_F32, stick_tc = P_F32;
  // FP32 256-point plane stages with the slab plane split over two-CTA
  // clusters (distributed shared memory): available, the stages that use
  // them (bit i for mode index i: G->r, r->G, apply), clusters resident
  bool cl_ok = false;
  int cl = 0;
  bool xq_all = false;  // every k-point has KF_XY_QUARTER
  bool zq_all = false;  // every k-point has KF_Z_QUARTER
  int cl_count[3] = {0, 0, 0};
  // generic-extent path (extents outside the compiled list, N0 != N1): one
  // runtime-length kernel per axis and a slab buffer S between y and x
  bool generic = false;
  GenParams gen[3] = {};  // per axis x, y, z: the schedules and the line groups of its kernel
  void* d_S = nullptr;
  size_t S_bytes = 0;
  int32_t inject = 0;              // fftb_plan_inject
  int32_t* h_status = nullptr;     // status word in mapped pinned host memory
  int32_t* d_status = nullptr;     // its device address
  // per-kernel timing (fftb_plan_set_timing)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int kind; int a, b; };
  std::vector<Rec> recs;
  int ev_used = 0;
};

namespace {

// the plane stage of mode index i (G->r, r->G, apply) prefetches
bool pf_active(const fftb_plan_s* p, int i) {
  if (p->bg && i < 2) return false;  // the grouped kernels do not prefetch
  if ((p->cl >> i) & 1) return false;  // nor do the cluster kernels
  if (!p->pf_fit[i] || p->pf_level == 0 || ((p->sched_plane >> i) & 1)) return false;
  if (i == 1 && p->layout != 0) return false;  // bulk copies take whole band-major cube rows
  return p->pf_level == 2 || p->pf_occ[i] >= p->plane_occ[i];
}
// resident plane CTAs per SM of the kernel mode index i uses
int occ_in_use(const fftb_plan_s* p, int i) {
  if (p->bg && i < 2) return p->bg_occ[i];
  if ((p->cl >> i) & 1) return 1;
  if ((p->sched_plane >> i) & 1) return p->alt_plane_occ[i];
  return pf_active(p, i) ? p->pf_occ[i] : p->plane_occ[i];
}
// CTAs of one full wave of the plane kernel mode index i uses
int plane_wave(const fftb_plan_s* p, int i) {
  return ((p->cl >> i) & 1) ? plane_cluster_size() * p->cl_count[i] : p->sms * occ_in_use(p, i);
}
// persistent z-stage CTAs of one full wave for the schedule in use
int stick_wave(const fftb_plan_s* p) { return p->sms * (p->sched_stick ? p->alt_stick_occ : p->stick_occ); }
// resident CTAs per SM of the plan's default-schedule z-stage kernels (the
// pruned FP32 ones where every k-point's entries lie within a quarter in z)
int default_stick_occ(const fftb_plan_s* p) {
  const int o = p->stick_prec == P_F32 && p->zq_all ? stick_zq_occupancy(p->n[2])
                                                      : stick_occupancy(p->stick_prec, p->n[2]);
  return std::max(1, o);
}

constexpr size_t kSmemLimit = 227 * 1024;

// For the plan's slab-plane buffer count: kernel shared-memory limits,
// resident CTAs per SM of every plane kernel (plain and prefetching), and
// persistent plane CTAs of one full wave.
fftb_status configure_planes(fftb_plan_s* p) {
  cudaError_t e = prepare_kernels(p->prec_kernel, p->n[0], p->n[1], p->n[2], p->xmax, p->a_bufs, p->a_glob);
  if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
  const int modes[3] = {M_G2R, M_R2G, M_APPLY};
  for (int i = 0; i < 3; ++i) {
    const int occ = plane_occupancy(p->prec_kernel, modes[i], p->n[0], p->n[1], p->xmax, p->a_bufs, p->a_glob);
    if (occ < 1) return fail(FFTB_ERR_UNSUPPORTED, "plane kernel cannot be resident on this device");
    p->plane_occ[i] = occ;
    p->pf_fit[i] = false;
    p->pf_occ[i] = 0;
  }
  if (p->prec_kernel == P_F32) {
    // prefetching plane kernels where their staging fits in shared memory
    for (int i = 0; i < 3; ++i) {
      if (!plane_pf_supported(modes[i], p->n[0], p->n[1], p->a_glob) ||
          plane_pf_smem(modes[i], p->n[0], p->n[1], p->xmax, p->a_bufs, p->tpitch, p->a_glob) > kSmemLimit)
        continue;
      e = prepare_plane_pf(modes[i], p->n[0], p->n[1], p->xmax, p->a_bufs, p->tpitch, p->a_glob);
      if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
      p->pf_occ[i] = plane_pf_occupancy(modes[i], p->n[0], p->n[1], p->xmax, p->a_bufs, p->tpitch, p->a_glob);
      p->pf_fit[i] = p->pf_occ[i] >= 1;
    }
  }
  // the alternative radix schedule of the plane length (FP32, slab planes in shared memory)
  p->alt_plane_ok = false;
  if (p->prec_kernel == P_F32 && !p->a_glob && alt_schedule(p->n[0]) &&
      plane_alt_smem(p->n[0], p->xmax, p->a_bufs) <= kSmemLimit) {
    e = prepare_alt(p->n[0], 0, p->xmax, p->a_bufs);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    bool ok = true;
    for (int i = 0; i < 3; ++i) {
      p->alt_plane_occ[i] = plane_alt_occupancy(modes[i], p->n[0], p->xmax, p->a_bufs);
      ok = ok && p->alt_plane_occ[i] >= 1;
    }
    p->alt_plane_ok = ok;
  }
  if (!p->alt_plane_ok) p->sched_plane = 0;
  // FP32 planes split over two-CTA clusters, where the half plane fits
  p->cl_ok = false;
  const size_t cls = plane_cluster_smem(p->n[0], p->n[1], p->xmax);
  if (p->prec_kernel == P_F32 && cls > 0 && cls <= kSmemLimit) {
    e = prepare_plane_cluster(p->n[0], p->xmax);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    bool ok = true;
    for (int i = 0; i < 3; ++i) {
      p->cl_count[i] = plane_cluster_count(modes[i], p->n[0], p->xmax);
      ok = ok && p->cl_count[i] >= 1;
    }
    p->cl_ok = ok;
  }
  if (!p->cl_ok) p->cl = 0;
  for (int i = 0; i < 3; ++i) p->plane_ctas[i] = plane_wave(p, i);
  return FFTB_OK;
}

// MIXED_TC plans: puts the tensor-core kernels the plan was built with (on)
// or the FP32 kernels, with their alternative schedules and prefetching
// (off), on the plan. Default radix schedules, one full wave of plane CTAs.
fftb_status set_tc(fftb_plan_s* p, bool on) {
  if (!p->tc_avail || on == p->tc_on) return FFTB_OK;
  const bool z_wave = p->tiles == stick_wave(p);
  p->tc_on = on;
  p->tc5 = on && p->tc5_ok;
  p->prec_kernel = on ? p->plane_tc : P_F32;
  p->stick_prec = on ? p->stick_tc : P_F32;
  p->sched_plane = 0;
  p->sched_stick = 0;
  p->bg = on ? 0 : p->bg_size;  // the grouped batch-fastest kernels are FP32 kernels
  fftb_status st = configure_planes(p);
  if (st != FFTB_OK) return st;
  p->stick_occ = default_stick_occ(p);
  p->alt_stick_ok = false;
  if (p->stick_prec == P_F32 && alt_schedule(p->n[2])) {
    cudaError_t e = prepare_alt(0, p->n[2], 0, 1);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    p->alt_stick_occ = stick_alt_occupancy(p->n[2]);
    p->alt_stick_ok = p->alt_stick_occ >= 1;
  }
  if (z_wave) p->tiles = stick_wave(p);
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // recorded with the other kernels
    p->gexec = nullptr;
  }
  return FFTB_OK;
}

bool valid_direction(int d) { return d == FFTB_G_TO_R || d == FFTB_R_TO_G || d == FFTB_ROUNDTRIP || d == FFTB_APPLY_LOCAL; }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void release(fftb_plan_s* p) {
  if (!p) return;
  if (p->d_tables) cudaFree(p->d_tables);
  if (p->d_T) cudaFree(p->d_T);
  if (p->d_A) cudaFree(p->d_A);
  if (p->d_stage_in) cudaFree(p->d_stage_in);
  if (p->d_stage_out) cudaFree(p->d_stage_out);
  if (p->d_stage_cube) cudaFree(p->d_stage_cube);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : p->hev) cudaEventDestroy(e);
  for (cudaStream_t st : p->hs)
    if (st) cudaStreamDestroy(st);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->h_status) cudaFreeHost(p->h_status);
  if (p->d_tc5w) cudaFree(p->d_tc5w);
  if (p->d_S) cudaFree(p->d_S);
  if (p->d_groups) cudaFree(p->d_groups);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
}

}  // namespace

static void debug_report(const fftb_plan_s* p, const char* when);

// n >= 1 with no prime factors but 2, 3 and 5, and at most nmax
static bool generic_extent_ok(int n, int nmax) {
  if (n < 1 || n > nmax) return false;
  for (int f : {2, 3, 5})
    while (n % f == 0) n /= f;
  return n == 1;
}

// Radix schedule of a runtime-length line (generic path): 8 while 8 divides
// what is left, then 4, 2, 3, 5.
static GenAxis generic_axis(int n) {
  GenAxis a{};
  a.n = n;
  int m = n;
  while (m % 8 == 0) { a.r[a.np++] = 8; m /= 8; }
  while (m % 4 == 0) { a.r[a.np++] = 4; m /= 4; }
  while (m % 2 == 0) { a.r[a.np++] = 2; m /= 2; }
  while (m % 3 == 0) { a.r[a.np++] = 3; m /= 3; }
  while (m % 5 == 0) { a.r[a.np++] = 5; m /= 5; }
  return a;
}

// Generic path: the per-axis schedules, the line groups each kernel holds in
// shared memory (up to 64 lines in about 96 KB), and the slab buffer.
static fftb_status setup_generic(fftb_plan_s* p) {
  GenParams g{};
  for (int a = 0; a < 3; ++a) g.ax[a] = generic_axis(p->n[a]);
  for (int a = 0; a < 3; ++a) {
    p->gen[a] = g;
    const int n = p->n[a];
    const int pitch = n | 1;  // odd pitch: Stockham strides of lines held side by side spread over the banks
    const size_t budget = (96u << 10) / p->csize;
    const int lpc = (int)std::max<size_t>(1, std::min<size_t>(64, (budget > (size_t)n ? budget - n : 0) / (2 * (size_t)pitch)));
    p->gen[a].lpc = lpc;
    p->gen[a].pitch = pitch;
  }
  p->S_bytes = (size_t)p->chunk * p->n[2] * std::max(p->xmax, 1) * p->n[1] * p->csize;
  if (cudaMalloc(&p->d_S, p->S_bytes) != cudaSuccess) return fail(FFTB_ERR_ALLOC, "cudaMalloc slab buffer failed");
  for (int a = 0; a < 3; ++a) {
    p->gen[a].S = p->d_S;
    p->gen[a].lim_S = (int64_t)(p->S_bytes / p->csize);
  }
  p->tiles = p->sms * 4;  // CTAs of a generic launch (about 96 KB of shared memory each: two per SM)
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_create(fftb_plan* out, const fftb_desc* d, fftb_direction dir,
                                         fftb_precision prec) {
  if (!out) return fail(FFTB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(FFTB_ERR_INVALID_ARG, "desc is NULL");
  if (!valid_direction(dir)) return fail(FFTB_ERR_INVALID_ARG, "unknown direction");
  if (prec != FFTB_FP64 && prec != FFTB_FP32 && prec != FFTB_MIXED_TC)
    return fail(FFTB_ERR_INVALID_ARG, "unknown precision");
  for (int i = 0; i < 3; ++i)
    if (d->n[i] < 1) return fail(FFTB_ERR_INVALID_ARG, "grid extents must be >= 1");
  if (d->n_kpoints < 1) return fail(FFTB_ERR_INVALID_ARG, "n_kpoints must be >= 1");
  if (d->layout != 0 && d->layout != 1) return fail(FFTB_ERR_INVALID_ARG, "layout must be 0 (band-major) or 1 (batch-fastest)");
  if (d->max_chunk_bands < 0) return fail(FFTB_ERR_INVALID_ARG, "max_chunk_bands must be >= 0");
  if (d->g_list && !d->g_count) return fail(FFTB_ERR_INVALID_ARG, "g_list given without g_count");
  // compiled kernels for the listed extents with N0 == N1; every other extent
  // whose prime factors are 2, 3 and 5 takes the generic-extent path
  const bool fast = grid_size_supported(d->n[0]) && grid_size_supported(d->n[1]) && grid_size_supported(d->n[2]) &&
                    plane_size_supported(d->n[0], d->n[1]);
  if (!fast) {
    for (int i = 0; i < 3; ++i)
      if (!generic_extent_ok(d->n[i], i == 2 ? 256 : 512))
        return fail(FFTB_ERR_UNSUPPORTED,
                    "grid extents must have no prime factors but 2, 3 and 5, with N0, N1 <= 512 and N2 <= 256");
  }

  fftb_plan_s* p = new (std::nothrow) fftb_plan_s();
  if (!p) return fail(FFTB_ERR_ALLOC, "host allocation failed");
  std::memcpy(p->n, d->n, sizeof(p->n));
  p->nk = d->n_kpoints;
  p->layout = d->layout;
  p->dir = dir;
  p->prec = prec;
  p->prec_kernel = (prec == FFTB_FP64) ? P_F64 : (prec == FFTB_MIXED_TC) ? P_TC : P_F32;
  p->generic = !fast;
  if (p->generic && p->prec_kernel == P_TC) p->prec_kernel = P_F32;  // the generic path has no tensor-core stage
  // MIXED_TC stages whose length has no tensor-core pass (no radix-8 pass in
  // its schedule: 24, 96, 160, ...) are FP32 arithmetic: they run on the FP32
  // kernels, with those kernels' alternative schedules and prefetching
  p->stick_prec = p->prec_kernel;
  if (p->prec_kernel == P_TC && !tc_pass_in_schedule(d->n[2])) p->stick_prec = P_F32;
  if (p->prec_kernel == P_TC && !(d->layout == 0 && tc5_supported(d->n[0], d->n[1])) &&
      !tc_pass_in_schedule(d->n[0]) && !tc_pass_in_schedule(d->n[1]))
    p->prec_kernel = P_F32;
  p->csize = (prec == FFTB_FP64) ? 16 : 8;
  p->geo.resize(p->nk);
  p->bands.resize(p->nk);
  const int64_t vol = (int64_t)d->n[0] * d->n[1] * d->n[2];
  int64_t goff = 0;
  for (int k = 0; k < p->nk; ++k) {
    const int32_t b = d->bands ? d->bands[k] : 1;
    if (b < 0) { release(p); return fail(FFTB_ERR_INVALID_ARG, "band counts must be >= 0"); }
    p->bands[k] = b;
    std::vector<int32_t> g;
    std::string err;
    const int32_t* gp;
    int64_t ngw;
    if (d->g_list) {
      ngw = d->g_count[k];
      if (ngw < 0) { release(p); return fail(FFTB_ERR_INVALID_ARG, "g_count must be >= 0"); }
      gp = d->g_list + 3 * goff;
      goff += ngw;
    } else {
      const double zero[3] = {0, 0, 0};
      err = sphere_by_cutoff(d->n, d->radius, d->kshift ? d->kshift + 3 * k : zero, g);
      if (!err.empty()) { release(p); return fail(FFTB_ERR_INVALID_ARG, "k-point " + std::to_string(k) + ": " + err); }
      gp = g.data();
      ngw = (int64_t)g.size() / 3;
    }
    err = build_geometry(d->n, gp, ngw, p->geo[k]);
    if (!err.empty()) { release(p); return fail(FFTB_ERR_INVALID_ARG, "k-point " + std::to_string(k) + ": " + err); }
    p->total_bands += b;
    p->sphere_elems += (int64_t)b * ngw;
    p->cube_elems += (int64_t)b * vol;
    p->smax = std::max(p->smax, p->geo[k].S);
    p->xmax = std::max(p->xmax, p->geo[k].X);
  }
  if (p->total_bands > 65535) { release(p); return fail(FFTB_ERR_UNSUPPORTED, "more than 65535 bands in one plan"); }

  const size_t smem_limit = kSmemLimit;
  if (!p->generic) {
  if (plane_smem(p->prec_kernel, p->n[0], p->n[1], p->xmax, 2) > smem_limit) p->a_bufs = 1;
  if (plane_smem(p->prec_kernel, p->n[0], p->n[1], p->xmax, p->a_bufs) > smem_limit && p->n[0] >= 128) {
    // slab planes in global memory, one buffer per CTA by default (two double
    // their L2 footprint: 30 % slower on the 256^3 round trip); room for two
    // is allocated so that fftb_plan_set_slab_buffers and the autotuner may
    // choose them
    p->a_bufs = 1;
    p->a_glob = true;
  }
  if (stick_smem(p->prec_kernel, p->n[2]) > smem_limit ||
      plane_smem(p->prec_kernel, p->n[0], p->n[1], p->xmax, p->a_bufs, p->a_glob) > smem_limit) {
    release(p);
    return fail(FFTB_ERR_UNSUPPORTED, "plane of this size and precision does not fit in shared memory");
  }
  const int ts = stick_tile(p->prec_kernel, p->n[2]);
  p->tiles = p->smax > 0 ? (p->smax + ts - 1) / ts : 1;
  }  // !generic
  const int32_t smax_pitch = (std::max<int32_t>(p->smax, 1) + 1) & ~1;
  p->tpitch = smax_pitch;

  // band chunk: keep the stick buffer near 48 MB (it then stays in L2), but
  // give every launch at least about 2048 (band, z) planes so the persistent
  // plane CTAs have several planes each; or as requested
  const size_t t_band = (size_t)p->n[2] * smax_pitch * p->csize;
  // (generic path: stick and slab buffers of a chunk within 512 MB)
  const size_t s_band = (size_t)p->n[2] * std::max(p->xmax, 1) * p->n[1] * p->csize;
  int chunk = d->max_chunk_bands > 0
                  ? d->max_chunk_bands
                  : p->generic ? (int)std::max<size_t>(1, (512u << 20) / (t_band + s_band))
                               : (int)std::max<size_t>({(size_t)1, (48u << 20) / t_band,
                                                        (size_t)((2048 + p->n[2] - 1) / p->n[2])});
  chunk = std::max(1, std::min(chunk, std::max(1, p->total_bands)));
  p->chunk = chunk;

  // ---- host tables
  std::vector<int32_t> stick_info, ent_pos, ent_zs, col_info, stick_xy;
  std::vector<BandInfo> band;
  std::vector<int16_t> xmap;
  int32_t sticks_so_far = 0;
  std::vector<KInfo> kinfo(p->nk);
  int64_t sph = 0, ent_base = 0;
  for (int k = 0; k < p->nk; ++k) {
    const KGeom& G = p->geo[k];
    const size_t first_band = band.size();
    // band-major: [B_k][ngw_k] and [B_k][N2][N1][N0]; batch-fastest (Sec. 3.3,
    // the batch dimension declared first): [ngw_k][B_k] and [N2][N1][N0][B_k]
    const bool bf = p->layout == 1;
    for (int b = 0; b < p->bands[k]; ++b) {
      BandInfo bi{};
      bi.sph = sph + (bf ? (int64_t)b : (int64_t)b * G.ngw);
      bi.cube = (int64_t)first_band * vol + (bf ? (int64_t)b : (int64_t)b * vol);
      band.push_back(bi);
    }
    kinfo[k].bstride = bf ? std::max(p->bands[k], 1) : 1;
    sph += (int64_t)p->bands[k] * G.ngw;
    kinfo[k].S = G.S;
    kinfo[k].X = G.X;
    kinfo[k].stick_base = sticks_so_far;
    kinfo[k].xmap_base = (int32_t)xmap.size();
    kinfo[k].col_base = (int32_t)(col_info.size() / 4);
    kinfo[k].flags = (G.contiguous_columns ? KF_CONTIGUOUS_COLUMNS : 0) | (G.canonical_sticks ? KF_CANONICAL_STICKS : 0);
    {
      bool quarter = true;  // every occupied stick within [-N0/4, N0/4] x [-N1/4, N1/4]
      for (int32_t x = 0; x < d->n[0]; ++x)
        if (G.xmap[x] >= 0 && x > d->n[0] / 4 && x < d->n[0] - d->n[0] / 4) quarter = false;
      for (int32_t xy : G.stick_xy) {
        const int32_t y = xy & 0xFFFF;
        if (y > d->n[1] / 4 && y < d->n[1] - d->n[1] / 4) quarter = false;
      }
      if (quarter) kinfo[k].flags |= KF_XY_QUARTER;
      p->xq_all = (k == 0 || p->xq_all) && quarter;
      bool zquarter = true;  // every entry within |z| <= N2/4
      for (int32_t zs : G.ent_zs) {
        const int32_t z = (int32_t)((uint32_t)zs >> 24);
        if (z > d->n[2] / 4 && z < d->n[2] - d->n[2] / 4) zquarter = false;
      }
      if (zquarter) kinfo[k].flags |= KF_Z_QUARTER;
      p->zq_all = (k == 0 || p->zq_all) && zquarter;
    }
    sticks_so_far += G.S;
    stick_records(G, d->n, (int32_t)ent_base, stick_info);
    for (int32_t v : G.ent_pos) ent_pos.push_back(v);
    for (int32_t v : G.ent_zs) ent_zs.push_back(v);
    for (int16_t v : G.xmap) xmap.push_back(v);
    slab_records(G, d->n, col_info);
    for (size_t b = first_band; b < band.size(); ++b) band[b].ki = kinfo[k];
    for (int32_t v : G.stick_xy) stick_xy.push_back(v);
    ent_base += G.ngw;
  }
  if (ent_base >= (int64_t(1) << 31)) { release(p); return fail(FFTB_ERR_UNSUPPORTED, "total sphere entries above 2^31"); }
  for (const BandInfo& bi : band) p->band_sph.push_back(bi.sph);
  p->band_sph.push_back(sph);
  TableParts tp;
  tp.band = std::move(band);
  tp.kinfo = std::move(kinfo);
  tp.stick_info = std::move(stick_info);
  tp.ent_pos = std::move(ent_pos);
  tp.ent_zs = std::move(ent_zs);
  tp.stick_xy = std::move(stick_xy);
  tp.col_info = std::move(col_info);
  tp.xmap = std::move(xmap);
  for (int dd = 0; dd < 3; ++dd) {
    if (p->prec_kernel == P_F64) make_twiddles<double>(p->n[dd], tp.tw[dd]);
    else make_twiddles<float>(p->n[dd], tp.tw[dd]);
  }
  const TableLayout tl = table_layout(tp);
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) { release(p); return cuda_fail(e, "cudaGetDevice"); }
  e = cudaMalloc(&p->d_tables, tl.total);
  if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaMalloc tables failed"); }
  p->tables_bytes = tl.total;
  std::vector<unsigned char> blob(tl.total);
  table_fill(tp, tl, blob.data());
  e = cudaMemcpy(p->d_tables, blob.data(), tl.total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { release(p); return cuda_fail(e, "cudaMemcpy tables"); }
  Geo& g = p->g;
  table_geo(g, p->d_tables, tl);
  g.n0 = p->n[0];
  g.n1 = p->n[1];
  g.n2 = p->n[2];
  g.smax = smax_pitch;
  g.xmax = p->xmax;

  p->T_bytes = (size_t)chunk * p->n[2] * smax_pitch * p->csize;
  e = cudaMalloc(&p->d_T, p->T_bytes);
  if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaMalloc stick scratch failed"); }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) { release(p); return cuda_fail(e, "device attribute"); }
  p->sms = sms;
  if (p->generic) {
    fftb_status gst = setup_generic(p);
    if (gst != FFTB_OK) { release(p); return gst; }
  }
  if (!p->generic) {
  fftb_status cst = configure_planes(p);
  if (cst != FFTB_OK) { release(p); return cst; }
  if (p->a_bufs == 2 && !p->a_glob) {
    // one slab buffer when that makes more CTAs resident (large grids)
    const int occ2 = occ_in_use(p, 0) + occ_in_use(p, 1) + occ_in_use(p, 2);
    p->a_bufs = 1;
    cst = configure_planes(p);
    if (cst != FFTB_OK) { release(p); return cst; }
    if (occ_in_use(p, 0) + occ_in_use(p, 1) + occ_in_use(p, 2) <= occ2) {
      p->a_bufs = 2;
      cst = configure_planes(p);
      if (cst != FFTB_OK) { release(p); return cst; }
    }
  }
  // the tcgen05 plane kernels read and write band-major cube planes
  if (p->prec_kernel == P_TC && p->layout == 0 && tc5_supported(p->n[0], p->n[1])) {
    // union over k-points of the occupied x values and the stick y values
    int xlo = 1 << 30, xhi = -(1 << 30), ylo = 1 << 30, yhi = -(1 << 30);
    bool columns_ok = true;
    for (int k = 0; k < p->nk; ++k) {
      const KGeom& G = p->geo[k];
      columns_ok = columns_ok && G.contiguous_columns;
      std::vector<int32_t> rec;
      slab_records(G, p->n, rec);
      for (int x = 0; x < p->n[0]; ++x) {
        const int xi = G.xmap[x];
        if (xi < 0) continue;
        const int xs = x < p->n[0] - p->n[0] / 2 ? x : x - p->n[0];
        xlo = std::min(xlo, xs);
        xhi = std::max(xhi, xs);
        if (rec[4 * xi + 1] > 0) {
          ylo = std::min(ylo, rec[4 * xi + 2]);
          yhi = std::max(yhi, rec[4 * xi + 2] + rec[4 * xi + 1] - 1);
        }
      }
    }
    if (columns_ok && xhi >= xlo && yhi >= ylo) {
      const Tc5Geo g0{xlo, xhi - xlo + 1, ylo, yhi - ylo + 1, nullptr};
      int occ_a = 0, occ_b = 0;
      bool fits = tc5_smem(M_G2R, p->n[0], g0, p->tpitch) <= kSmemLimit &&
                  tc5_smem(M_R2G, p->n[0], g0, p->tpitch) <= kSmemLimit;
      if (fits) {
        e = tc5_prepare(M_G2R, p->n[0], g0, p->tpitch, &occ_a);
        if (e == cudaSuccess) e = tc5_prepare(M_R2G, p->n[0], g0, p->tpitch, &occ_b);
        if (e != cudaSuccess) { release(p); return cuda_fail(e, "tensor-core kernel attributes"); }
        if (occ_a >= 1 && occ_b >= 1) {
          // the DFT-matrix images of both directions, built once on the device
          const size_t wa = align_up(tc5_weight_bytes(M_G2R, p->n[0], g0), 256);
          const size_t wb = tc5_weight_bytes(M_R2G, p->n[0], g0);
          e = cudaMalloc(&p->d_tc5w, wa + wb);
          if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaMalloc tensor-core matrices failed"); }
          p->tc5g[0] = g0;
          p->tc5g[0].w = p->d_tc5w;
          p->tc5g[1] = g0;
          p->tc5g[1].w = static_cast<unsigned char*>(p->d_tc5w) + wa;
          e = tc5_build_weights(M_G2R, p->n[0], p->tc5g[0], p->g.tw0, const_cast<void*>(p->tc5g[0].w));
          if (e == cudaSuccess) e = tc5_build_weights(M_R2G, p->n[0], p->tc5g[1], p->g.tw0, const_cast<void*>(p->tc5g[1].w));
          if (e != cudaSuccess) { release(p); return cuda_fail(e, "tensor-core matrices"); }
          p->tc5 = true;
          p->tc5_ctas = sms * std::min(occ_a, occ_b);
          p->stick_prec = P_F32;
          e = prepare_kernels(P_F32, p->n[0], p->n[1], p->n[2], p->xmax, p->a_bufs, false);
          if (e != cudaSuccess) { release(p); return cuda_fail(e, "kernel attributes"); }
        }
      }
    }
  }
  if (p->prec != FFTB_FP64 && p->zq_all) {  // FP32 z stages (MIXED_TC: once its tensor cores are off)
    e = prepare_stick_zq(p->n[2]);
    if (e != cudaSuccess) { release(p); return cuda_fail(e, "kernel attributes"); }
  }
  p->stick_occ = default_stick_occ(p);
  if (p->stick_prec == P_F32 && alt_schedule(p->n[2])) {
    e = prepare_alt(0, p->n[2], 0, 1);
    if (e != cudaSuccess) { release(p); return cuda_fail(e, "kernel attributes"); }
    p->alt_stick_occ = stick_alt_occupancy(p->n[2]);
    p->alt_stick_ok = p->alt_stick_occ >= 1;
  }
  p->tiles = sms * p->stick_occ;  // z stage: one wave of persistent CTAs (the autotuner may pick one warp per task pair)
  p->tc5_ok = p->tc5;
  p->plane_tc = p->prec_kernel;
  p->stick_tc = p->stick_prec;
  p->tc_avail = p->tc5 || p->prec_kernel == P_TC || p->stick_prec == P_TC;
  p->tc_on = p->tc_avail;
  }  // !generic
  e = cudaHostAlloc(reinterpret_cast<void**>(&p->h_status), sizeof(int32_t), cudaHostAllocMapped);
  if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaHostAlloc status word failed"); }
  *p->h_status = 0;
  e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&p->d_status), p->h_status, 0);
  if (e != cudaSuccess) { release(p); return cuda_fail(e, "status word device address"); }
  if (!p->generic && p->layout == 1 && (p->prec_kernel == P_F32 || p->tc_avail) && p->n[0] == p->n[1] &&
      p->total_bands > 0) {
    // batch-fastest: plane stages over groups of bands of one k-point, where they fit (FP32
    // kernels: in MIXED_TC plans while the tensor cores are off)
    const int bgs = plane_bg_group(p->n[0]);
    if (bgs > 1 && plane_bg_smem(p->n[0], p->n[1], p->xmax, bgs) <= kSmemLimit) {
      e = prepare_plane_bg(p->n[0], p->xmax);
      if (e != cudaSuccess) { release(p); return cuda_fail(e, "kernel attributes"); }
      const int o0 = plane_bg_occupancy(M_G2R, p->n[0], p->xmax), o1 = plane_bg_occupancy(M_R2G, p->n[0], p->xmax);
      if (o0 >= 1 && o1 >= 1) {
        p->band_grp.assign(p->total_bands, -1);
        int b0 = 0;
        for (int k = 0; k < p->nk; ++k) {
          for (int b = 0; b < p->bands[k]; b += bgs) {
            p->band_grp[b0 + b] = (int32_t)p->groups.size();
            p->groups.push_back(make_int2(b0 + b, std::min(bgs, p->bands[k] - b)));
          }
          b0 += p->bands[k];
        }
        e = cudaMalloc(&p->d_groups, p->groups.size() * sizeof(int2));
        if (e == cudaSuccess)
          e = cudaMemcpy(p->d_groups, p->groups.data(), p->groups.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "band group table"); }
        // a launch takes whole groups: the stick buffer holds at least one
        const size_t need = (size_t)std::max(p->chunk, bgs) * p->n[2] * p->tpitch * p->csize;
        if (need > p->T_bytes) {
          cudaFree(p->d_T);
          p->d_T = nullptr;
          p->T_bytes = 0;
          if (cudaMalloc(&p->d_T, need) != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaMalloc stick scratch failed"); }
          p->T_bytes = need;
        }
        p->bg_size = bgs;
        p->bg = p->tc_on ? 0 : bgs;
        p->bg_occ[0] = o0;
        p->bg_occ[1] = o1;
        for (int i = 0; i < 2; ++i) p->plane_ctas[i] = plane_wave(p, i);
      }
    }
  }
  if (p->a_glob) {
    // one slab-plane block (room for two buffers) per persistent CTA: as many as the
    // most resident CTAs of any plane kernel variant (plain or prefetching)
    int occ = 1;
    for (int i = 0; i < 3; ++i) occ = std::max({occ, p->plane_occ[i], p->pf_fit[i] ? p->pf_occ[i] : 0});
    const int ctas = std::max({p->sms * occ, p->plane_ctas[0], p->plane_ctas[1], p->plane_ctas[2]});
    p->a_blocks = ctas;
    p->A_bytes = (size_t)ctas * 2 * p->n[1] * (size_t)(p->xmax + 16) * p->csize;
    e = cudaMalloc(&p->d_A, p->A_bytes);
    if (e != cudaSuccess) { release(p); return fail(FFTB_ERR_ALLOC, "cudaMalloc slab planes failed"); }
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { release(p); return cuda_fail(e, "plan synchronise"); }
  debug_report(p, "plan created");
  *out = p;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_ngw(fftb_plan p, int32_t k, int64_t* ngw) {
  if (!p || !ngw) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  if (k < 0 || k >= p->nk) return fail(FFTB_ERR_INVALID_ARG, "k-point out of range");
  *ngw = p->geo[k].ngw;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_sphere(fftb_plan p, int32_t k, int32_t* g_out) {
  if (!p || !g_out) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  if (k < 0 || k >= p->nk) return fail(FFTB_ERR_INVALID_ARG, "k-point out of range");
  if (!p->geo[k].g.empty()) std::memcpy(g_out, p->geo[k].g.data(), p->geo[k].g.size() * 4);
  return FFTB_OK;
}

static int count_chunks(const fftb_plan_s* p, int first, int bands);
// output scalings an execute launches: the cube by scale_g2r (G->r, round
// trip), the sphere by the product of the factors its path applies
static double sphere_scale(const fftb_plan_s* p) {
  if (p->dir == FFTB_G_TO_R) return 1.0;
  return p->scale_r2g * ((p->dir == FFTB_ROUNDTRIP || p->dir == FFTB_APPLY_LOCAL) ? p->scale_g2r : 1.0);
}
static int scale_launches(const fftb_plan_s* p) {
  const bool cube = p->scale_g2r != 1.0 && (p->dir == FFTB_G_TO_R || p->dir == FFTB_ROUNDTRIP);
  return (cube ? 1 : 0) + (sphere_scale(p) != 1.0 ? 1 : 0);
}
// Stage kernels per band chunk (the generic path runs the y and x stages as
// two kernels, and the fused apply as y, x-apply, y)
static int kernels_per_chunk(const fftb_plan_s* p) {
  const int g = p->generic ? 1 : 0;
  switch (p->dir) {
    case FFTB_G_TO_R: return 2 + g;
    case FFTB_R_TO_G: return 2 + g;
    case FFTB_ROUNDTRIP: return 4 + 2 * g;
    case FFTB_APPLY_LOCAL: return 3 + 2 * g;
  }
  return 0;
}

// FFTB_DEBUG=1 in the environment: one line on stderr per plan decision
// (after creation and after autotuning) with the launch configuration.
static void debug_report(const fftb_plan_s* p, const char* when) {
  const char* e = std::getenv("FFTB_DEBUG");
  if (!e || !*e || std::strcmp(e, "0") == 0) return;
  fftb_plan_info_t i{};
  fftb_plan_get_info(const_cast<fftb_plan_s*>(p), &i);
  std::fprintf(stderr,
               "[fftb] %s: grid %dx%dx%d dir %d prec %d layout %d k-points %d bands %d | sticks %d slabs %d | "
               "chunk %d bands, %lld kernels/execute | z CTAs %d, plane CTAs %d | slab buffers %d%s | "
               "prefetch mask %d | schedule plane %d stick %d | tcgen05 %d | mma.sync %d | clusters %d | "
               "band group %d | PDL %d | scratch %lld bytes\n",
               when, p->n[0], p->n[1], p->n[2], (int)p->dir, (int)p->prec, p->layout, p->nk, p->total_bands,
               i.max_sticks, i.max_slabs, i.chunk_bands, (long long)i.kernels_per_execute, i.stick_ctas,
               i.plane_ctas, i.slab_buffers, i.slab_planes_global ? " (global)" : "", i.prefetch,
               i.radix_schedule_plane, i.radix_schedule_stick, i.tensor_core_planes, i.tensor_core_passes,
               i.plane_clusters & 7, i.plane_band_group, i.dependent_launch, (long long)i.scratch_bytes);
}

FFTB_EXPORT fftb_status fftb_plan_get_info(fftb_plan p, fftb_plan_info_t* info) {
  if (!p || !info) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  info->sphere_elems = p->sphere_elems;
  info->cube_elems = p->cube_elems;
  info->scratch_bytes = (int64_t)(p->T_bytes + p->tables_bytes + p->S_bytes + p->A_bytes);
  info->total_bands = p->total_bands;
  info->max_sticks = p->smax;
  info->max_slabs = p->xmax;
  info->chunk_bands = p->chunk;
  info->kernels_per_execute = count_chunks(p, 0, p->total_bands) * kernels_per_chunk(p) +
                              (p->total_bands > 0 ? scale_launches(p) : 0);
  info->scale_g2r = p->scale_g2r;
  info->scale_r2g = p->scale_r2g;
  info->complex_bytes = p->csize;
  info->stick_ctas = p->tiles;
  info->plane_ctas = p->plane_ctas[p->dir == FFTB_R_TO_G ? 1 : p->dir == FFTB_APPLY_LOCAL ? 2 : 0];
  info->prefetch = 0;
  for (int i = 0; i < 3; ++i)
    if (pf_active(p, i)) info->prefetch |= 1 << i;
  info->slab_buffers = p->a_bufs;
  const int used = p->dir == FFTB_G_TO_R ? 1 : p->dir == FFTB_R_TO_G ? 2 : p->dir == FFTB_APPLY_LOCAL ? 4 : 3;
  info->slab_planes_global = p->a_glob && (p->cl & used) != used ? 1 : 0;
  info->plane_clusters = p->cl | (p->cl_ok ? 8 : 0);
  {
    const int n = p->n[0];
    const bool z = !p->generic && p->zq_all && p->stick_prec == P_F32 && !p->sched_stick;
    const bool planes = !p->generic && p->xq_all && p->prec_kernel == P_F32 && !p->tc5 && (p->cl & used) == 0 &&
                        (n == 64 || n == 96 || n == 128 || n == 256 || (n == 160 && p->sched_plane));
    info->pruned_lines = (z ? 1 : 0) | (planes ? 2 : 0);
  }
  info->tensor_core_planes = p->tc5 ? 3 : 0;
  info->radix_schedule_plane = p->sched_plane;
  info->radix_schedule_stick = p->sched_stick;
  info->dependent_launch = p->pdl ? 1 : 0;
  info->plane_band_group = p->bg;
  info->graph_launches = p->graph_launches;
  info->generic_path = p->generic ? 1 : 0;
  info->tensor_core_passes = (p->stick_prec == P_TC ? 1 : 0) | (p->prec_kernel == P_TC && !p->tc5 ? 2 : 0);
  info->tensor_cores_available = p->tc_avail ? 1 : 0;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_set_potential(fftb_plan p, const void* v) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (v && (reinterpret_cast<uintptr_t>(v) % (p->csize / 2)) != 0)
    return fail(FFTB_ERR_INVALID_ARG, "potential pointer misaligned");
  p->d_V = v;
  return FFTB_OK;
}

enum StageKind { K_STICK_G2R = 0, K_PLANE_G2R = 1, K_PLANE_R2G = 2, K_STICK_R2G = 3, K_PLANE_APPLY = 4 };
static const char* const kStageName[5] = {"fftb z stage G->r", "fftb y/x stages G->r", "fftb x/y stages r->G",
                                          "fftb z stage r->G", "fftb y/x apply"};

// RAII NVTX range
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static cudaEvent_t next_event(fftb_plan_s* p, int* idx) {
  if (p->ev_used == (int)p->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->ev_pool.push_back(e);
  }
  *idx = p->ev_used;
  return p->ev_pool[p->ev_used++];
}

// Launches one stage kernel, bracketed by events when timing is enabled.
static cudaError_t stage(fftb_plan_s* p, int kind, const Launch& L) {
  NvtxRange range(kStageName[kind]);
  int a = -1, b = -1;
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (p->timing) {
    ea = next_event(p, &a);
    eb = next_event(p, &b);
    if (!ea || !eb) return cudaErrorMemoryAllocation;
    cudaEventRecord(ea, L.stream);
  }
  cudaError_t e;
  const int pk = p->prec_kernel;
  if (p->generic) {
    // z, y, x stages as separate runtime-length kernels (stage 0 z, 1 y, 2 x, 3 x apply)
    const bool f64 = pk == P_F64;
    const int ctas = p->tiles;
    auto gen = [&](int st, int sign) { return launch_generic(f64, st, sign, L, p->gen[st == 3 ? 0 : 2 - st], ctas); };
    int n = 0;
    switch (kind) {
      case K_STICK_G2R: e = gen(0, +1); n = 1; break;
      case K_PLANE_G2R: e = gen(1, +1); if (e == cudaSuccess) e = gen(2, +1); n = 2; break;
      case K_PLANE_R2G: e = gen(2, -1); if (e == cudaSuccess) e = gen(1, -1); n = 2; break;
      case K_STICK_R2G: e = gen(0, -1); n = 1; break;
      default:
        e = gen(1, +1);
        if (e == cudaSuccess) e = gen(3, +1);
        if (e == cudaSuccess) e = gen(1, -1);
        n = 3;
        break;
    }
    if (e == cudaSuccess) p->launches += n;
    if (p->timing) {
      cudaEventRecord(eb, L.stream);
      p->recs.push_back({kind, a, b});
    }
    return e;
  }
  // bulk copies read the cube from 16-byte aligned rows
  const bool cube_in_16 = (reinterpret_cast<uintptr_t>(L.cube_in) % 16) == 0;
  switch (kind) {
    case K_STICK_G2R:
      e = p->sched_stick                         ? launch_stick_alt(M_G2R, L, p->tiles)
          : (p->stick_prec == P_F32 && p->zq_all) ? launch_stick_zq(M_G2R, L, p->tiles)
                                                  : launch_stick(p->stick_prec, M_G2R, L, p->tiles);
      break;
    case K_PLANE_G2R: {
      Launch Lp = L;
      Lp.plane_ctas = p->plane_ctas[0];
      Lp.pf = pf_active(p, 0);
      if (p->bg) e = launch_plane_bg(M_G2R, Lp);
      else if (p->tc5) e = tc5_launch(M_G2R, Lp, p->tc5g[0], p->tc5_ctas);
      else if (p->cl & 1) e = launch_plane_cluster(M_G2R, Lp);
      else if (p->sched_plane & 1) e = launch_plane_alt(M_G2R, Lp);
      else e = Lp.pf ? launch_plane_pf(M_G2R, Lp) : launch_plane(pk, M_G2R, Lp);
      break;
    }
    case K_PLANE_R2G: {
      Launch Lp = L;
      Lp.plane_ctas = p->plane_ctas[1];
      Lp.pf = pf_active(p, 1) && cube_in_16;
      if (p->bg) e = launch_plane_bg(M_R2G, Lp);
      else if (p->tc5 && cube_in_16) e = tc5_launch(M_R2G, Lp, p->tc5g[1], p->tc5_ctas);
      else if (p->cl & 2) e = launch_plane_cluster(M_R2G, Lp);
      else if (p->sched_plane & 2) {
        Lp.pf = cube_in_16;  // the alternative kernel loads whole cube rows by bulk copies
        e = launch_plane_alt(M_R2G, Lp);
      }
      else e = Lp.pf ? launch_plane_pf(M_R2G, Lp) : launch_plane(pk, M_R2G, Lp);
      break;
    }
    case K_STICK_R2G:
      e = p->sched_stick                         ? launch_stick_alt(M_R2G, L, p->tiles)
          : (p->stick_prec == P_F32 && p->zq_all) ? launch_stick_zq(M_R2G, L, p->tiles)
                                                  : launch_stick(p->stick_prec, M_R2G, L, p->tiles);
      break;
    default: {
      Launch Lp = L;
      Lp.plane_ctas = p->plane_ctas[2];
      Lp.pf = pf_active(p, 2);
      if (p->cl & 4) e = launch_plane_cluster(M_APPLY, Lp);
      else if (p->sched_plane & 4) e = launch_plane_alt(M_APPLY, Lp);
      else e = Lp.pf ? launch_plane_pf(M_APPLY, Lp) : launch_plane(pk, M_APPLY, Lp);
      break;
    }
  }
  if (e == cudaSuccess) ++p->launches;
  if (p->timing) {
    cudaEventRecord(eb, L.stream);
    p->recs.push_back({kind, a, b});
  }
  return e;
}

static bool aligned(const void* q, int a) { return (reinterpret_cast<uintptr_t>(q) % (uintptr_t)a) == 0; }

// The band chunk that starts at band b0 (< end): the plan's chunk of bands,
// or for grouped plans whole band groups up to that many bands (at least one
// group; b0 starts a group). Sets the chunk's bands and its groups.
static void chunk_at(const fftb_plan_s* p, int b0, int end, int* nb, int* g0, int* ng) {
  if (!p->bg) {
    *nb = std::min(p->chunk, end - b0);
    *g0 = *ng = 0;
    return;
  }
  int g = p->band_grp[b0], n = 0;
  *g0 = g;
  while (g < (int)p->groups.size() && p->groups[g].x < end && (n == 0 || n + p->groups[g].y <= p->chunk)) {
    n += p->groups[g].y;
    ++g;
  }
  *nb = n;
  *ng = g - *g0;
}
static int count_chunks(const fftb_plan_s* p, int first, int bands) {
  int n = 0;
  for (int b0 = first, nb = 0, g0, ng; b0 < first + bands; b0 += nb, ++n) chunk_at(p, b0, first + bands, &nb, &g0, &ng);
  return n;
}

// Enqueues every band chunk's stages for the bands [first, first + bands)
// (grouped plans: from a group start, whole groups).
static fftb_status enqueue(fftb_plan_s* p, int bands, const void* in, void* out, void* cube, cudaStream_t s,
                           int first = 0) {
  Launch L{};
  L.g = p->g;
  L.T = p->d_T;
  L.V = p->d_V;
  L.a_bufs = p->a_bufs;
  L.a_glob = p->d_A;
  L.a_blocks = p->a_blocks;
  L.inject = p->inject;
  L.status = p->d_status;
  L.pdl = p->pdl ? 1 : 0;
  L.xq = p->xq_all ? 1 : 0;
  L.zq = p->zq_all ? 1 : 0;
  L.groups = static_cast<const int2*>(p->d_groups);
  L.lim_sph = p->sphere_elems;
  L.lim_cube = p->cube_elems;
  L.lim_T = (int64_t)(p->T_bytes / p->csize);
  L.lim_V = (int64_t)p->n[0] * p->n[1] * p->n[2];
  L.stream = s;
  if (p->bg && (first >= p->total_bands || p->band_grp[first] < 0))
    return fail(FFTB_ERR_INVALID_ARG, "a grouped launch must start at a band group");
  for (int b0 = first, nb = 0; b0 < first + bands; b0 += nb) {
    chunk_at(p, b0, first + bands, &nb, &L.grp0, &L.ngrp);
    L.band0 = b0;
    L.nb = nb;
    cudaError_t e = cudaSuccess;
    switch (p->dir) {
      case FFTB_G_TO_R:
        L.sph_in = in;
        L.cube_out = out;
        e = stage(p, K_STICK_G2R, L);
        if (e == cudaSuccess) e = stage(p, K_PLANE_G2R, L);
        break;
      case FFTB_R_TO_G:
        L.cube_in = in;
        L.sph_out = out;
        e = stage(p, K_PLANE_R2G, L);
        if (e == cudaSuccess) e = stage(p, K_STICK_R2G, L);
        break;
      case FFTB_ROUNDTRIP:
        L.sph_in = in;
        L.cube_out = cube;
        L.cube_in = cube;
        L.sph_out = out;
        e = stage(p, K_STICK_G2R, L);
        if (e == cudaSuccess) e = stage(p, K_PLANE_G2R, L);
        if (e == cudaSuccess) e = stage(p, K_PLANE_R2G, L);
        if (e == cudaSuccess) e = stage(p, K_STICK_R2G, L);
        break;
      case FFTB_APPLY_LOCAL:
        L.sph_in = in;
        L.sph_out = out;
        e = stage(p, K_STICK_G2R, L);
        if (e == cudaSuccess) e = stage(p, K_PLANE_APPLY, L);
        if (e == cudaSuccess) e = stage(p, K_STICK_R2G, L);
        break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  }
  // Optional normalisation, after every chunk's stages, over this call's
  // output ranges (whole k-point blocks in the batch-fastest layout). The
  // maps are linear: the round trip's r->G stage reads the unscaled cube and
  // its sphere output takes both factors.
  const int64_t vol = (int64_t)p->n[0] * p->n[1] * p->n[2];
  if (p->scale_g2r != 1.0 && (p->dir == FFTB_G_TO_R || p->dir == FFTB_ROUNDTRIP)) {
    unsigned char* c = static_cast<unsigned char*>(p->dir == FFTB_G_TO_R ? out : cube);
    cudaError_t e = launch_scale(p->csize, c + (size_t)first * vol * p->csize, (int64_t)bands * vol, p->scale_g2r, L,
                                 p->sms);
    if (e != cudaSuccess) return cuda_fail(e, "scale launch");
    ++p->launches;
  }
  const double ss = sphere_scale(p);
  if (ss != 1.0) {
    unsigned char* o = static_cast<unsigned char*>(out);
    const int64_t a = p->band_sph[first], b = p->band_sph[std::min(first + bands, p->total_bands)];
    cudaError_t e = launch_scale(p->csize, o + (size_t)a * p->csize, b - a, ss, L, p->sms);
    if (e != cudaSuccess) return cuda_fail(e, "scale launch");
    ++p->launches;
  }
  return FFTB_OK;
}

// Direct launches, or the recorded CUDA graph of this buffer set. The legacy
// default stream cannot be captured: for it the graph is recorded on a
// plan-owned stream and launched on the default stream.
static fftb_status launch_all(fftb_plan_s* p, int bands, const void* in, void* out, void* cube, cudaStream_t s) {
  bool graph = p->use_graph && !p->timing && bands == p->total_bands;
  if (graph && s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) graph = false;
  }
  if (!graph) return enqueue(p, bands, in, out, cube, s);
  if (!s && !p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(FFTB_ERR_CUDA, "capture stream creation failed");
  cudaStream_t cap = s ? s : p->cap_stream;
  const int64_t per_exec = (int64_t)count_chunks(p, 0, p->total_bands) * kernels_per_chunk(p) + scale_launches(p);
  if (!(p->gexec && p->g_in == in && p->g_out == out && p->g_cube == cube && p->g_V == p->d_V)) {
    const int64_t before = p->launches;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    fftb_status st = enqueue(p, bands, in, out, cube, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    p->launches = before;
    if (st != FFTB_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    if (p->gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(p->gexec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
      }
    }
    if (!p->gexec) e = cudaGraphInstantiate(&p->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->gexec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    p->g_in = in;
    p->g_out = out;
    p->g_cube = cube;
    p->g_V = p->d_V;
  }
  cudaError_t e = cudaGraphLaunch(p->gexec, s);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  ++p->graph_launches;
  p->launches += per_exec;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_execute(fftb_plan p, const void* in, void* out, void* cube, void* stream) {
  NvtxRange range("fftb_execute");
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->total_bands == 0) return FFTB_OK;
  if (!in || !out) return fail(FFTB_ERR_INVALID_ARG, "in and out must be device pointers");
  if (!aligned(in, p->csize) || !aligned(out, p->csize) || (cube && !aligned(cube, p->csize)))
    return fail(FFTB_ERR_INVALID_ARG, "buffers must be aligned to the complex element size");
  if (in == out) return fail(FFTB_ERR_INVALID_ARG, "in and out must not overlap");
  if (p->dir == FFTB_ROUNDTRIP && !cube) return fail(FFTB_ERR_INVALID_ARG, "ROUNDTRIP needs a cube buffer");
  if (p->dir != FFTB_ROUNDTRIP && cube) return fail(FFTB_ERR_INVALID_ARG, "cube buffer only for ROUNDTRIP");
  if (p->dir == FFTB_APPLY_LOCAL && !p->d_V) return fail(FFTB_ERR_INVALID_ARG, "APPLY_LOCAL needs fftb_set_potential");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(FFTB_ERR_INVALID_ARG, "current device differs from the plan's device");

  return launch_all(p, p->total_bands, in, out, cube, static_cast<cudaStream_t>(stream));
}

// The error a nonzero device status word stands for (bits STATUS_BOUNDS of a
// checked build, else a bounded wait that ran out).
static fftb_status device_status_error(int32_t st, const char* tail) {
  if (st & 2)
    return fail(FFTB_ERR_DEVICE_BOUNDS, std::string("a checked kernel found an index outside its buffer; ") + tail);
  return fail(FFTB_ERR_DEVICE_TIMEOUT, std::string("a plane-stage wait for an asynchronous copy ran out; ") + tail);
}

static fftb_status ensure(void** ptr, size_t* have, size_t need) {
  if (*have >= need && *ptr) return FFTB_OK;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *have = 0;
  if (cudaMalloc(ptr, need ? need : 16) != cudaSuccess) return fail(FFTB_ERR_ALLOC, "cudaMalloc staging failed");
  *have = need;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_execute_host(fftb_plan p, const void* in_host, void* out_host, void* cube_dev,
                                          void* stream) {
  NvtxRange range("fftb_execute_host");
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (!in_host || !out_host) return fail(FFTB_ERR_INVALID_ARG, "in_host and out_host must be given");
  if (p->total_bands == 0) return FFTB_OK;
  if (p->dir == FFTB_APPLY_LOCAL && !p->d_V) return fail(FFTB_ERR_INVALID_ARG, "APPLY_LOCAL needs fftb_set_potential");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(FFTB_ERR_INVALID_ARG, "current device differs from the plan's device");
  const size_t sph_b = (size_t)p->sphere_elems * p->csize, cube_b = (size_t)p->cube_elems * p->csize;
  const bool in_cube = p->dir == FFTB_R_TO_G, out_cube = p->dir == FFTB_G_TO_R;
  fftb_status st = ensure(&p->d_stage_in, &p->stage_in_bytes, in_cube ? cube_b : sph_b);
  if (st == FFTB_OK) st = ensure(&p->d_stage_out, &p->stage_out_bytes, out_cube ? cube_b : sph_b);
  if (st == FFTB_OK && p->dir == FFTB_ROUNDTRIP && !cube_dev) {
    st = ensure(&p->d_stage_cube, &p->stage_cube_bytes, cube_b);
    cube_dev = p->d_stage_cube;
  }
  if (st != FFTB_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Band pieces pipelined over three streams: the copy in of piece i + 1 and
  // the copy out of piece i - 1 overlap the transform of piece i, so only the
  // first piece's copy in and the last piece's copy out are exposed. Band-major
  // batches split into pieces of about 8192 (band, z) planes, at least two and
  // at most 16, with a first and a last piece of about 2048 planes where the
  // batch holds at least 32768 (a piece's launches stay large enough to fill
  // the GPU: on the 64^3 x 64 workload this is two pieces, which measured best there; kernels
  // reading or writing page-locked host memory directly over the CPU-GPU link
  // measured slower than the copies). A batch-fastest piece must be whole
  // k-points (a band range of one k-point is not contiguous there): split at
  // the k-point start nearest the middle, or not at all.
  std::vector<int> bounds;
  if (p->layout == 1) {
    int best = 0, b = 0;
    for (int k = 0; k + 1 < p->nk; ++k) {
      b += p->bands[k];
      if (b > 0 && b < p->total_bands &&
          (best == 0 || std::abs(2 * b - p->total_bands) < std::abs(2 * best - p->total_bands)))
        best = b;
    }
    bounds = best > 0 ? std::vector<int>{0, best, p->total_bands} : std::vector<int>{0, p->total_bands};
  } else {
    // the first and the last piece (whose copy in and copy out are the exposed
    // ones) about 2048 planes where the batch is large enough, the pieces
    // between them about 8192
    const int edge = (2048 + p->n[2] - 1) / p->n[2];
    const int nb = p->total_bands;
    const bool edges = nb >= 4 * edge && (int64_t)nb * p->n[2] >= 4 * 8192;
    const int b0 = edges ? edge : 0, b1 = edges ? nb - edge : nb;
    const int64_t planes = (int64_t)(b1 - b0) * p->n[2];
    int np = (int)std::max<int64_t>(edges ? 1 : 2, std::min<int64_t>(16, planes / 8192));
    np = std::max(1, std::min(np, b1 - b0));
    if (edges) bounds.push_back(0);
    for (int i = 0; i <= np; ++i) bounds.push_back(b0 + (int)((int64_t)(b1 - b0) * i / np));
    if (edges) bounds.push_back(nb);
  }
  const int pieces = (int)bounds.size() - 1;
  if (!p->hs[0]) {
    for (int i = 0; i < 3; ++i)
      if (cudaStreamCreateWithFlags(&p->hs[i], cudaStreamNonBlocking) != cudaSuccess)
        return fail(FFTB_ERR_CUDA, "stream creation failed");
  }
  while ((int)p->hev.size() < 2 * pieces + 2) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(FFTB_ERR_CUDA, "event creation failed");
    p->hev.push_back(e);
  }
  const int64_t vol = (int64_t)p->n[0] * p->n[1] * p->n[2];
  auto bytes_of = [&](bool cube, int b) -> size_t {  // byte offset of band b in a batch
    return (size_t)(cube ? (int64_t)b * vol : p->band_sph[b]) * p->csize;
  };
  cudaEvent_t ev_begin = p->hev[2 * pieces], ev_end = p->hev[2 * pieces + 1];
  cudaError_t e = cudaEventRecord(ev_begin, s);
  for (int i = 0; e == cudaSuccess && i < 3; ++i) e = cudaStreamWaitEvent(p->hs[i], ev_begin, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  const unsigned char* hin = static_cast<const unsigned char*>(in_host);
  unsigned char* hout = static_cast<unsigned char*>(out_host);
  unsigned char* din = static_cast<unsigned char*>(p->d_stage_in);
  unsigned char* dout = static_cast<unsigned char*>(p->d_stage_out);
  for (int i = 0; i < pieces; ++i) {
    const int b0 = bounds[i], b1 = bounds[i + 1];
    if (b1 <= b0) continue;
    const size_t i0 = bytes_of(in_cube, b0), i1 = bytes_of(in_cube, b1);
    const size_t o0 = bytes_of(out_cube, b0), o1 = bytes_of(out_cube, b1);
    e = cudaMemcpyAsync(din + i0, hin + i0, i1 - i0, cudaMemcpyHostToDevice, p->hs[0]);
    if (e == cudaSuccess) e = cudaEventRecord(p->hev[2 * i], p->hs[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hs[1], p->hev[2 * i], 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy in");
    st = enqueue(p, b1 - b0, din, dout, p->dir == FFTB_ROUNDTRIP ? cube_dev : nullptr, p->hs[1], b0);
    if (st != FFTB_OK) return st;
    e = cudaEventRecord(p->hev[2 * i + 1], p->hs[1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->hs[2], p->hev[2 * i + 1], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + o0, dout + o0, o1 - o0, cudaMemcpyDeviceToHost, p->hs[2]);
    if (e != cudaSuccess) return cuda_fail(e, "copy out");
  }
  e = cudaEventRecord(ev_end, p->hs[2]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_end, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
  if (const int32_t st = *reinterpret_cast<volatile int32_t*>(p->h_status)) {
    *p->h_status = 0;
    return device_status_error(st, "the result is invalid");
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_check(fftb_plan p) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device synchronise");
  if (const int32_t st = *reinterpret_cast<volatile int32_t*>(p->h_status)) {
    *p->h_status = 0;
    return device_status_error(st, "results since the previous check are invalid");
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_prefetch(fftb_plan p, int32_t level) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->generic) return fail(FFTB_ERR_UNSUPPORTED, "a plan on the generic-extent path has no kernel variants");
  if (level < 0 || level > 2) return fail(FFTB_ERR_INVALID_ARG, "prefetch level must be 0, 1 or 2");
  for (int i = 0; i < 3; ++i) {
    const bool was = pf_active(p, i);
    const int old = p->pf_level;
    p->pf_level = level;
    const bool now = pf_active(p, i);
    p->pf_level = old;
    if (was != now) p->plane_ctas[i] = p->sms * (now ? p->pf_occ[i] : p->plane_occ[i]);
  }
  if (p->pf_level != level && p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // recorded with the other kernels
    p->gexec = nullptr;
  }
  p->pf_level = level;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_slab_buffers(fftb_plan p, int32_t nbuf) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->generic) return fail(FFTB_ERR_UNSUPPORTED, "a plan on the generic-extent path has no kernel variants");
  if (nbuf != 1 && nbuf != 2) return fail(FFTB_ERR_INVALID_ARG, "slab buffers must be 1 or 2");
  if (!p->a_glob && plane_smem(p->prec_kernel, p->n[0], p->n[1], p->xmax, nbuf) > kSmemLimit)
    return fail(FFTB_ERR_UNSUPPORTED, "two slab planes do not fit in shared memory for this plan");
  if (nbuf == p->a_bufs) return FFTB_OK;
  const int old = p->a_bufs;
  p->a_bufs = nbuf;
  fftb_status st = configure_planes(p);
  if (st != FFTB_OK) {
    p->a_bufs = old;
    configure_planes(p);
    return st;
  }
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_radix_schedule(fftb_plan p, int32_t plane, int32_t stick) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->generic) return fail(FFTB_ERR_UNSUPPORTED, "a plan on the generic-extent path has no kernel variants");
  if (plane < 0 || plane > 1 || stick < 0 || stick > 1) return fail(FFTB_ERR_INVALID_ARG, "schedule must be 0 or 1");
  if (plane && !p->alt_plane_ok) return fail(FFTB_ERR_UNSUPPORTED, "no alternative radix schedule for this plane stage");
  if (stick && !p->alt_stick_ok) return fail(FFTB_ERR_UNSUPPORTED, "no alternative radix schedule for this z stage");
  const bool stick_wave_before = p->tiles == stick_wave(p);
  p->sched_plane = plane ? 7 : 0;
  p->sched_stick = stick;
  if (stick_wave_before) p->tiles = stick_wave(p);
  for (int i = 0; i < 3; ++i) p->plane_ctas[i] = plane_wave(p, i);
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_pdl(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->pdl != (enable != 0) && p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->pdl = enable != 0;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_scale(fftb_plan p, double g2r, double r2g) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (!std::isfinite(g2r) || !std::isfinite(r2g)) return fail(FFTB_ERR_INVALID_ARG, "scale factors must be finite");
  if ((g2r != p->scale_g2r || r2g != p->scale_r2g) && p->gexec) {
    cudaGraphExecDestroy(p->gexec);  // recorded with the other scalings
    p->gexec = nullptr;
  }
  p->scale_g2r = g2r;
  p->scale_r2g = r2g;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_band_groups(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->generic) return fail(FFTB_ERR_UNSUPPORTED, "a plan on the generic-extent path has no kernel variants");
  if (enable && !p->bg_size)
    return fail(FFTB_ERR_UNSUPPORTED, "no grouped plane kernels for this plan (batch-fastest FP32, N0 == N1, fitting)");
  if (enable && p->tc_on)
    return fail(FFTB_ERR_UNSUPPORTED, "the grouped plane kernels are FP32: turn the tensor cores off first");
  const int bg = enable ? p->bg_size : 0;
  if (bg == p->bg) return FFTB_OK;
  p->bg = bg;
  for (int i = 0; i < 2; ++i) p->plane_ctas[i] = plane_wave(p, i);
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_plane_clusters(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (enable && !p->cl_ok)
    return fail(FFTB_ERR_UNSUPPORTED, "no cluster plane kernels for this plan (FP32, 256-point planes, half plane fitting)");
  const int cl = enable ? 7 : 0;
  if (cl == p->cl) return FFTB_OK;
  p->cl = cl;
  for (int i = 0; i < 3; ++i) p->plane_ctas[i] = plane_wave(p, i);
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_tensor_cores(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (p->prec != FFTB_MIXED_TC) return fail(FFTB_ERR_UNSUPPORTED, "tensor-core stages exist in MIXED_TC plans only");
  return set_tc(p, enable != 0);
}

FFTB_EXPORT fftb_status fftb_plan_inject(fftb_plan p, int32_t flags) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (flags & ~FFTB_INJECT_SKIP_FIRST_PREFETCH) return fail(FFTB_ERR_INVALID_ARG, "unknown injection flag");
  if (p->inject != flags && p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  p->inject = flags;
  return FFTB_OK;
}

FFTB_EXPORT int64_t fftb_plan_launches(fftb_plan p) { return p ? p->launches : -1; }

FFTB_EXPORT fftb_status fftb_destroy(fftb_plan p) {
  release(p);
  return FFTB_OK;
}

FFTB_EXPORT const char* fftb_error_string(fftb_status s) {
  switch (s) {
    case FFTB_OK: return "success";
    case FFTB_ERR_INVALID_ARG: return "invalid argument";
    case FFTB_ERR_UNSUPPORTED: return "unsupported request";
    case FFTB_ERR_ALLOC: return "allocation failed";
    case FFTB_ERR_CUDA: return "CUDA error";
    case FFTB_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case FFTB_ERR_DEVICE_BOUNDS: return "device-side bounds check failed";
  }
  return "unknown status";
}

FFTB_EXPORT const char* fftb_last_error(void) { return g_last_error.c_str(); }

FFTB_EXPORT const char* fftb_version(void) { return "fftb-gb300 0.1 (sm_103a)"; }

FFTB_EXPORT fftb_status fftb_sphere_enumerate(const int32_t n[3], double radius, const double* kshift,
                                              int32_t* g_out, int64_t capacity, int64_t* ngw) {
  if (!n || !ngw) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < 3; ++i)
    if (n[i] < 1) return fail(FFTB_ERR_INVALID_ARG, "grid extents must be >= 1");
  const double zero[3] = {0, 0, 0};
  std::vector<int32_t> g;
  const std::string err = sphere_by_cutoff(n, radius, kshift ? kshift : zero, g);
  if (!err.empty()) return fail(FFTB_ERR_INVALID_ARG, err);
  *ngw = (int64_t)g.size() / 3;
  if (g_out && capacity > 0) {
    const int64_t m = std::min<int64_t>(capacity, *ngw);
    std::memcpy(g_out, g.data(), (size_t)m * 3 * sizeof(int32_t));
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_box_enumerate(const int32_t n[3], int32_t* g_out, int64_t capacity) {
  if (!n || !g_out) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < 3; ++i)
    if (n[i] < 1) return fail(FFTB_ERR_INVALID_ARG, "grid extents must be >= 1");
  const int64_t vol = (int64_t)n[0] * n[1] * n[2];
  if (capacity < vol) return fail(FFTB_ERR_INVALID_ARG, "g_out holds fewer than N0 N1 N2 triples");
  const int32_t h0 = n[0] / 2, h1 = n[1] / 2, h2 = n[2] / 2;
  int32_t* o = g_out;
  for (int32_t gy = -h1; gy < n[1] - h1; ++gy)
    for (int32_t gx = -h0; gx < n[0] - h0; ++gx)
      for (int32_t gz = -h2; gz < n[2] - h2; ++gz) {
        *o++ = gx;
        *o++ = gy;
        *o++ = gz;
      }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_glist_from_offsets(const int32_t n[3], const int32_t lo[3], const int32_t hi[3],
                                                const int64_t* offsets, const int32_t* z_index, int64_t nnz,
                                                int32_t* g_out) {
  if (!n || !lo || !hi || !offsets || (nnz > 0 && (!z_index || !g_out))) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  if (nnz < 0) return fail(FFTB_ERR_INVALID_ARG, "nnz must be >= 0");
  for (int i = 0; i < 3; ++i) {
    if (n[i] < 1) return fail(FFTB_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (hi[i] < lo[i]) return fail(FFTB_ERR_INVALID_ARG, "domain upper corner below its lower corner");
    if ((int64_t)hi[i] - lo[i] + 1 > n[i]) return fail(FFTB_ERR_INVALID_ARG, "domain wider than the grid (would alias)");
  }
  const int64_t nx = (int64_t)hi[0] - lo[0] + 1, ny = (int64_t)hi[1] - lo[1] + 1;
  const int64_t cols = nx * ny;
  if (offsets[0] != 0 || offsets[cols] != nnz) return fail(FFTB_ERR_INVALID_ARG, "offsets must run from 0 to nnz");
  // a domain coordinate v is the frequency v mod N, as a signed component
  auto freq = [](int64_t v, int32_t N) {
    int64_t m = v % N;
    if (m < 0) m += N;
    return (int32_t)(m >= N - N / 2 ? m - N : m);
  };
  for (int64_t c = 0; c < cols; ++c) {
    if (offsets[c + 1] < offsets[c]) return fail(FFTB_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const int32_t gx = freq(lo[0] + c % nx, n[0]), gy = freq(lo[1] + c / nx, n[1]);
    for (int64_t e = offsets[c]; e < offsets[c + 1]; ++e) {
      const int32_t z = z_index[e];
      if (z < lo[2] || z > hi[2]) return fail(FFTB_ERR_INVALID_ARG, "z index outside the domain");
      g_out[3 * e] = gx;
      g_out[3 * e + 1] = gy;
      g_out[3 * e + 2] = freq(z, n[2]);
    }
  }
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_sphere_sticks(const int32_t n[3], const int32_t* g, int64_t ngw,
                                           int32_t* n_sticks, int32_t* n_slabs) {
  if (!n || (!g && ngw > 0) || !n_sticks || !n_slabs) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < 3; ++i)
    if (n[i] < 1) return fail(FFTB_ERR_INVALID_ARG, "grid extents must be >= 1");
  KGeom geo;
  const std::string err = build_geometry(n, g, ngw, geo);
  if (!err.empty()) return fail(FFTB_ERR_INVALID_ARG, err);
  *n_sticks = geo.S;
  *n_slabs = geo.X;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_timing(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  p->timing = enable != 0;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_stage_times(fftb_plan p, double* ms, int64_t* launches) {
  if (!p || !ms || !launches) return fail(FFTB_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < FFTB_STAGE_KINDS; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (const auto& r : p->recs) {
    cudaError_t e = cudaEventSynchronize(p->ev_pool[r.b]);
    if (e != cudaSuccess) return cuda_fail(e, "event synchronise");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, p->ev_pool[r.a], p->ev_pool[r.b]);
    if (e != cudaSuccess) return cuda_fail(e, "event elapsed time");
    ms[r.kind] += t;
    launches[r.kind] += 1;
  }
  p->recs.clear();
  p->ev_used = 0;
  return FFTB_OK;
}

FFTB_EXPORT fftb_status fftb_plan_set_graph(fftb_plan p, int32_t enable) {
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  p->use_graph = enable != 0;
  return FFTB_OK;
}

namespace {

std::string tune_key(const fftb_plan_s* p) {
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, p->device);
  std::ostringstream k;
  k << p->n[0] << "x" << p->n[1] << "x" << p->n[2] << "|S" << p->smax << "|X" << p->xmax << "|B" << p->total_bands
    << "|K" << p->nk << "|d" << (int)p->dir << "|p" << (int)p->prec << "|L" << p->layout << "|" << prop.name;
  std::string out = k.str();
  for (char& c : out)
    if (c == ' ') c = '_';
  return out;
}

// One autotuner candidate: everything it may change on a plan.
struct TuneChoice {
  int chunk = 1, tiles = 0, level = 1, a_bufs = 2;
  int ctas[3] = {0, 0, 0};  // -1: one full wave of the kernel in use
  int sched_plane = 0, sched_stick = 0;  // radix schedule variants
  int pdl = 1;                           // programmatic dependent launch
  int bg = 0;                            // band group of the plane stages (batch-fastest)
  int tc = 0;                            // MIXED_TC: tensor-core kernels in use
  int cl = 0;                            // plane stages on two-CTA clusters
};

TuneChoice current_choice(const fftb_plan_s* p) {
  TuneChoice c;
  c.chunk = p->chunk;
  c.tiles = p->tiles;
  c.level = p->pf_level;
  c.a_bufs = p->a_bufs;
  c.sched_plane = p->sched_plane;
  c.sched_stick = p->sched_stick;
  c.pdl = p->pdl ? 1 : 0;
  c.bg = p->bg;
  c.tc = p->tc_on ? 1 : 0;
  c.cl = p->cl;
  for (int i = 0; i < 3; ++i) c.ctas[i] = p->plane_ctas[i];
  return c;
}

bool tune_cache_lookup(const std::string& key, TuneChoice* out) {
  const char* path = std::getenv("FFTB_TUNE_CACHE");
  if (!path || !*path) return false;
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    std::string k;
    TuneChoice c;
    if ((ls >> k >> c.chunk >> c.ctas[0] >> c.ctas[1] >> c.ctas[2] >> c.tiles >> c.level >> c.a_bufs >>
         c.sched_plane >> c.sched_stick >> c.pdl >> c.bg >> c.tc >> c.cl) &&
        k == key && c.chunk >= 1 && c.level >= 0 && c.level <= 2 && (c.a_bufs == 1 || c.a_bufs == 2) &&
        c.sched_plane >= 0 && c.sched_plane <= 7 && (c.sched_stick == 0 || c.sched_stick == 1) &&
        (c.pdl == 0 || c.pdl == 1) && c.bg >= 0 && c.bg <= 4 && (c.tc == 0 || c.tc == 1) &&
        c.cl >= 0 && c.cl <= 7) {
      *out = c;
      found = true;  // the last entry wins
    }
  }
  return found;
}

void tune_cache_store(const std::string& key, const TuneChoice& c) {
  const char* path = std::getenv("FFTB_TUNE_CACHE");
  if (!path || !*path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << c.chunk << " " << c.ctas[0] << " " << c.ctas[1] << " " << c.ctas[2] << " " << c.tiles << " "
    << c.level << " " << c.a_bufs << " " << c.sched_plane << " " << c.sched_stick << " " << c.pdl << " " << c.bg
    << " " << c.tc << " " << c.cl << "\n";
}

fftb_status resize_T(fftb_plan_s* p, int chunk) {
  const size_t need = (size_t)chunk * p->n[2] * p->tpitch * p->csize;
  if (need <= p->T_bytes) return FFTB_OK;
  if (p->d_T) cudaFree(p->d_T);
  p->d_T = nullptr;
  p->T_bytes = 0;
  if (cudaMalloc(&p->d_T, need) != cudaSuccess) return fail(FFTB_ERR_ALLOC, "cudaMalloc stick scratch failed");
  p->T_bytes = need;
  return FFTB_OK;
}

// Puts a candidate on the plan (slab buffers first: they change the
// resident CTAs per SM).
fftb_status apply_choice(fftb_plan_s* p, const TuneChoice& c) {
  if (p->tc_avail && (c.tc != 0) != p->tc_on) {
    fftb_status st = set_tc(p, c.tc != 0);
    if (st != FFTB_OK) {
      set_tc(p, !(c.tc != 0));
      return st;
    }
  }
  if (c.a_bufs != p->a_bufs) {
    const int old = p->a_bufs;
    p->a_bufs = c.a_bufs;
    fftb_status st = configure_planes(p);
    if (st != FFTB_OK) {
      p->a_bufs = old;
      configure_planes(p);
      return st;
    }
  }
  fftb_status st = resize_T(p, std::max(c.chunk, p->bg_size));
  if (st != FFTB_OK) return st;
  p->chunk = c.chunk;
  p->bg = (c.bg && p->bg_size && !p->tc_on) ? p->bg_size : 0;
  p->cl = p->cl_ok ? c.cl : 0;
  p->pf_level = c.level;
  p->sched_plane = p->alt_plane_ok ? c.sched_plane : 0;
  p->sched_stick = (c.sched_stick && p->alt_stick_ok) ? 1 : 0;
  p->pdl = c.pdl != 0;
  p->tiles = c.tiles < 0 ? stick_wave(p) : c.tiles;
  for (int i = 0; i < 3; ++i) p->plane_ctas[i] = c.ctas[i] >= 0 ? c.ctas[i] : plane_wave(p, i);
  return FFTB_OK;
}

}  // namespace

FFTB_EXPORT fftb_status fftb_plan_autotune(fftb_plan p, int32_t trials) {
  NvtxRange range("fftb_plan_autotune");
  if (!p) return fail(FFTB_ERR_INVALID_ARG, "NULL plan");
  if (trials < 1) return fail(FFTB_ERR_INVALID_ARG, "trials must be >= 1");
  if (p->total_bands == 0 || p->generic) return FFTB_OK;  // the generic-extent path has one kernel per stage
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device) return fail(FFTB_ERR_INVALID_ARG, "current device differs from the plan's device");
  const std::string key = tune_key(p);
  TuneChoice cached;
  if (tune_cache_lookup(key, &cached)) {
    fftb_status st = apply_choice(p, cached);
    if (st != FFTB_OK) return st;
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    return FFTB_OK;
  }
  // trial buffers: the whole batch, or the longest band prefix within 4 GiB
  const int64_t vol = (int64_t)p->n[0] * p->n[1] * p->n[2];
  int64_t max_ngw = 0;
  for (const auto& G : p->geo) max_ngw = std::max(max_ngw, G.ngw);
  const bool cube_io = p->dir == FFTB_G_TO_R || p->dir == FFTB_R_TO_G || p->dir == FFTB_ROUNDTRIP;
  const size_t band_bytes = (size_t)p->csize * (2 * max_ngw + (cube_io ? vol : 0));
  const size_t budget = (size_t)4 << 30;
  const int bands = (int)std::max<int64_t>(1, std::min<int64_t>(p->total_bands, (int64_t)(budget / std::max<size_t>(band_bytes, 1))));
  const size_t sph_b = (size_t)p->sphere_elems * p->csize;
  // a batch-fastest band spreads over its whole k-point block of the cube:
  // cover the blocks of every k-point the band prefix touches
  int cube_bands = bands;
  if (p->layout == 1) {
    cube_bands = 0;
    for (int k = 0; k < p->nk && cube_bands < bands; ++k) cube_bands += p->bands[k];
  }
  const size_t cube_b = (size_t)cube_bands * vol * p->csize;
  void *d_in = nullptr, *d_out = nullptr, *d_cube = nullptr, *d_v = nullptr;
  auto cleanup = [&]() {
    if (d_in) cudaFree(d_in);
    if (d_out) cudaFree(d_out);
    if (d_cube) cudaFree(d_cube);
    if (d_v) cudaFree(d_v);
  };
  // a band prefix may still index the whole sphere batch: size for the real offsets
  const size_t in_full = p->dir == FFTB_R_TO_G ? cube_b : sph_b;
  const size_t out_full = p->dir == FFTB_G_TO_R ? cube_b : sph_b;
  if (cudaMalloc(&d_in, in_full) != cudaSuccess || cudaMalloc(&d_out, out_full) != cudaSuccess ||
      (p->dir == FFTB_ROUNDTRIP && cudaMalloc(&d_cube, cube_b) != cudaSuccess)) {
    cleanup();
    return fail(FFTB_ERR_ALLOC, "autotune buffers");
  }
  cudaMemset(d_in, 0, in_full);
  const void* saved_v = p->d_V;
  if (p->dir == FFTB_APPLY_LOCAL && !p->d_V) {
    if (cudaMalloc(&d_v, (size_t)vol * p->csize / 2) != cudaSuccess) {
      cleanup();
      return fail(FFTB_ERR_ALLOC, "autotune potential");
    }
    cudaMemset(d_v, 0, (size_t)vol * p->csize / 2);
    p->d_V = d_v;
  }
  // chunk candidates
  std::vector<int> chunks;
  const size_t t_band = (size_t)p->n[2] * p->tpitch * p->csize;
  for (int c : {bands, (bands + 1) / 2, (bands + 3) / 4, (int)((24u << 20) / t_band), (int)((48u << 20) / t_band),
                (int)((96u << 20) / t_band)}) {
    c = std::max(1, std::min(c, bands));
    if (std::find(chunks.begin(), chunks.end(), c) == chunks.end()) chunks.push_back(c);
  }
  const int max_chunk = *std::max_element(chunks.begin(), chunks.end());
  fftb_status st = resize_T(p, std::max(max_chunk, p->bg_size));
  if (st != FFTB_OK) {
    p->d_V = saved_v;
    cleanup();
    return st;
  }
  const TuneChoice saved = current_choice(p);
  const bool saved_timing = p->timing, saved_graph = p->use_graph;
  const int64_t saved_launches = p->launches;
  p->timing = false;
  p->use_graph = false;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  TuneChoice best_c = saved;
  // times one candidate; keeps it if it is the fastest so far
  auto trial = [&](const TuneChoice& c) -> fftb_status {
    fftb_status s2 = apply_choice(p, c);
    if (s2 != FFTB_OK) return s2;
    s2 = enqueue(p, bands, d_in, d_out, d_cube, nullptr);  // warm-up
    if (s2 != FFTB_OK) return s2;
    cudaEventRecord(e0, nullptr);
    for (int t = 0; t < trials && s2 == FFTB_OK; ++t) s2 = enqueue(p, bands, d_in, d_out, d_cube, nullptr);
    cudaEventRecord(e1, nullptr);
    cudaError_t ce = cudaEventSynchronize(e1);
    if (s2 != FFTB_OK) return s2;
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune run");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_c = current_choice(p);
    }
    return FFTB_OK;
  };
  // stage 1: kernel variant (slab-plane buffers, prefetch level), each with a
  // full wave of persistent plane CTAs, at the plan's chunk and at the
  // largest chunk (a variant with fewer resident CTAs can need long launches)
  // (MIXED_TC: first with the tensor-core kernels, then with the FP32 ones)
  std::vector<int> tcs = {saved.tc};
  if (p->tc_avail) tcs.push_back(1 - saved.tc);
  std::vector<int> bgs = {0};
  if (p->bg_size) bgs.push_back(p->bg_size);
  std::vector<int> chunks1 = {saved.chunk};
  if (max_chunk != saved.chunk) chunks1.push_back(max_chunk);
  for (int tcv : tcs) {
  if (st != FFTB_OK) break;
  if (p->tc_avail) {
    TuneChoice c = saved;
    c.tc = tcv;
    c.sched_plane = c.sched_stick = 0;
    c.tiles = c.tiles ? -1 : 0;
    c.ctas[0] = c.ctas[1] = c.ctas[2] = -1;
    st = apply_choice(p, c);
    if (st != FFTB_OK) break;
  }
  std::vector<int> nbufs = {saved.a_bufs};
  {
    const int other = 3 - saved.a_bufs;
    if (p->a_glob || plane_smem(p->prec_kernel, p->n[0], p->n[1], p->xmax, other) <= kSmemLimit)
      nbufs.push_back(other);
  }
  std::vector<int> stick_scheds = {0};
  if (p->alt_stick_ok) stick_scheds.push_back(1);
  for (int ck : chunks1)
  for (int bgv : bgs)
  for (int nb : nbufs) {
    if (st != FFTB_OK) break;
    for (int ss : stick_scheds) {
      std::vector<int> masks;  // kernel choices already timed for this slab-buffer count
      // plane schedule per stage the direction uses (bits: G->r 1, r->G 2, apply 4)
      const int used = p->dir == FFTB_G_TO_R ? 1 : p->dir == FFTB_R_TO_G ? 2 : p->dir == FFTB_APPLY_LOCAL ? 4 : 3;
      std::vector<int> sps;
      for (int m = 0; m <= 7; ++m)
        if ((m & ~used) == 0 && (m == 0 || p->alt_plane_ok)) sps.push_back(m);
      for (int sp : sps) {
        for (int lv : {saved.level, 0, 1, 2})
        for (int clv = 0; clv <= 7; ++clv) {
          if ((clv & ~used) || (clv && !p->cl_ok)) continue;  // per stage the direction uses
          TuneChoice c = saved;
          c.tc = tcv;
          c.cl = clv;
          c.a_bufs = nb;
          c.level = lv;
          c.sched_plane = sp;
          c.sched_stick = ss;
          c.bg = bgv;
          c.chunk = ck;
          c.tiles = c.tiles ? -1 : 0;              // z-stage: the same kind, one full wave of its schedule
          c.ctas[0] = c.ctas[1] = c.ctas[2] = -1;  // one full wave of the variant
          st = apply_choice(p, c);
          if (st != FFTB_OK) break;
          // what the kernels in use depend on (the grouped G->r / r->G kernels on neither)
          int mask = (p->bg ? 64 | (p->sched_plane & 4) : p->sched_plane) << 3;
          for (int i = 0; i < 3; ++i)
            if (pf_active(p, i)) mask |= 1 << i;
          if (p->cl) {  // the stages on the cluster kernels have no other variants
            for (int i = 0; i < 3; ++i)
              if ((p->cl >> i) & 1) mask &= ~((1 << i) | (8 << i));
            mask |= p->cl << 10;
          }
          if (std::find(masks.begin(), masks.end(), mask) != masks.end()) continue;
          masks.push_back(mask);
          st = trial(current_choice(p));
          if (st != FFTB_OK) break;
        }
        if (st != FFTB_OK) break;
      }
      if (st != FFTB_OK) break;
    }
  }
  }  // tcv
  // stage 2: chunk, persistent plane CTAs per SM (0: one CTA per plane) and
  // z-stage CTAs for the chosen variant
  const TuneChoice variant = best_c;
  if (st == FFTB_OK) st = apply_choice(p, variant);
  const int mi = p->dir == FFTB_R_TO_G ? 1 : p->dir == FFTB_APPLY_LOCAL ? 2 : 0;
  std::vector<int> mults;
  for (int m : {occ_in_use(p, mi), occ_in_use(p, mi) - 1, 0})
    if ((m > 0 || (m == 0 && !p->a_glob)) && std::find(mults.begin(), mults.end(), m) == mults.end())
      mults.push_back(m);
  for (size_t k = 0; st == FFTB_OK && k < chunks.size() * mults.size() * 2; ++k) {
    TuneChoice c = variant;
    c.chunk = chunks[k / (2 * mults.size())];
    const int m = mults[(k / 2) % mults.size()];
    c.tiles = (k & 1) ? stick_wave(p) : 0;
    for (int i = 0; i < 3; ++i)
      c.ctas[i] = m == 0 ? 0 : ((p->cl >> i) & 1) ? plane_wave(p, i) : p->sms * std::min(m, occ_in_use(p, i));
    st = trial(c);
  }
  // stage 3: the best schedule with and without programmatic dependent launch
  // (early launch helps short stages; on long ones the waiting CTAs can cost
  // more than the hidden launch latency)
  if (st == FFTB_OK) {
    TuneChoice c = best_c;
    c.pdl = 1 - c.pdl;
    st = trial(c);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->timing = saved_timing;
  p->use_graph = saved_graph;
  p->launches = saved_launches;
  p->d_V = saved_v;
  cleanup();
  if (st != FFTB_OK) {
    apply_choice(p, saved);
    return st;
  }
  // a chunk tuned on a band prefix covers the whole batch too
  st = apply_choice(p, best_c);
  if (st != FFTB_OK) return st;
  if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
  tune_cache_store(key, best_c);
  debug_report(p, "autotuned");
  return FFTB_OK;
}
