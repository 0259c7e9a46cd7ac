// fftb_internal.h -- host-side types shared by the plan code and the kernel
// launchers. No CUDA templates here; the .cu files own the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace fftb {

// Runtime line schedule of one axis (generic-extent path): length and radices.
constexpr int GEN_MAXP = 12;
struct GenAxis {
  int32_t n, np;
  int32_t r[GEN_MAXP];
};
// Parameters of a generic-extent stage launch: the three axes, the slab
// buffer S [chunk bands][N2][xmax][N1], and the line group held per CTA.
struct GenParams {
  GenAxis ax[3];  // x, y, z
  void* S;
  int64_t lim_S;  // S elements (bounds checks of a checked build)
  int32_t lpc;    // lines per CTA group
  int32_t pitch;  // shared-memory line pitch (elements)
};

// Per-k-point geometry as the kernels see it.
struct KInfo {
  int32_t S;           // occupied (x,y) sticks
  int32_t X;           // occupied x values (y-z slabs)
  int32_t stick_base;  // sticks of earlier k-points; stick_ent uses stick_base + k
  int32_t xmap_base;   // first entry of this k in xmap (k * N0)
  int32_t col_base;    // first entry of this k in col_info (sum of X over earlier k)
  int32_t flags;       // KF_* bits
  int32_t bstride;     // elements between consecutive sphere entries and between
                       //   consecutive cube points of one band: 1 band-major, B_k
                       //   batch-fastest (the band index is then the fastest)
};
// Every slab column's sticks have consecutive gy (always true for a cutoff
// sphere); the plane stage then indexes stick rows directly.
constexpr int32_t KF_CONTIGUOUS_COLUMNS = 1;
// Every stick's entries have consecutive gz and consecutive positions in the
// sphere list (the canonical order of a cutoff sphere); the z stage then
// indexes the coefficient list directly.
constexpr int32_t KF_CANONICAL_STICKS = 2;
// Every occupied stick (x, y) satisfies |x| <= N0/4 and |y| <= N1/4 (signed),
// as for the cutoff spheres of the paper's shape rule, cube width = twice the
// sphere diameter: the y and x lines' inputs (G -> r) and needed outputs
// (r -> G) then avoid the middle half of the line, and the kernels may drop
// those elements at compile time.
constexpr int32_t KF_XY_QUARTER = 4;
// Every sphere entry satisfies |z| <= N2/4 (signed): the z lines' inputs and
// needed outputs avoid the middle half of the line in the same way.
constexpr int32_t KF_Z_QUARTER = 8;

// Per band: its k-point's geometry and the offsets (complex elements) of
// its first sphere entry and first cube point, read in one 48-byte load.
struct __align__(16) BandInfo {
  KInfo ki;
  int64_t sph;
  int64_t cube;
};

// Device tables for all k-points (concatenated) plus twiddles.
struct Geo {
  const BandInfo* band;      // [total_bands]
  const int4* stick_info;    // [sum S_k] per stick: first entry, end entry (global),
                             //   list position of the first entry, signed gz of it
  const int32_t* ent_pos;    // [sum ngw] position of the entry within its k's sphere list
  const int32_t* ent_zs;     // [sum ngw] (z index << 24) | local stick index
  const int16_t* xmap;       // [n_k * N0] slab index of x, or -1
  const int4* col_info;      // [sum X_k] per slab: first stick (local), sticks, signed gy of
                             //   the first stick, 0
  const int32_t* stick_xy;   // [sum S_k] (xi << 16) | y index
  const void* tw0;           // [N0] e^{+2 pi j m / N0} in the plan's real type
  const void* tw1;           // [N1]
  const void* tw2;           // [N2]
  int32_t n0, n1, n2;
  int32_t smax;              // T pitch: max sticks over k, rounded up to even (rows start
                             //   on 16-byte boundaries for bulk copies)
  int32_t xmax;              // max slabs over k
};

// One launch over the bands [band0, band0 + nb).
struct Launch {
  Geo g;
  int32_t band0, nb;
  const void* sph_in;   // sphere batch read by the z-stage (G -> r)
  void* sph_out;        // sphere batch written by the z-stage (r -> G)
  const void* cube_in;  // cube batch read by the plane stage (r -> G)
  void* cube_out;       // cube batch written by the plane stage (G -> r)
  void* T;              // stick scratch [nb][N2][smax]
  const void* V;        // potential (apply)
  int32_t plane_ctas;   // persistent plane-stage CTAs (0: one per plane)
  int32_t a_bufs;       // slab-plane buffers of the plane stage (1 or 2)
  void* a_glob;         // slab planes in global memory (per CTA), or NULL: shared memory
  int32_t a_blocks;     // per-CTA slab-plane blocks a_glob holds (a launch uses at most that many CTAs)
  int32_t pf;           // plane stage: prefetch its inputs with bulk async copies
  int32_t inject;       // INJECT_* bits (tests of the bounded waits)
  int32_t* status;      // device-visible status word (STATUS_* bits), set on a failed wait
  int32_t pdl;          // launch with programmatic dependent launch (overlaps launch and prologue)
  int32_t xq;           // every k-point of the plan has KF_XY_QUARTER (plane kernel variant choice)
  int32_t zq;           // every k-point of the plan has KF_Z_QUARTER (z-stage kernel variant choice)
  const int2* groups;   // batch-fastest band groups (first band, bands), plan-global list
  int32_t grp0, ngrp;   // the groups of this launch (they cover [band0, band0 + nb))
  // buffer extents in complex elements from the base pointers above, read by
  // the bounds checks of a checked build (FFTB_CHECK) only
  int64_t lim_sph, lim_cube, lim_T, lim_V;
  cudaStream_t stream;
};

enum Prec { P_F64 = 0, P_F32 = 1, P_TC = 2 };
// Launch::inject: the first prefetch of CTA 0 (warp 0) is not issued, so its
// bounded wait runs out and the kernel reports STATUS_WAIT_TIMEOUT.
constexpr int32_t INJECT_SKIP_FIRST_PREFETCH = 1;
enum Mode { M_G2R = 1, M_R2G = -1, M_APPLY = 2 };

bool grid_size_supported(int n);
bool plane_size_supported(int n0, int n1);
// Dynamic shared memory (bytes) of each kernel for one k geometry.
size_t stick_smem(int prec, int n2);
// a_glob: the slab planes live in global memory (only the warp scratch and
// twiddles are in shared memory)
size_t plane_smem(int prec, int n0, int n1, int xmax, int a_bufs, bool a_glob = false);
int stick_tile(int prec, int n2);
// Resident z-stage CTAs per SM (after prepare_kernels).
int stick_occupancy(int prec, int n2);
// Raise the dynamic shared-memory limit of the kernels a plan uses.
cudaError_t prepare_kernels(int prec, int n0, int n1, int n2, int xmax, int a_bufs, bool a_glob = false);
// Resident plane-stage CTAs per SM for this geometry (after prepare_kernels).
int plane_occupancy(int prec, int mode, int n0, int n1, int xmax, int a_bufs, bool a_glob = false);
// ctas: persistent z-stage CTAs (0: one warp per task)
cudaError_t launch_stick(int prec, int mode, const Launch& L, int ctas);
cudaError_t launch_plane(int prec, int mode, const Launch& L);
// FP32 plane kernels with bulk-copy prefetch of their inputs (mode M_*; tp =
// the stick-row pitch Geo::smax). Unsupported combinations return false, 0
// or cudaErrorInvalidValue.
// ag: the variant with slab planes in global memory (grids 128-256).
bool plane_pf_supported(int mode, int n0, int n1, bool ag = false);
size_t plane_pf_smem(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag = false);
cudaError_t prepare_plane_pf(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag = false);
int plane_pf_occupancy(int mode, int n0, int n1, int xmax, int a_bufs, int tp, bool ag = false);
cudaError_t launch_plane_pf(int mode, const Launch& L);
// FP32 kernels with the alternative radix schedule of a length (k_f32_alt.cu;
// lengths 64, 96, 128, 160): whether n has one, shared memory, kernel
// attributes, resident CTAs per SM, launches.
bool alt_schedule(int n);
size_t plane_alt_smem(int n, int xmax, int a_bufs);
cudaError_t prepare_alt(int n0, int n2, int xmax, int a_bufs);
int plane_alt_occupancy(int mode, int n, int xmax, int a_bufs);
int stick_alt_occupancy(int n);
cudaError_t launch_plane_alt(int mode, const Launch& L);
// FP32 y/x stages of batch-fastest plans over groups of bands of one k-point
// (k_f32_bg.cu; N0 == N1): the group size of a length (0: none), shared
// memory (0 if bg is not that size), kernel attributes, resident CTAs per SM
// (G -> r or r -> G), launch over L.groups[grp0 .. grp0 + ngrp).
int plane_bg_group(int n);
size_t plane_bg_smem(int n0, int n1, int xmax, int bg);
cudaError_t prepare_plane_bg(int n, int xmax);
int plane_bg_occupancy(int mode, int n, int xmax);
cudaError_t launch_plane_bg(int mode, const Launch& L);
// FP32 y/x stages with the slab plane split over a cluster of two CTAs
// (k_cluster.cu; N0 == N1 = 256): shared memory per CTA of one mode, or the
// largest over the modes (mode 0; 0: no such kernel), kernel attributes,
// clusters resident at once, launch (L.plane_ctas CTAs, two per cluster; 0:
// one cluster per plane).
size_t plane_cluster_smem(int n0, int n1, int xmax, int mode = 0);
cudaError_t prepare_plane_cluster(int n, int xmax);
int plane_cluster_count(int mode, int n, int xmax);
int plane_cluster_size();
cudaError_t launch_plane_cluster(int mode, const Launch& L);
// Multiplies n complex elements (csize bytes each) at data by s on L.stream
// (k_scale.cu): the optional output normalisation.
cudaError_t launch_scale(int csize, void* data, int64_t n, double s, const Launch& L, int sms);
cudaError_t launch_stick_alt(int mode, const Launch& L, int ctas);
// FP32 z-stage kernels that drop the middle half of each z line (k_f32_zq.cu;
// default schedule; launches whose k-points all have KF_Z_QUARTER)
cudaError_t prepare_stick_zq(int n2);
int stick_zq_occupancy(int n2);  // resident CTAs per SM (after prepare_stick_zq)
cudaError_t launch_stick_zq(int mode, const Launch& L, int ctas);
// MIXED_TC plane stage on the 5th-generation tensor cores (k_tc5.cu): the
// union over k-points of the occupied x values [xlo, xlo + xu) and of the
// stick y values [ylo, ylo + yu) (signed grid indices), and the device image
// of the direction's DFT matrices (tc5_build_weights).
struct Tc5Geo {
  int32_t xlo, xu, ylo, yu;
  const void* w;
};
bool tc5_supported(int n0, int n1);
// generic-extent path: stage 0 z, 1 y, 2 x, 3 fused x apply; sign +1 G -> r, -1 r -> G
cudaError_t launch_generic(bool fp64, int stage, int sign, const Launch& L, const GenParams& P, int ctas);
// the default line schedule of length n has a tensor-core (radix-8) pass
bool tc_pass_in_schedule(int n);
size_t tc5_weight_bytes(int mode, int n, const Tc5Geo& P);
// writes the split-FP16 DFT matrices of `mode` into img (device), from the
// plan's twiddle table tw (device, float2 e^{+2 pi i m / n}); asynchronous
cudaError_t tc5_build_weights(int mode, int n, const Tc5Geo& P, const void* tw, void* img);
size_t tc5_smem(int mode, int n, const Tc5Geo& P, int smax);
// raises the shared-memory limit and reports resident CTAs per SM
cudaError_t tc5_prepare(int mode, int n, const Tc5Geo& P, int smax, int* occupancy);
// ctas: persistent CTAs (0: enough for every plane)
cudaError_t tc5_launch(int mode, const Launch& L, const Tc5Geo& P, int ctas);
// Sets the calling thread's message for fftb_last_error().
void set_last_error(const std::string& msg);

}  // namespace fftb
