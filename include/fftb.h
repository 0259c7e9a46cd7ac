/*
 * fftb.h -- batched, pruned plane-wave 3D FFT between a cutoff sphere of
 * coefficients and the full real-space cube, on one GPU (sm_103a).
 *
 * The operation (Sec. 2.2 of Popovici, Del Ben, Marques, Canning, "Flexible
 * Multi-Dimensional FFTs for Plane Wave Density Functional Theory Codes"):
 *
 *   G -> r   R_b[x,y,z] = sum_{G in sphere} c_b(G) exp(+2 pi j (gx x/N0 + gy y/N1 + gz z/N2))
 *   r -> G   c_b(G)     = sum_{x,y,z} R_b[x,y,z] exp(-2 pi j (gx x/N0 + gy y/N1 + gz z/N2))
 *
 * Neither direction is scaled, so r->G after G->r multiplies by N0*N1*N2.
 * The sign of G->r follows the plane-wave expansion psi(r) = sum_g c(g)
 * e^{j g r} (Sec. 2.2); the sign of r->G follows omega_n = e^{-j 2 pi/n}
 * (Sec. 2.1). The sphere is the set of integer G with |G + k| <= r in grid
 * units (the cutoff rule 1/2 |g|^2 <= E_cut, Sec. 2.2), components in
 * [-N/2, N/2). G sits at cube index (gx mod N0, gy mod N1, gz mod N2).
 *
 * The padding is staged as in Fig. 3: z-FFTs run only on occupied (x,y)
 * sticks, y-FFTs only on occupied x-slabs, and x-FFTs on full lines; the
 * reverse direction prunes its outputs the same way.
 *
 * Data layout (all complex data interleaved re,im; float for FP32 and
 * MIXED_TC plans, double for FP64 plans), fftb_desc.layout = 0 (band-major):
 *   sphere batch : concatenation over k-points of [B_k][ngw_k]
 *   cube batch   : concatenation over k-points of [B_k][N2][N1][N0] (x fastest,
 *                  Sec. 2.1: n0 is the fastest dimension in memory)
 *   potential V  : real, [N2][N1][N0]
 * fftb_desc.layout = 1 (batch-fastest: the batch dimension declared first is
 * the fastest in memory, Sec. 3.3), per k-point:
 *   sphere batch : concatenation over k-points of [ngw_k][B_k]
 *   cube batch   : concatenation over k-points of [N2][N1][N0][B_k]
 * The arithmetic is the same in both layouts (results are bit-identical up to
 * the permutation); batch-fastest cube rows are read and written point by
 * point B_k elements apart, so its r -> G stage does not use bulk copies and
 * MIXED_TC plans run their plane stages on the mma.sync path.
 * Within one k-point the sphere order is the user's list order, or for a
 * cutoff sphere the canonical order: sorted by gy, then gx, then gz, each
 * ascending over signed values (the offset array over the xy projection of
 * Sec. 3.3 / Fig. 6, one contiguous run per (gx, gy) stick).
 *
 * Errors: every call returns a status code; no exception crosses this ABI
 * (the paper's plan builder throws on an unsupported pattern, Sec. 3.1;
 * here that is FFTB_ERR_UNSUPPORTED). fftb_last_error() gives a message.
 * Pointers named *_dev are device pointers owned by the caller; the library
 * never frees them. Host pointers are read during the call only.
 */
#ifndef FFTB_H
#define FFTB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftb_plan_s* fftb_plan;

typedef enum {
  FFTB_OK = 0,
  FFTB_ERR_INVALID_ARG = 1,    /* bad size, pointer, index or argument combination */
  FFTB_ERR_UNSUPPORTED = 2,    /* valid request this build has no kernel for       */
  FFTB_ERR_ALLOC = 3,          /* device or host allocation failed                 */
  FFTB_ERR_CUDA = 4,           /* a CUDA runtime call failed                       */
  FFTB_ERR_DEVICE_TIMEOUT = 5, /* a device-side bounded wait gave up               */
  FFTB_ERR_DEVICE_BOUNDS = 6   /* a checked build (FFTB_CHECK, libfftb_check.so)
                                  found a kernel index outside its buffer; the
                                  access was skipped                              */
} fftb_status;

typedef enum {
  FFTB_G_TO_R = 1,        /* sphere -> cube                                      */
  FFTB_R_TO_G = -1,       /* cube -> sphere                                      */
  FFTB_ROUNDTRIP = 0,     /* sphere -> cube (kept) -> sphere                     */
  FFTB_APPLY_LOCAL = 2    /* sphere -> V(r) * psi(r) -> sphere; cube never stored */
} fftb_direction;

typedef enum {
  FFTB_FP64 = 0,          /* complex128 storage and arithmetic                   */
  FFTB_FP32 = 1,          /* complex64 storage and arithmetic                    */
  FFTB_MIXED_TC = 2       /* complex64 storage; split-precision tensor-core radix stages:
                             the y/x stages of grids 16-64 (N0 == N1, band-major) as dense
                             tcgen05 products, radix-8 passes on mma.sync at the lengths
                             whose schedule has one (64, 128); a stage of any other length
                             (no tensor-core pass: 24, 96, 160, ...) runs the FP32 kernels */
} fftb_precision;

/* Plan description. Either radius (+ kshift) or g_list describes the spheres. */
typedef struct {
  int32_t n[3];            /* N0 (x), N1 (y), N2 (z) grid extents                 */
  int32_t n_kpoints;       /* number of spheres (k-points), >= 1                   */
  const int32_t* bands;    /* host, n_kpoints band counts (each >= 0); NULL = 1 each */
  double radius;           /* cutoff radius r in grid units (used when g_list == NULL) */
  const double* kshift;    /* host, n_kpoints * 3 shifts (kx,ky,kz) in grid units; NULL = 0 */
  const int32_t* g_list;   /* host, optional explicit spheres: concatenated (gx,gy,gz)
                              triples of every k-point, in the order the data uses;
                              copied at plan creation                                */
  const int64_t* g_count;  /* host, n_kpoints sizes of g_list's parts (with g_list)  */
  int32_t layout;          /* 0 = band-major sphere and cube, 1 = batch-fastest      */
  int32_t max_chunk_bands; /* bands per launch chunk; 0 = chosen by the plan         */
} fftb_desc;

/* Plan facts, for allocation and reporting. */
typedef struct {
  int64_t sphere_elems;    /* complex elements of the whole sphere batch            */
  int64_t cube_elems;      /* complex elements of the whole cube batch              */
  int64_t scratch_bytes;   /* device scratch the plan owns                          */
  int32_t total_bands;     /* sum of bands over k-points                            */
  int32_t max_sticks;      /* largest number of occupied (x,y) sticks over k-points */
  int32_t max_slabs;       /* largest number of occupied x values over k-points     */
  int32_t chunk_bands;     /* bands per launch chunk                                */
  int32_t kernels_per_execute; /* kernel launches one fftb_execute issues           */
  int32_t complex_bytes;   /* 8 (FP32, MIXED_TC) or 16 (FP64)                       */
  int32_t stick_ctas;      /* z-stage CTAs per launch (0: one warp per stick group)  */
  int32_t plane_ctas;      /* persistent plane-stage CTAs of this direction (0: one per plane) */
  int32_t prefetch;        /* plane stages that prefetch their inputs with bulk asynchronous
                              copies: bit 0 G->r, bit 1 r->G, bit 2 apply               */
  int32_t slab_buffers;    /* slab planes per plane-stage CTA (1 or 2)                  */
  int32_t tensor_core_planes; /* MIXED_TC plane stages whose y and x DFTs run as dense
                              split-FP16 products on the 5th-generation tensor cores
                              (tcgen05, FP32 accumulators in tensor memory): bit 0 G->r,
                              bit 1 r->G; grids 16, 32, 48, 64 with N0 == N1. Their
                              z stage then runs in FP32.                                */
  int32_t slab_planes_global; /* 1: the slab planes live in a per-CTA block of global
                              memory (planes too large for shared memory: FP64 from
                              160, any precision at 256), 0: in shared memory          */
  int32_t radix_schedule_plane; /* plane stages whose y/x lines use the alternative
                              radix schedule (fftb_plan_set_radix_schedule, or the
                              autotuner per stage): bit 0 G->r, bit 1 r->G, bit 2 apply */
  int32_t radix_schedule_stick; /* the same for the z lines                            */
  int32_t dependent_launch;   /* 1: stage kernels use programmatic dependent launch
                              (fftb_plan_set_pdl, or the autotuner's choice)          */
  int32_t plane_band_group;   /* batch-fastest FP32 plans: bands of one k-point whose
                              G->r / r->G plane stages one CTA runs together, so cube
                              rows move band-contiguous (4 up to 96 points, 2 at 128);
                              0: one band per plane (every other plan)                */
  int64_t graph_launches;     /* executes so far that ran as one CUDA graph launch       */
  double scale_g2r;           /* output normalisation factors (fftb_plan_set_scale)     */
  double scale_r2g;
  int32_t generic_path;       /* 1: extents outside the compiled list (N0 != N1, or an
                              extent not in 12..256 of the list): runtime-length z,
                              y and x kernels with a slab buffer between y and x    */
  int32_t tensor_core_passes; /* MIXED_TC: stages whose radix-8 passes run on mma.sync
                              (bit 0 z, bit 1 plane); 0 where no stage has one      */
  int32_t tensor_cores_available; /* MIXED_TC: 1 if the plan has tensor-core kernels for
                              some stage (in use or not: fftb_plan_set_tensor_cores)  */
  int32_t plane_clusters;     /* plane stages on two-CTA clusters, each CTA holding half
                              of the slab plane in shared memory (bit 0 G->r, bit 1
                              r->G, bit 2 apply; fftb_plan_set_plane_clusters, or the
                              autotuner per stage); bit 3: the plan has those kernels
                              (FP32, 256-point planes)                               */
  /* slab_planes_global above is 1 while a stage the direction uses keeps its
     slab planes in global memory. */
  int32_t pruned_lines;       /* stages that run the kernel variants dropping the middle
                              half of every line at compile time (every k-point's
                              sphere within a quarter of the grid per axis, as with
                              cube width = twice the sphere diameter): bit 0 the z
                              stages, bit 1 the plane stages (FP32 kernels)          */
} fftb_plan_info_t;

/* Builds the spheres, stick/slab tables and twiddles on the host, uploads
 * them to the current CUDA device and allocates the plan's scratch. The only
 * call that allocates device memory or synchronises the device.
 * Paper: the sphere is the cutoff rule of Sec. 2.2 (1/2 |g|^2 <= E_cut, here
 * |G + k| <= r in grid units) or an explicit list / offset array (Sec. 3.3,
 * Fig. 6); the plan fixes the 1D DFT factorisations (Sec. 2.1) and the staged
 * padding order of Fig. 3 (z, then y, then x): the create construct of the
 * paper's API (Sec. 3.1), a transform object built once from its description
 * and then executed (Sec. 3.2).
 * Errors: INVALID_ARG for a bad description (grid extent outside the
 * supported list, sphere that does not fit the grid and would alias, G
 * outside [-N/2, N/2), duplicate G, negative bands, layout other than 0 or
 * 1); UNSUPPORTED for a valid request without a kernel; ALLOC; CUDA. *out is
 * NULL on error. */
fftb_status fftb_plan_create(fftb_plan* out, const fftb_desc* desc,
                             fftb_direction direction, fftb_precision precision);

/* Number of G vectors of one k-point's sphere. */
fftb_status fftb_plan_ngw(fftb_plan plan, int32_t kpoint, int64_t* ngw);

/* Copies one k-point's sphere, ngw*3 int32 (gx,gy,gz), into host memory, in
 * the order the sphere data uses. */
fftb_status fftb_plan_sphere(fftb_plan plan, int32_t kpoint, int32_t* g_out);

/* Fills *info. */
fftb_status fftb_plan_get_info(fftb_plan plan, fftb_plan_info_t* info);

/* Sets the real potential V (device, [N2][N1][N0], float for FP32/MIXED_TC,
 * double for FP64) used by FFTB_APPLY_LOCAL plans. Borrowed: it must stay
 * valid while executes that use it are in flight. */
fftb_status fftb_set_potential(fftb_plan plan, const void* v_dev);

/* Enqueues the transform on `stream` (a cudaStream_t; NULL = legacy default
 * stream). Asynchronous: no synchronisation and no allocation.
 * Paper: G_TO_R is psi(r) = sum_g c(g) e^{+j g r} over the sphere (Sec. 2.2),
 * computed by padding one dimension at a time and transforming it (Fig. 3);
 * R_TO_G is the forward DFT with omega_n = e^{-j 2 pi / n} (Sec. 2.1) sampled
 * on the sphere; APPLY_LOCAL fuses padding, both transforms and the
 * pointwise product (Sec. 2.3). No scaling in either direction. The execute
 * construct of the paper's API (Sec. 3.1).
 *   G_TO_R      : in_dev = sphere batch, out_dev = cube batch, cube_dev NULL
 *   R_TO_G      : in_dev = cube batch,   out_dev = sphere batch, cube_dev NULL
 *   ROUNDTRIP   : in_dev = sphere batch, out_dev = sphere batch,
 *                 cube_dev = cube batch that receives the real-space cube
 *   APPLY_LOCAL : in_dev = sphere batch, out_dev = sphere batch, cube_dev NULL,
 *                 out = P_sphere DFT_fwd(V * DFT_inv(pad(in)))
 * in_dev and out_dev must not overlap; buffers are aligned to the complex
 * element size (8 bytes FP32/MIXED_TC, 16 bytes FP64). */
fftb_status fftb_execute(fftb_plan plan, const void* in_dev, void* out_dev,
                         void* cube_dev, void* stream);

/* As fftb_execute, but in_host / out_host are host buffers (pinned for
 * full-speed copies and for overlap). Copies the input to plan-owned device
 * staging, runs the transform, copies the result back and synchronises
 * `stream`. The bands go through in pieces on three plan-owned streams, so
 * the copy in of one piece, the transform of the previous one and the copy
 * out of the one before that overlap: band-major plans cut the batch into
 * about (bands x N2) / 8192 pieces, at least 2 and at most 16 (never more
 * than the bands), the first and the last of about 2048 (band, z) planes
 * where the batch holds at least 32768 (their copy in and copy out are the
 * ones left exposed); batch-fastest plans split only at k-point boundaries, and
 * a single k-point goes in one piece. The call is ordered
 * after earlier work on `stream` and returns when all of it is done. The
 * staging buffers and streams are created on the first call and kept with
 * the plan. For ROUNDTRIP cube_dev is a device cube batch (may be NULL:
 * plan-owned). A device wait that ran out returns FFTB_ERR_DEVICE_TIMEOUT. */
fftb_status fftb_execute_host(fftb_plan plan, const void* in_host, void* out_host,
                              void* cube_dev, void* stream);

/* Per-kernel timing, for profiling. While enabled, fftb_execute records a
 * CUDA event pair around every kernel it launches, on the execute's stream
 * (the events are created by the first timed execute). Disabled by default.
 * Kinds: 0 z-stage G->r, 1 plane G->r, 2 plane r->G, 3 z-stage r->G,
 * 4 plane apply (FFTB_STAGE_KINDS entries). */
#define FFTB_STAGE_KINDS 5
fftb_status fftb_plan_set_timing(fftb_plan plan, int32_t enable);

/* Waits for the recorded events, writes for each kind the summed kernel
 * milliseconds and launch count since the previous query (arrays of
 * FFTB_STAGE_KINDS entries), then starts a new accumulation. */
fftb_status fftb_plan_stage_times(fftb_plan plan, double* ms, int64_t* launches);

/* CUDA-graph execution. When enabled, fftb_execute records its launch
 * sequence (every band chunk, every stage) into a CUDA graph the first time
 * it sees a given set of buffers (in, out, cube, potential) and replays the
 * instantiated graph on later calls with the same buffers; new buffers update
 * the graph. Recording and instantiation allocate host-side driver
 * resources. On the legacy default stream (NULL), which cannot be captured,
 * the graph is recorded on a plan-owned stream and launched on the default
 * stream. Not used while per-kernel timing is enabled or when `stream` is
 * itself being captured (the kernels then go into the caller's graph).
 * Disabled by default. */
fftb_status fftb_plan_set_graph(fftb_plan plan, int32_t enable);

/* Autotuner: times the candidate schedules of this plan -- first the kernel
 * variant (slab-plane buffers, prefetch level, radix schedules of the plane
 * and z lines), then bands per launch chunk,
 * persistent CTAs of the plane stage and z-stage CTAs -- with `trials` timed
 * executes each on device buffers it allocates and frees (at most 4 GiB;
 * larger batches are tuned on a prefix of the bands), keeps the fastest and
 * reallocates the plan's scratch to fit. If the environment variable
 * FFTB_TUNE_CACHE names a file, results are read from and appended to it,
 * keyed by grid, sphere sizes, bands, direction, precision and device.
 * Synchronises the device. */
fftb_status fftb_plan_autotune(fftb_plan plan, int32_t trials);

/* Bulk-copy prefetch in the plane stage (FP32 plans, slab planes in shared
 * or in global memory). A prefetching plane kernel receives each plane's
 * stick row (G->r, apply) or each warp's next cube rows (r->G; band-major
 * cube buffers 16-byte aligned, grids of 64 and up) through cp.async.bulk
 * copies completed on shared-memory mbarriers, issued one step ahead of
 * their use; the other kernels load with ordinary instructions. Batch-
 * fastest plans prefetch stick rows only (their cube rows are strided). level 0: never; 1 (default): where the staging buffers fit
 * in shared memory without lowering the resident CTAs per SM; 2: wherever
 * they fit. Changing the level resets the persistent plane CTAs of the
 * affected stages to one full wave; fftb_plan_autotune also tries the
 * levels. fftb_plan_info_t.prefetch says which stages prefetch.
 * Errors: INVALID_ARG for a level outside 0..2. */
fftb_status fftb_plan_set_prefetch(fftb_plan plan, int32_t level);

/* Slab-plane buffers of the plane stage: 2 (default where it fits in shared
 * memory) lets a CTA start the next plane's y stage while slower warps
 * finish the current plane's x stage, at twice the memory; 1 halves that
 * memory (more resident CTAs per SM on large grids, or slab planes that stay
 * in L2 when they live in global memory, where 1 is the default) for a
 * second block barrier per plane. Resets the
 * persistent plane CTAs to one full wave; fftb_plan_autotune also tries
 * both. Errors: INVALID_ARG for a count other than 1 or 2; UNSUPPORTED when
 * 2 do not fit in shared memory. */
fftb_status fftb_plan_set_slab_buffers(fftb_plan plan, int32_t nbuf);

/* Radix schedule of the FP32 line FFTs: 0 the default, 1 the alternative for
 * the lengths that have one (64 = 16x4, 96 = 12x8, 128 = 8x16; 160 = 40x4 for
 * the y/x lines and 10x4x4 for the z lines; the defaults are 8x8, 6x4x4, 16x8,
 * and 4x4x2x5 for the y/x lines and 40x4 for the z lines of 160), separately
 * for the y/x lines of the plane stages (here all three at once; the
 * autotuner chooses per stage) and the z lines. The alternative plane schedule excludes the bulk-copy
 * prefetch. Resets the persistent CTAs to one full wave; fftb_plan_autotune
 * also tries the schedules. Errors: INVALID_ARG for
 * values other than 0/1; UNSUPPORTED where no alternative exists (other
 * lengths, FP64, MIXED_TC plane stages, slab planes in global memory). */
fftb_status fftb_plan_set_radix_schedule(fftb_plan plan, int32_t plane, int32_t stick);

/* Programmatic dependent launch between the stage kernels of an execute (on
 * by default; fftb_plan_autotune measures both and keeps the faster): each
 * kernel may launch while its predecessor drains, runs its prologue (twiddle
 * tables, barriers, tensor memory) and waits for the predecessor to complete
 * before touching stage data, so launch latency and prologues overlap the
 * previous kernel's tail. 0 launches them plainly. */
fftb_status fftb_plan_set_pdl(fftb_plan plan, int32_t enable);

/* Optional normalisation (both 1 by default: the transforms are unscaled as
 * in Sec. 2.1-2.2). G->r outputs (the cube of G_TO_R and ROUNDTRIP) are
 * multiplied by g2r; r->G outputs by r2g, and the sphere output of ROUNDTRIP
 * and APPLY_LOCAL by g2r * r2g (the maps are linear). E.g. r2g = 1/(N0 N1 N2)
 * makes the round trip the identity. A factor other than 1 adds one
 * elementwise kernel over that output per execute. INVALID_ARG for a
 * non-finite factor. */
fftb_status fftb_plan_set_scale(fftb_plan plan, double g2r, double r2g);

/* Batch-fastest FP32 plans with N0 == N1 up to 128 run their G->r and r->G
 * plane stages over groups of bands of one k-point (on by default;
 * fftb_plan_autotune measures both): UNSUPPORTED to enable where the plan has
 * no grouped kernels. Results are identical either way. MIXED_TC plans of
 * that shape have them too, in use while their tensor cores are off. */
fftb_status fftb_plan_set_band_groups(fftb_plan plan, int32_t enable);

/* FP32 plans with 256-point planes (N0 == N1 = 256) whose half slab plane,
 * 128 rows of the occupied x-slabs, fits in shared memory (up to about 150
 * slabs): 1 runs the y and x stages on clusters of two CTAs, on two SMs,
 * that share each (band, z) plane, each holding half of its rows and
 * writing the other half's y outputs into its partner's shared memory
 * (distributed shared memory, Sec. 3.1's transposes within a cluster); 0 the
 * single-CTA kernels, whose 256-point slab planes live in global memory.
 * Sets all three plane stages; fftb_plan_autotune times both kinds per
 * stage. Results are the same to rounding. Resets the persistent plane CTAs
 * to one full wave. Errors: UNSUPPORTED to enable where the plan has no
 * cluster kernels. */
fftb_status fftb_plan_set_plane_clusters(fftb_plan plan, int32_t enable);

/* MIXED_TC plans: 1 (the default) runs the stages that have tensor-core
 * kernels on them (tensor_core_planes, tensor_core_passes), 0 runs every
 * stage on the FP32 kernels, with their radix schedules and prefetching
 * (FP32 arithmetic also meets the MIXED_TC error bound, rel. L2 <= 1e-5).
 * fftb_plan_autotune times both and keeps the faster. Resets the radix
 * schedules to the defaults and the persistent CTAs to one full wave. A no-op
 * where no stage has tensor-core kernels (tensor_cores_available = 0).
 * Errors: UNSUPPORTED for FP32 and FP64 plans. */
fftb_status fftb_plan_set_tensor_cores(fftb_plan plan, int32_t enable);

/* Device status. Every wait of a plane kernel on an asynchronous copy gives
 * up after one second; the CTA then lets its copies in flight land, leaves,
 * and sets the plan's status word (mapped host memory), so the context stays
 * usable but the result is invalid. fftb_plan_check synchronises the device,
 * returns FFTB_ERR_DEVICE_TIMEOUT if the word is set since the previous check
 * (and clears it), else FFTB_OK. fftb_execute_host checks it after its own
 * synchronisation. In the checked build (libfftb_check.so, compiled with
 * FFTB_CHECK: every global and slab-plane index of the stick and plane kernels
 * is tested against its buffer before the access) an index outside its buffer
 * is skipped and reported the same way, as FFTB_ERR_DEVICE_BOUNDS. */
fftb_status fftb_plan_check(fftb_plan plan);

/* Test hook for the bounded waits: with FFTB_INJECT_SKIP_FIRST_PREFETCH the
 * first prefetch of CTA 0 (warp 0 in r->G) is not issued in each prefetching
 * plane launch (also in the launches of the 160-point two-pass schedule, whose
 * cube rows (r->G) and stick values (G->r) arrive by bulk copies in each
 * warp's exchange rows: warp 0's first copy), so its wait runs out (about one
 * second, twice: the wait, then the exit's wait for copies in flight) and the
 * status word is set. 0 turns injection off. Unknown bits:
 * FFTB_ERR_INVALID_ARG. */
#define FFTB_INJECT_SKIP_FIRST_PREFETCH 1
fftb_status fftb_plan_inject(fftb_plan plan, int32_t flags);

/* Kernel launches this plan has issued so far (all executes). */
int64_t fftb_plan_launches(fftb_plan plan);

/* Releases the plan's device memory and tables (the clean-up construct of
 * the paper's API, Sec. 3.1). NULL is accepted. Only call it when no execute
 * of the plan is in flight. */
fftb_status fftb_destroy(fftb_plan plan);

/* Static description of a status code. */
const char* fftb_error_string(fftb_status status);

/* Message of the last error raised on the calling thread ("" if none). */
const char* fftb_last_error(void);

/* Allocation-free G -> r. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- real-time or embedded
 * hosts that forbid device allocation after start-up, programs whose device
 * memory is handed out entirely by their own allocator or pool, and libraries
 * that must not change the memory footprint of their caller. Creating a plan
 * allocates; this call does not, and needs no plan.
 *
 * Computes what a G_TO_R FP32 plan for one cutoff sphere computes (same
 * kernels): in_dev = [bands][ngw] complex64 sphere coefficients in canonical
 * order (fftb_sphere_enumerate gives the G list), out_dev = [bands][N2][N1][N0]
 * complex64 cube. Both are caller-owned device buffers, 8-byte aligned.
 * Enqueued on `stream`. The geometry tables are built on the host and
 * uploaded with a copy from pageable host memory on `stream`: the call may
 * block the host until those bytes are staged (about 50 bytes per band plus
 * the sphere's records); the transform itself runs asynchronously.
 *
 * Scratch: the stick buffer and the geometry tables live in two file-scope
 * device arrays of FFTB_NOALLOC_SCRATCH_BYTES and FFTB_NOALLOC_TABLE_BYTES,
 * which every GPU that loads the library holds until the process exits.
 * Bands are processed in chunks that fit the scratch. Limits, each rejected
 * with FFTB_ERR_UNSUPPORTED and a message saying which:
 *   - one band's stick buffer (N2 * sticks * 8 bytes) above the scratch;
 *   - tables above FFTB_NOALLOC_TABLE_BYTES (48 bytes per band plus about
 *     8 bytes per sphere entry: some 40 000 bands of the 160^3, |G| <= 40
 *     sphere per call);
 *   - more than 65535 bands per call (the plans' limit);
 *   - a slab plane (N1 x occupied x values, complex64) that does not fit in
 *     shared memory beside the kernel's exchange rows: on 256-point grids
 *     from |G| <= 41 (83 occupied x values) up, on 128- and 160-point grids
 *     only for spheres far wider than the cube-width = 2 x diameter rule
 *     (a plan keeps such slab planes in device memory instead).
 * Every call shares the arrays and leaves its contents there; nothing in them
 * needs to start at zero. Calls that overlap on the GPU (different streams or
 * host threads) race on the arrays and must be serialised by the caller.
 * The first call on a device looks up the arrays' device addresses once for
 * that device (cudaGetSymbolAddress, with the device current) and keeps them
 * for the life of the process; make that first call before any stream
 * capture. A device reset ends the context those addresses belong to: calls
 * after cudaDeviceReset are not supported.
 * Errors: INVALID_ARG (bad pointer, alignment, sphere that does not fit the
 * grid), UNSUPPORTED (grid extent, the limits above, or `stream` being
 * captured while the pageable table upload is issued), CUDA. */
#define FFTB_NOALLOC_SCRATCH_BYTES (16u << 20)
#define FFTB_NOALLOC_TABLE_BYTES (4u << 20)
fftb_status fftb_g2r_noalloc(const int32_t n[3], double radius, const double* kshift,
                             int32_t bands, const void* in_dev, void* out_dev, void* stream);

/* Host-only helpers (no GPU needed). */

/* Enumerates the cutoff sphere |G + k| <= r of an N0 x N1 x N2 grid (Sec.
 * 2.2) in canonical order (gy, then gx, then gz ascending). kshift may be
 * NULL (k = 0). Sets *ngw; when g_out is non-NULL writes min(ngw, capacity)
 * (gx,gy,gz) triples. INVALID_ARG if the sphere does not fit the grid. */
fftb_status fftb_sphere_enumerate(const int32_t n[3], double radius, const double* kshift,
                                  int32_t* g_out, int64_t capacity, int64_t* ngw);

/* Validates an explicit sphere (components in [-N/2, N/2), no duplicates)
 * and reports its occupied (x,y) sticks and occupied x values: the offset
 * array over the xy projection (Sec. 3.3, Fig. 6) has n_sticks runs. */
fftb_status fftb_sphere_sticks(const int32_t n[3], const int32_t* g, int64_t ngw,
                               int32_t* n_sticks, int32_t* n_slabs);

/* The whole frequency box of an N0 x N1 x N2 grid, every G with components
 * in [-N/2, N/2), in canonical order (gy, then gx, then gz ascending): as a
 * g_list it makes a plan the unpruned 3D transform of the full cube (the
 * classical cuboid transform of Sec. 3.2 / Fig. 5, and the fully padded
 * baseline of Sec. 2.3 that staged padding prunes). Writes N0 N1 N2 triples
 * to g_out (host, capacity checked: INVALID_ARG if capacity is smaller). */
fftb_status fftb_box_enumerate(const int32_t n[3], int32_t* g_out, int64_t capacity);

/* The sphere of an offset array over a bounding domain (Sec. 3.3, Fig. 6 and
 * the domain of Fig. 7), as a g_list in the order of the data. The domain has
 * the inclusive corners lo[3] and hi[3] (any lower corner, e.g. 0..N-1 or a
 * box around the sphere); its xy projection is dense and its z dimension is
 * compressed like CSR rows: column c = (y - lo[1]) * (hi[0] - lo[0] + 1) +
 * (x - lo[0]) (x fastest) holds the entries offsets[c] .. offsets[c+1] - 1,
 * and entry e lies at z = z_index[e] (a domain coordinate in [lo[2], hi[2]]).
 * A domain coordinate v is the frequency v mod N, written to g_out as the
 * signed component in [-N/2, N/2) (N - 1 is -1). offsets has one entry per
 * column plus one, from 0 up to nnz, non-decreasing; g_out (host) takes nnz
 * triples. INVALID_ARG for a domain wider than the grid, a malformed offset
 * array or a z outside the domain; duplicates are caught at plan creation. */
fftb_status fftb_glist_from_offsets(const int32_t n[3], const int32_t lo[3], const int32_t hi[3],
                                    const int64_t* offsets, const int32_t* z_index, int64_t nnz,
                                    int32_t* g_out);

/* Library version string. */
const char* fftb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFTB_H */
