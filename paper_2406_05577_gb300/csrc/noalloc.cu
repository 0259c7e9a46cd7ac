// noalloc.cu -- fftb_g2r_noalloc: the G -> r transform for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time or embedded hosts that
// forbid device allocation after start-up, programs whose device memory is
// handed out entirely by their own allocator or pool (a cudaMalloc behind its
// back would break its accounting or fail), and libraries that must not
// change the memory footprint of the process that calls them. Creating a plan
// allocates, so those callers cannot use fftb_plan_create. This entry point
// needs no plan and allocates nothing: the stick scratch and the geometry
// tables live in the two file-scope arrays below, which every GPU that loads
// the library holds until the process exits.
//
// The first call on a device looks up the arrays' device addresses
// (cudaGetSymbolAddress, once per device, with that device current) and
// keeps them for the life of the process; make that first call before any
// stream capture. A device reset (cudaDeviceReset) ends the context those
// addresses belong to: calls after a reset are not supported.
//
// The scratch is the stick buffer T between the z-stage and the plane stage
// (the same kernels as a G_TO_R plan). Every call shares both arrays and
// leaves the last call's contents in them; nothing in them needs to start at
// zero, because each call writes every table word and every T entry it later
// reads. Calls that overlap on the GPU (two streams, or two host threads)
// race on the arrays: serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fftb.h"
#include "fftb_internal.h"
#include "geometry.h"
#include "tables.h"

namespace fftb {
template <typename T, bool TC> size_t plane_smem_t(int, int, int, int, bool);
template <typename T, bool TC> int stick_tile_t(int);
template <typename T, bool TC> cudaError_t launch_stick_t(int, const Launch&, int);
template <typename T, bool TC> cudaError_t launch_plane_t(int, const Launch&);
template <typename T, bool TC> cudaError_t prepare_t(int, int, int, int, int, bool);
}  // namespace fftb

static __device__ __align__(256) unsigned char g_noalloc_scratch[FFTB_NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) unsigned char g_noalloc_tables[FFTB_NOALLOC_TABLE_BYTES];

namespace {

fftb_status err(fftb_status s, const std::string& m) {
  fftb::set_last_error(m);  // read back with fftb_last_error()
  return s;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices];
void* g_tables_ptr[kMaxDevices];

// Once per device, with that device current: device addresses of the arrays.
fftb_status device_arrays(int dev, void** scratch, void** tables) {
  if (dev < 0 || dev >= kMaxDevices) return err(FFTB_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* s = nullptr;
    void* t = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&s, g_noalloc_scratch);
    if (e != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&t, g_noalloc_tables);
    if (e != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("cudaGetSymbolAddress(tables): ") + cudaGetErrorString(e));
    g_tables_ptr[dev] = t;
    g_scratch_ptr[dev] = s;
  }
  *scratch = g_scratch_ptr[dev];
  *tables = g_tables_ptr[dev];
  return FFTB_OK;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) fftb_status fftb_g2r_noalloc(
    const int32_t n[3], double radius, const double* kshift, int32_t bands, const void* in_dev,
    void* out_dev, void* stream) {
  using namespace fftb;
  if (!n) return err(FFTB_ERR_INVALID_ARG, "n is NULL");
  if (bands < 0) return err(FFTB_ERR_INVALID_ARG, "bands must be >= 0");
  if (bands > 65535) return err(FFTB_ERR_UNSUPPORTED, "at most 65535 bands per call (as per plan)");
  if (!grid_size_supported(n[0]) || !grid_size_supported(n[1]) || !grid_size_supported(n[2]) ||
      !plane_size_supported(n[0], n[1]))
    return err(FFTB_ERR_UNSUPPORTED, "grid extents must be one of 12,16,20,24,32,40,48,64,96,128,160,256 with N0 == N1");
  if (bands == 0) return FFTB_OK;
  if (!in_dev || !out_dev) return err(FFTB_ERR_INVALID_ARG, "in_dev and out_dev must be device pointers");
  if ((reinterpret_cast<uintptr_t>(in_dev) | reinterpret_cast<uintptr_t>(out_dev)) % 8 != 0)
    return err(FFTB_ERR_INVALID_ARG, "buffers must be 8-byte aligned (complex64)");

  const double zero[3] = {0, 0, 0};
  std::vector<int32_t> g;
  std::string e = sphere_by_cutoff(n, radius, kshift ? kshift : zero, g);
  if (!e.empty()) return err(FFTB_ERR_INVALID_ARG, e);
  KGeom G;
  e = build_geometry(n, g.data(), (int64_t)g.size() / 3, G);
  if (!e.empty()) return err(FFTB_ERR_INVALID_ARG, e);

  // stick scratch: as many bands per launch as the static array holds
  const int32_t smax = std::max<int32_t>(G.S, 1);
  const size_t t_band = (size_t)n[2] * smax * 8;
  if (t_band > FFTB_NOALLOC_SCRATCH_BYTES)
    return err(FFTB_ERR_UNSUPPORTED, "one band's stick buffer (" + std::to_string(t_band) +
                                         " bytes) exceeds FFTB_NOALLOC_SCRATCH_BYTES");
  const int chunk = (int)std::min<size_t>((size_t)bands, FFTB_NOALLOC_SCRATCH_BYTES / t_band);
  const int a_bufs = plane_smem_t<float, false>(n[0], n[1], G.X, 2, false) <= 227 * 1024 ? 2 : 1;
  if (plane_smem_t<float, false>(n[0], n[1], G.X, a_bufs, false) > 227 * 1024)
    return err(FFTB_ERR_UNSUPPORTED, "the slab plane (N1 x " + std::to_string(G.X) +
                                         " occupied x values) does not fit in shared memory; this entry point has "
                                         "no global slab-plane scratch (a plan has)");

  // tables of a one-k-point plan, packed by the plans' own helper
  KInfo ki{G.S, G.X, 0, 0, 0,
           (G.contiguous_columns ? KF_CONTIGUOUS_COLUMNS : 0) | (G.canonical_sticks ? KF_CANONICAL_STICKS : 0), 1};
  const int64_t vol = (int64_t)n[0] * n[1] * n[2];
  TableParts tp;
  tp.band.resize((size_t)bands);
  for (int b = 0; b < bands; ++b) {
    tp.band[b].ki = ki;
    tp.band[b].sph = (int64_t)b * G.ngw;
    tp.band[b].cube = (int64_t)b * vol;
  }
  tp.kinfo.push_back(ki);
  stick_records(G, n, 0, tp.stick_info);
  slab_records(G, n, tp.col_info);
  tp.ent_pos = G.ent_pos;
  tp.ent_zs = G.ent_zs;
  tp.stick_xy = G.stick_xy;
  tp.xmap = G.xmap;
  for (int d = 0; d < 3; ++d) make_twiddles<float>(n[d], tp.tw[d]);
  const TableLayout tl = table_layout(tp);
  if (tl.total > FFTB_NOALLOC_TABLE_BYTES)
    return err(FFTB_ERR_UNSUPPORTED, "geometry tables for " + std::to_string(bands) + " bands (" +
                                         std::to_string(tl.total) + " bytes: 48 per band plus the sphere's records) "
                                         "exceed FFTB_NOALLOC_TABLE_BYTES; split the bands over several calls");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the table upload below copies from pageable host memory, which a stream
  // capture does not take
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(ce));
  if (cap != cudaStreamCaptureStatusNone)
    return err(FFTB_ERR_UNSUPPORTED, "stream is being captured: the table upload copies from pageable host memory");
  int dev = 0;
  ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  void* scratch = nullptr;
  void* tables = nullptr;
  fftb_status st = device_arrays(dev, &scratch, &tables);
  if (st != FFTB_OK) return st;
  ce = prepare_t<float, false>(n[0], n[1], n[2], G.X, a_bufs, false);
  if (ce != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(ce));

  std::vector<unsigned char> blob(tl.total);
  table_fill(tp, tl, blob.data());
  // pageable source: the copy returns once the bytes are staged (it may block
  // the host until then), so blob may go when the call returns
  ce = cudaMemcpyAsync(tables, blob.data(), tl.total, cudaMemcpyHostToDevice, s);
  if (ce != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(ce));

  Launch L{};
  table_geo(L.g, tables, tl);
  L.g.n0 = n[0];
  L.g.n1 = n[1];
  L.g.n2 = n[2];
  L.g.smax = smax;
  L.g.xmax = G.X;
  L.sph_in = in_dev;
  L.cube_out = out_dev;
  L.T = scratch;
  L.a_bufs = a_bufs;
  L.lim_sph = (int64_t)bands * G.ngw;
  L.lim_cube = (int64_t)bands * vol;
  L.lim_T = (int64_t)(FFTB_NOALLOC_SCRATCH_BYTES / 8);
  L.lim_V = 0;
  L.stream = s;
  for (int b0 = 0; b0 < bands; b0 += chunk) {
    L.band0 = b0;
    L.nb = std::min(chunk, bands - b0);
    ce = launch_stick_t<float, false>(M_G2R, L, 0);
    if (ce == cudaSuccess) ce = launch_plane_t<float, false>(M_G2R, L);
    if (ce != cudaSuccess) return err(FFTB_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(ce));
  }
  return FFTB_OK;
}
