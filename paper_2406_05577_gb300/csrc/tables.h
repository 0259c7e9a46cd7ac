// tables.h -- the device tables a transform reads (band records, k-point
// records, stick / entry / slab records, the x -> slab map, per-axis
// twiddles), packed into one host blob with 256-byte aligned parts. Plans and
// the allocation-free entry point build their tables through these helpers,
// so both hand the kernels the same layout.
#pragma once

#include <cmath>
#include <cstring>
#include <vector>

#include "fftb_internal.h"

namespace fftb {

// e^{+2 pi j m / n}, m = 0..n-1, evaluated in double and rounded once to T.
template <typename T> void make_twiddles(int n, std::vector<unsigned char>& out) {
  out.resize(sizeof(T) * 2 * (size_t)n);
  T* p = reinterpret_cast<T*>(out.data());
  for (int m = 0; m < n; ++m) {
    const double a = 2.0 * M_PI * (double)m / (double)n;
    p[2 * m] = (T)std::cos(a);
    p[2 * m + 1] = (T)std::sin(a);
  }
}

// The host-side sources of the tables; empty record lists are padded with a
// zero entry when packed (the kernels may read them as a dummy).
struct TableParts {
  std::vector<BandInfo> band;
  std::vector<KInfo> kinfo;
  std::vector<int32_t> stick_info, ent_pos, ent_zs, stick_xy, col_info;
  std::vector<int16_t> xmap;
  std::vector<unsigned char> tw[3];
};

enum { TP_BAND, TP_KINFO, TP_STICK, TP_POS, TP_ZS, TP_XY, TP_XMAP, TP_TW0, TP_TW1, TP_TW2, TP_COL, TP_COUNT };

// Byte offsets of every part and the blob size.
struct TableLayout {
  size_t off[TP_COUNT];
  size_t total;
};

inline TableLayout table_layout(TableParts& t) {
  if (t.band.empty()) t.band.push_back(BandInfo{});
  if (t.kinfo.empty()) t.kinfo.push_back(KInfo{});
  if (t.ent_pos.empty()) t.ent_pos.push_back(0);
  if (t.ent_zs.empty()) t.ent_zs.push_back(0);
  if (t.stick_xy.empty()) t.stick_xy.push_back(0);
  if (t.stick_info.empty()) t.stick_info.assign(4, 0);
  if (t.col_info.empty()) t.col_info.assign(4, 0);
  if (t.xmap.empty()) t.xmap.push_back(-1);
  const size_t bytes[TP_COUNT] = {t.band.size() * sizeof(BandInfo), t.kinfo.size() * sizeof(KInfo),
                                  t.stick_info.size() * 4, t.ent_pos.size() * 4, t.ent_zs.size() * 4,
                                  t.stick_xy.size() * 4, t.xmap.size() * 2, t.tw[0].size(), t.tw[1].size(),
                                  t.tw[2].size(), t.col_info.size() * 4};
  TableLayout L{};
  size_t total = 0;
  for (int i = 0; i < TP_COUNT; ++i) {
    L.off[i] = total;
    total = (total + bytes[i] + 255) / 256 * 256;
  }
  L.total = total;
  return L;
}

// Copies every part to its offset in blob (blob holds L.total bytes).
inline void table_fill(const TableParts& t, const TableLayout& L, unsigned char* blob) {
  std::memset(blob, 0, L.total);
  auto put = [&](int i, const void* src, size_t bytes) {
    if (bytes) std::memcpy(blob + L.off[i], src, bytes);
  };
  put(TP_BAND, t.band.data(), t.band.size() * sizeof(BandInfo));
  put(TP_KINFO, t.kinfo.data(), t.kinfo.size() * sizeof(KInfo));
  put(TP_STICK, t.stick_info.data(), t.stick_info.size() * 4);
  put(TP_POS, t.ent_pos.data(), t.ent_pos.size() * 4);
  put(TP_ZS, t.ent_zs.data(), t.ent_zs.size() * 4);
  put(TP_XY, t.stick_xy.data(), t.stick_xy.size() * 4);
  put(TP_XMAP, t.xmap.data(), t.xmap.size() * 2);
  for (int d = 0; d < 3; ++d) put(TP_TW0 + d, t.tw[d].data(), t.tw[d].size());
  put(TP_COL, t.col_info.data(), t.col_info.size() * 4);
}

// The kernels' table pointers for a blob uploaded to device address base.
inline void table_geo(Geo& g, const void* base, const TableLayout& L) {
  const unsigned char* b = static_cast<const unsigned char*>(base);
  g.band = reinterpret_cast<const BandInfo*>(b + L.off[TP_BAND]);
  g.stick_info = reinterpret_cast<const int4*>(b + L.off[TP_STICK]);
  g.ent_pos = reinterpret_cast<const int32_t*>(b + L.off[TP_POS]);
  g.ent_zs = reinterpret_cast<const int32_t*>(b + L.off[TP_ZS]);
  g.stick_xy = reinterpret_cast<const int32_t*>(b + L.off[TP_XY]);
  g.col_info = reinterpret_cast<const int4*>(b + L.off[TP_COL]);
  g.xmap = reinterpret_cast<const int16_t*>(b + L.off[TP_XMAP]);
  g.tw0 = b + L.off[TP_TW0];
  g.tw1 = b + L.off[TP_TW1];
  g.tw2 = b + L.off[TP_TW2];
}

}  // namespace fftb
