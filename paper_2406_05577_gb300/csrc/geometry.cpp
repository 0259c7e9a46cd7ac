// geometry.cpp -- sphere enumeration and stick/slab tables (host).
// Built with -ffp-contract=off: the squared distance is evaluated left to
// right in IEEE double without fused multiply-adds, so sphere membership is
// reproducible bit for bit.
#include "geometry.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace fftb {

static inline bool in_ball(int64_t gx, int64_t gy, int64_t gz, const double k[3], double r2) {
  const double ax = (double)gx + k[0];
  const double ay = (double)gy + k[1];
  const double az = (double)gz + k[2];
  double d = ax * ax;
  d = d + ay * ay;
  d = d + az * az;
  return d <= r2;
}

std::string sphere_by_cutoff(const int32_t n[3], double radius, const double k[3],
                             std::vector<int32_t>& g) {
  g.clear();
  if (!(radius >= 0.0) || !std::isfinite(radius)) return "radius must be finite and >= 0";
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(k[d])) return "k-shift must be finite";
  const double r2 = radius * radius;
  // Aliasing check: enumerate the ball over a box one cell wider than its
  // extent; every member must have components inside [-N/2, N/2).
  int64_t lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = (int64_t)std::floor(-radius - k[d]) - 1;
    hi[d] = (int64_t)std::ceil(radius - k[d]) + 1;
    // a ball wider than the grid cannot fit; also bounds the loops below
    if (hi[d] - lo[d] > (int64_t)n[d] + 4) return "sphere does not fit the grid";
  }
  for (int64_t gy = lo[1]; gy <= hi[1]; ++gy)
    for (int64_t gx = lo[0]; gx <= hi[0]; ++gx)
      for (int64_t gz = lo[2]; gz <= hi[2]; ++gz) {
        if (!in_ball(gx, gy, gz, k, r2)) continue;
        const int64_t v[3] = {gx, gy, gz};
        for (int d = 0; d < 3; ++d) {
          const int64_t h = n[d] / 2;
          if (v[d] < -h || v[d] >= n[d] - h) return "sphere does not fit the grid";
        }
      }
  // Canonical order: gy, then gx, then gz, ascending over signed values.
  const int64_t h0 = n[0] / 2, h1 = n[1] / 2, h2 = n[2] / 2;
  for (int64_t gy = -h1; gy < n[1] - h1; ++gy)
    for (int64_t gx = -h0; gx < n[0] - h0; ++gx)
      for (int64_t gz = -h2; gz < n[2] - h2; ++gz)
        if (in_ball(gx, gy, gz, k, r2)) {
          g.push_back((int32_t)gx);
          g.push_back((int32_t)gy);
          g.push_back((int32_t)gz);
        }
  return "";
}

static inline int32_t wrap(int32_t v, int32_t n) {
  const int32_t m = v % n;
  return m < 0 ? m + n : m;
}

std::string build_geometry(const int32_t n[3], const int32_t* g, int64_t ngw, KGeom& out) {
  out = KGeom();
  out.ngw = ngw;
  if (ngw < 0) return "negative sphere size";
  if (ngw >= (int64_t(1) << 31)) return "sphere too large";
  if (n[2] > 256) return "N2 above 256 is not supported";
  out.g.assign(g, g + 3 * ngw);
  // range and duplicate checks
  std::vector<uint8_t> seen((size_t)n[0] * n[1] * n[2], 0);
  for (int64_t i = 0; i < ngw; ++i) {
    for (int d = 0; d < 3; ++d) {
      const int32_t h = n[d] / 2;
      const int32_t v = g[3 * i + d];
      if (v < -h || v >= n[d] - h) return "G component outside [-N/2, N/2)";
    }
    const size_t cell = ((size_t)wrap(g[3 * i + 2], n[2]) * n[1] + wrap(g[3 * i + 1], n[1])) * n[0] +
                        wrap(g[3 * i], n[0]);
    if (seen[cell]) return "duplicate G vector in sphere list";
    seen[cell] = 1;
  }
  std::vector<int32_t> order((size_t)ngw);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (g[3 * a] != g[3 * b]) return g[3 * a] < g[3 * b];
    if (g[3 * a + 1] != g[3 * b + 1]) return g[3 * a + 1] < g[3 * b + 1];
    return g[3 * a + 2] < g[3 * b + 2];
  });
  // occupied x values, ascending signed
  std::vector<int32_t> xs;
  for (int64_t i = 0; i < ngw; ++i) xs.push_back(g[3 * i]);
  std::sort(xs.begin(), xs.end());
  xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
  out.X = (int32_t)xs.size();
  out.xmap.assign(n[0], (int16_t)-1);
  for (size_t i = 0; i < xs.size(); ++i) out.xmap[wrap(xs[i], n[0])] = (int16_t)i;

  out.col_start.assign((size_t)out.X + 1, 0);
  out.ent_pos.resize(ngw);
  out.ent_zs.resize(ngw);
  int32_t s = -1;
  int32_t py = 0, px = 0;
  for (int64_t j = 0; j < ngw; ++j) {
    const int32_t i = order[j];
    const int32_t gx = g[3 * i], gy = g[3 * i + 1], gz = g[3 * i + 2];
    if (s < 0 || gx != px || gy != py) {
      if (s >= 0 && gx == px && gy != py + 1) out.contiguous_columns = false;
      ++s;
      px = gx;
      py = gy;
      out.stick_ent.push_back((int32_t)j);
      const int32_t xi = out.xmap[wrap(gx, n[0])];
      out.stick_xy.push_back((xi << 16) | wrap(gy, n[1]));
      out.col_start[xi + 1] = s + 1;
    }
    if (j > 0 && out.stick_ent.back() != (int32_t)j &&
        (gz != g[3 * order[j - 1] + 2] + 1 || i != order[j - 1] + 1))
      out.canonical_sticks = false;
    out.ent_pos[j] = i;
    out.ent_zs[j] = (wrap(gz, n[2]) << 24) | s;
  }
  out.S = s + 1;
  out.stick_ent.push_back((int32_t)ngw);
  for (int32_t xi = 1; xi <= out.X; ++xi) out.col_start[xi] = std::max(out.col_start[xi], out.col_start[xi - 1]);
  // the entry records hold the stick index in 24 bits
  if (out.S >= (1 << 24)) return "too many sticks (limit 16777215)";
  return "";
}

static inline int32_t signed_index(int32_t v, int32_t n) { return v < n - n / 2 ? v : v - n; }

void stick_records(const KGeom& g, const int32_t n[3], int32_t ent_base, std::vector<int32_t>& out4) {
  for (int32_t s = 0; s < g.S; ++s) {
    const int32_t e0 = g.stick_ent[s], e1 = g.stick_ent[s + 1];
    out4.push_back(e0 + ent_base);
    out4.push_back(e1 + ent_base);
    out4.push_back(g.ent_pos[e0]);
    out4.push_back(signed_index((int32_t)((uint32_t)g.ent_zs[e0] >> 24), n[2]));
  }
}

void slab_records(const KGeom& g, const int32_t n[3], std::vector<int32_t>& out4) {
  for (int32_t xi = 0; xi < g.X; ++xi) {
    const int32_t sa = g.col_start[xi], sb = g.col_start[xi + 1];
    out4.push_back(sa);
    out4.push_back(sb - sa);
    out4.push_back(sb > sa ? signed_index(g.stick_xy[sa] & 0xFFFF, n[1]) : 0);
    out4.push_back(0);
  }
}

}  // namespace fftb
