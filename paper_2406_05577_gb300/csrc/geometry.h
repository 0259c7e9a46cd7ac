// geometry.h -- host-side sphere enumeration and stick / slab tables.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace fftb {

// One k-point's sphere and the tables the kernels index it with.
//   sticks (occupied (x,y) columns) are numbered x-major: by gx, then gy,
//   so the sticks of one x-slab are consecutive (the offset array over the
//   xy projection of Sec. 3.3 / Fig. 6, regrouped slab by slab);
//   entries are the sphere's G sorted by stick and then gz;
//   stick_ent[s] .. stick_ent[s+1] are the entries of stick s (S + 1 values);
//   ent_pos[j] is entry j's position in the caller's sphere list;
//   ent_zs[j]  = (gz mod N2) << 24 | s;
//   xmap[x] = xi of x = gx mod N0 (rank of gx among occupied x), or -1;
//   col_start[xi] .. col_start[xi+1] are the sticks of slab xi (X + 1 values);
//   stick_xy[s] = xi << 16 | (gy mod N1).
struct KGeom {
  int64_t ngw = 0;
  std::vector<int32_t> g;  // ngw * 3, the caller's order
  int32_t S = 0, X = 0;
  bool contiguous_columns = true;  // each slab's sticks have consecutive gy
  bool canonical_sticks = true;    // each stick: consecutive gz at consecutive list positions
  std::vector<int32_t> stick_ent, ent_pos, ent_zs, col_start, stick_xy;
  std::vector<int16_t> xmap;
};

// Per-stick and per-slab records the kernels read in one 16-byte load:
//   stick: {first entry + ent_base, end entry + ent_base, list position of the
//           first entry, signed gz of the first entry}
//   slab : {first stick, number of sticks, signed gy of the first stick, 0}
void stick_records(const KGeom& g, const int32_t n[3], int32_t ent_base, std::vector<int32_t>& out4);
void slab_records(const KGeom& g, const int32_t n[3], std::vector<int32_t>& out4);

// Cutoff sphere |G + k| <= r (Sec. 2.2), components in [-N/2, N/2), in
// canonical order (gy, gx, gz ascending). Returns "" or an error message
// (the sphere does not fit the grid and would alias).
std::string sphere_by_cutoff(const int32_t n[3], double radius, const double k[3],
                             std::vector<int32_t>& g);

// Builds the tables for a sphere given as ngw (gx,gy,gz) triples. Returns ""
// or an error message (component out of range, duplicate G, size limit).
std::string build_geometry(const int32_t n[3], const int32_t* g, int64_t ngw, KGeom& out);

}  // namespace fftb
