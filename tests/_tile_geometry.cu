// Host-side check of the tile geometry (GeoT in rt_step_kernel.cuh) for every
// compiled tile shape, in both layouts: the double/pair kernels' and the
// quad kernel's (odd box and x-array rows, y innermost).  Built and run by
// tests/test_tile_geometry.py; prints OK when every check holds.
//  - the cross-shaped staging set (tile plus a two-cell halo per active
//    axis) maps into [0, nbox) without collisions;
//  - the slope index of axis d over l_d in [-1, T_d] (the extension layer)
//    and the tile's other coordinates maps into that axis's slice of the
//    slope array without collisions, and likewise the flux index over the
//    T_d + 1 faces;
//  - the compile-time constants agree with the runtime Geo the host sizes
//    shared memory with;
//  - in the quad layout with two or more axes, the box row, the x-slope row
//    and the x-flux row have odd lengths, and eight cells consecutive in y
//    fall on eight different 16-byte bank groups in each of the three.
#include <cstdio>
#include <vector>

#include "rt_step_kernel.cuh"

using namespace rtg::stepk;

static int failures = 0;
#define CHECK(c)                                                               \
  do {                                                                         \
    if (!(c)) {                                                                \
      std::printf("failed: %s (line %d, shape %d:%dx%dx%d q%d)\n", #c, __LINE__, \
                  DIM, TX, TY, TZ, (int)Q);                                    \
      ++failures;                                                              \
    }                                                                          \
  } while (0)

template <int DIM, int TX, int TY, int TZ, bool Q>
void check() {
  using G = GeoT<DIM, TX, TY, TZ, Q>;
  Geo r;
  r.init(DIM, TX, TY, TZ, Q);
  CHECK(G::nbox == r.nbox && G::SL3 == r.sl_off[3] && G::FX3 == r.fx_off[3] && G::B0 == r.B[0] && G::B1 == r.B[1]);
  const int T[3] = {TX, TY, TZ};
  // staging set
  std::vector<int> box(G::nbox, 0);
  int staged = 0;
  for (int z = -kHalo; z < TZ + kHalo; ++z)
    for (int y = -kHalo; y < TY + kHalo; ++y)
      for (int x = -kHalo; x < TX + kHalo; ++x) {
        const int l[3] = {x, y, z};
        int outside = 0, bad = 0;
        for (int d = 0; d < 3; ++d) {
          if (d >= DIM && l[d] != 0) bad = 1;
          if (l[d] < 0 || l[d] >= T[d]) ++outside;
        }
        if (bad || outside > 1) continue;   // only the cross-shaped part is staged
        const int b = (x + kHalo) + G::B0 * ((DIM >= 2 ? y + kHalo : 0) + G::B1 * (DIM >= 3 ? z + kHalo : 0));
        CHECK(b >= 0 && b < G::nbox);
        if (b >= 0 && b < G::nbox) {
          CHECK(box[b] == 0);
          box[b] = 1;
        }
        ++staged;
      }
  CHECK(staged == r.ncross);
  // slopes and fluxes per axis
  std::vector<int> sl(G::SL3, 0), fx(G::FX3, 0);
  for (int d = 0; d < DIM; ++d) {
    for (int z = (d == 2 ? -1 : 0); z < (d == 2 ? TZ + 1 : TZ); ++z)
      for (int y = (d == 1 ? -1 : 0); y < (d == 1 ? TY + 1 : TY); ++y)
        for (int x = (d == 0 ? -1 : 0); x < (d == 0 ? TX + 1 : TX); ++x) {
          const int i = G::sl_off(d) + G::sl_idx(d, x, y, z);
          CHECK(i >= r.sl_off[d] && i < r.sl_off[d + 1]);
          if (i >= 0 && i < G::SL3) {
            CHECK(sl[i] == 0);
            sl[i] = 1;
          }
          if ((d == 0 ? x : d == 1 ? y : z) < T[d]) {   // the next cell's slope is one step on
            const int j = G::sl_off(d) + G::sl_idx(d, d == 0 ? x + 1 : x, d == 1 ? y + 1 : y, d == 2 ? z + 1 : z);
            CHECK(j == i + G::sl_step(d));
          }
        }
    for (int z = 0; z < (d == 2 ? TZ + 1 : TZ); ++z)
      for (int y = 0; y < (d == 1 ? TY + 1 : TY); ++y)
        for (int x = 0; x < (d == 0 ? TX + 1 : TX); ++x) {
          const int f = d == 0 ? x : d == 1 ? y : z;
          const int i = G::fx_off(d) + G::fx_idx(d, f, x, y, z);
          CHECK(i >= r.fx_off[d] && i < r.fx_off[d + 1]);
          if (i >= 0 && i < G::FX3) {
            CHECK(fx[i] == 0);
            fx[i] = 1;
          }
          if (f < T[d]) CHECK(G::fx_idx(d, f + 1, x, y, z) == G::fx_idx(d, f, x, y, z) + G::fx_step(d));
        }
  }
  // the quad layout's odd rows
  if (Q && DIM >= 2) {
    CHECK(G::B0 % 2 == 1 && G::RX % 2 == 1 && G::RXF % 2 == 1);
    for (int x = -1; x <= TX; ++x) {
      for (int z = 0; z < TZ; ++z)
        for (int y0 = 0; y0 + 8 <= TY; y0 += 8) {
          int gb = 0, gs = 0, gf = 0;
          for (int y = y0; y < y0 + 8; ++y) {
            gb |= 1 << (((x + kHalo) + G::B0 * ((y + kHalo) + G::B1 * (DIM >= 3 ? z + kHalo : 0))) & 7);
            gs |= 1 << (G::sl_idx(0, x, y, z) & 7);
            if (x >= 0) gf |= 1 << (G::fx_idx(0, x, x, y, z) & 7);
          }
          CHECK(gb == 0xff && gs == 0xff && (x < 0 || gf == 0xff));
        }
    }
  }
}

template <bool Q>
void all() {
  check<3, 8, 8, 4, Q>();
  check<3, 16, 8, 4, Q>();
  check<3, 8, 4, 4, Q>();
  check<3, 4, 4, 4, Q>();
  check<2, 32, 16, 1, Q>();
  check<2, 16, 16, 1, Q>();
  check<2, 16, 8, 1, Q>();
  check<2, 8, 8, 1, Q>();
  check<2, 8, 4, 1, Q>();
  check<1, 512, 1, 1, Q>();
  check<1, 256, 1, 1, Q>();
  check<1, 128, 1, 1, Q>();
  check<1, 64, 1, 1, Q>();
  check<1, 32, 1, 1, Q>();
}

int main() {
  all<false>();
  all<true>();
  if (failures == 0) std::printf("OK\n");
  return failures == 0 ? 0 : 1;
}
