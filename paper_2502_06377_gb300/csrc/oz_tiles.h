// Lower-tile enumeration of the digit-pair launches (internal): a symmetric
// product takes only the 128-row x bn-column output tiles that reach the
// diagonal or below it, numbered row by row, so that the persistent CTAs that
// own every gridDim-th tile get balanced shares.  Host-compilable for checks
// on the CPU.
#pragma once

#if defined(__CUDACC__)
#define OZT_HD __host__ __device__ __forceinline__
#else
#define OZT_HD inline
#endif

namespace ibmi {

constexpr int OZT_BM = 128;   // rows of an output tile

// Tiles of tile row mt: those whose first column is at most the row tile's
// last row (at most grid_n).
OZT_HD int oz_lower_row_tiles(int mt, int grid_n, int bn) {
  const int n = ((mt + 1) * OZT_BM + bn - 1) / bn;
  return n < grid_n ? n : grid_n;
}

// Tiles of a lower launch with grid_m tile rows.
OZT_HD int oz_lower_tiles(int grid_m, int grid_n, int bn) {
  int n = 0;
  for (int mt = 0; mt < grid_m; ++mt) n += oz_lower_row_tiles(mt, grid_n, bn);
  return n;
}

// Tile (mt, ntl) of lower index tl (0 <= tl < oz_lower_tiles).
OZT_HD void oz_lower_tile(int tl, int grid_n, int bn, int& mt, int& ntl) {
  mt = 0;
  for (int n = oz_lower_row_tiles(0, grid_n, bn); tl >= n; n = oz_lower_row_tiles(mt, grid_n, bn)) {
    tl -= n;
    ++mt;
  }
  ntl = tl;
}

}  // namespace ibmi
