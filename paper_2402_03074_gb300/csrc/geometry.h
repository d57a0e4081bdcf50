// geometry.h -- launch geometry of the fused 2D stage: how a grid is cut into work items of
// (band of columns) x (chunk of rows).  Host code in plain C++ (no CUDA types), shared by the
// single-solve launch (stage2d.cu), the batched launches (batch.cu, static_batch.cu) and the
// serving loop (server.cu).
//
// A block of bw threads covers a band of at most bw - 2 output columns plus one ring column
// on each side, and sweeps a chunk of rows (one ring row above and below).  The time of a
// launch is set by its waves of items over the resident block slots and by the rows of an
// item: a block's row sweep is bound by the latency of its own instruction stream, so a block
// alone on an SM is not faster than one of two sharing it.
#pragma once

namespace hw {

// lanes (threads in whole warps) that `bands` equal bands over nx columns occupy, each band
// with its two ring columns
inline int band_lanes(int nx, int bands) {
  const int w = (nx + bands - 1) / bands;
  return bands * 32 * ((w + 2 + 31) / 32);
}

// Default band count for blocks of bw threads: the widest bands (at most bw - 2 output
// columns).  With lane_aware (the FP64 kernels, whose two blocks per SM keep the FP64 pipe
// busy with three active warps each), bands of at most bw - 34 columns when they leave fewer
// idle lanes (2048 columns: 22 bands of 94 columns in 96 lanes each rather than 17 of 121 in
// 128).
inline int default_bands(int nx, int bw, bool lane_aware) {
  int b = (nx + (bw - 2) - 1) / (bw - 2);
  if (lane_aware && bw > 34) {
    const int b3 = (nx + (bw - 34) - 1) / (bw - 34);
    if (b3 <= nx && 100LL * band_lanes(nx, b3) < 99LL * band_lanes(nx, b)) b = b3;
  }
  return b;
}

// Equal bands: the output columns per band for `bands` requested bands, and the band count
// that leaves no band empty.
inline void split_bands(int nx, int bands_req, int* bands, int* wout) {
  *wout = (nx + bands_req - 1) / bands_req;
  *bands = (nx + *wout - 1) / *wout;
}

// Single-solve launch: bands as above (or fixed, but never wider than bw - 2 columns) and row
// chunks sized so that bands x chunks fills the `slots` resident blocks once (or fixed rows).
struct Geom2D {
  int bands, wout, chunks, rows;
};
inline Geom2D geom2d(int nx, int ny, int bw, int slots, int rows_fixed, int bands_fixed,
                     bool lane_aware) {
  Geom2D g;
  const int bwide = (nx + (bw - 2) - 1) / (bw - 2);
  int b = bands_fixed > 0 ? (bands_fixed < nx ? bands_fixed : nx) : default_bands(nx, bw, lane_aware);
  if (bands_fixed > 0 && b < bwide) b = bwide;  // a band is at most bw - 2 columns wide
  split_bands(nx, b, &g.bands, &g.wout);
  if (rows_fixed > 0) {
    g.rows = rows_fixed < ny ? rows_fixed : ny;
  } else {
    int ch = slots / g.bands;
    if (ch < 1) ch = 1;
    if (ch > ny) ch = ny;
    g.rows = (ny + ch - 1) / ch;
  }
  g.chunks = (ny + g.rows - 1) / g.rows;
  return g;
}

// Rows per work item for the 2D solves of one batched class (bands[s] bands and ny[s] rows
// each) whose persistent launch has `slots` resident blocks.  The launch runs
// ceil(items / slots) waves, a partial last wave costing a whole item time, and an item costs
// its rows plus about 1.5 rows (its two ring rows of the y pass and the three-row window
// prologue); the rows minimising waves x (rows + 1.5) give the shortest launch, the smallest
// such rows (the most items) winning ties.
inline int batch_rows(const int* bands, const int* ny, int n, int slots) {
  if (n <= 0 || slots <= 0) return 32;
  int nymax = 1;
  for (int s = 0; s < n; ++s) nymax = ny[s] > nymax ? ny[s] : nymax;
  int best = 4;
  double best_cost = 1e300;
  for (int r = 4; r <= (nymax > 4 ? nymax : 4); ++r) {
    long long items = 0;
    for (int s = 0; s < n; ++s) items += (long long)bands[s] * ((ny[s] + r - 1) / r);
    const long long waves = (items + slots - 1) / slots;
    const double cost = (double)waves * (r + 1.5);
    if (cost < best_cost) {
      best_cost = cost;
      best = r;
    }
  }
  return best;
}

}  // namespace hw
