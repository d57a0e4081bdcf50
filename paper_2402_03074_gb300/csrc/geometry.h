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

// Single-solve launch: bands as above (or fixed, but never wider than bw - 2 columns), swept
// by one wave of blocks in one of two layouts:
//  * chunks: row chunks sized so that bands x chunks fills the `slots` resident blocks once
//    (or fixed rows); a block sweeps one chunk of one band;
//  * segments (seg > 0): the bands' rows taken one after another (band-row q = band ny + row)
//    and cut into `blocks` equal segments of seg band-rows, one per block; a segment that
//    crosses the end of a band is swept as two (or more) pieces.  When the band count does not
//    divide the slots, chunks leave slots empty (2048^2 in 94-column bands: 22 x 13 = 286 of
//    304), while segments fill them (303 blocks of 149 band-rows instead of 158 rows).
// Fixed rows > 0 give chunks of that height, fixed rows < -1 segments of -rows band-rows; the
// default (0) takes segments where they cost at least 2 % less than chunks, a piece costing
// its rows plus about 1.5 rows (its two ring rows of the y pass and the window prologue)
// (2048^2 FP64: 29.05 ms instead of 29.65 ms per stage; a 0.6 % estimate, as for the
// FP32-bulk kernel's 17 bands on 456 slots, measured nothing).
struct Geom2D {
  int bands, wout, chunks, rows;
  int seg;     // > 0: segment layout, band-rows per block
  int blocks;  // blocks of the launch (bands x chunks, or the segments)
};
inline Geom2D geom2d(int nx, int ny, int bw, int slots, int rows_fixed, int bands_fixed,
                     bool lane_aware) {
  Geom2D g;
  const int bwide = (nx + (bw - 2) - 1) / (bw - 2);
  int b = bands_fixed > 0 ? (bands_fixed < nx ? bands_fixed : nx) : default_bands(nx, bw, lane_aware);
  if (bands_fixed > 0 && b < bwide) b = bwide;  // a band is at most bw - 2 columns wide
  split_bands(nx, b, &g.bands, &g.wout);
  g.seg = 0;
  if (rows_fixed > 0) {
    g.rows = rows_fixed < ny ? rows_fixed : ny;
  } else {
    int ch = slots / g.bands;
    if (ch < 1) ch = 1;
    if (ch > ny) ch = ny;
    g.rows = (ny + ch - 1) / ch;
  }
  g.chunks = (ny + g.rows - 1) / g.rows;
  g.blocks = g.bands * g.chunks;
  const long long total = (long long)g.bands * ny;
  long long seg = 0;
  if (rows_fixed < -1) {
    seg = -(long long)rows_fixed;
  } else if (rows_fixed == 0 && slots > 0 && g.bands <= slots) {
    const long long s = (total + slots - 1) / slots;
    const long long pieces = 1 + (s - 1 + ny - 1) / ny;   // most pieces a segment can have
    if ((double)s + 1.5 * (double)pieces < 0.98 * ((double)g.rows + 1.5)) seg = s;
  }
  if (seg > 0) {
    if (seg > total) seg = total;
    g.seg = (int)seg;
    g.blocks = (int)((total + seg - 1) / seg);
  }
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
