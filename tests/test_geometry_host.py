"""Host logic of the launch geometry (paper_2402_03074_gb300/csrc/geometry.h): the header is
plain C++, compiled here with g++ into a small driver, and checked for the properties the
launches rely on -- every column and row covered exactly once by items no wider than a
block allows, one wave of blocks for the single-solve launch, the lane-aware band choice,
and the batched rows choice against brute force over the wave model."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2402_03074_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "geometry.h"
int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'G') {
      int nx, ny, bw, slots, rf, bf, lane;
      if (std::scanf("%d %d %d %d %d %d %d", &nx, &ny, &bw, &slots, &rf, &bf, &lane) != 7) return 2;
      const hw::Geom2D g = hw::geom2d(nx, ny, bw, slots, rf, bf, lane != 0);
      std::printf("%d %d %d %d %d %d\n", g.bands, g.wout, g.chunks, g.rows, g.seg, g.blocks);
    } else if (op == 'R') {
      int slots, n;
      if (std::scanf("%d %d", &slots, &n) != 2) return 2;
      std::vector<int> b(n > 0 ? n : 1), y(n > 0 ? n : 1);
      for (int s = 0; s < n; ++s)
        if (std::scanf("%d %d", &b[s], &y[s]) != 2) return 2;
      std::printf("%d\n", hw::batch_rows(b.data(), y.data(), n, slots));
    } else if (op == 'L') {
      int nx, bands;
      if (std::scanf("%d %d", &nx, &bands) != 2) return 2;
      std::printf("%d\n", hw::band_lanes(nx, bands));
    } else {
      return 3;
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def geo(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("geometry")
    src, exe = d / "driver.cc", d / "driver"
    src.write_text(DRIVER)
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)

    def run(lines):
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                           text=True, check=True)
        return [list(map(int, ln.split())) for ln in r.stdout.strip().splitlines()]
    return run


def _waves_cost(bands, nys, slots, r):
    items = sum(b * math.ceil(y / r) for b, y in zip(bands, nys))
    return math.ceil(items / slots) * (r + 1.5), items


def test_single_solve_covers_the_grid_in_one_wave(geo):
    rng = np.random.default_rng(7)
    cases = []
    for _ in range(300):
        nx, ny = (int(v) for v in rng.integers(1, 5000, size=2))
        slots = int(rng.choice([152, 304, 456, 608]))
        bw = int(rng.choice([64, 96, 128, 192]))
        cases.append((nx, ny, bw, slots, 0, 0, int(rng.integers(0, 2))))
    cases += [(1, 1, 128, 304, 0, 0, 1), (2, 3, 128, 304, 0, 0, 0), (126, 1, 128, 304, 0, 0, 0),
              (127, 2, 128, 304, 0, 0, 1), (4096, 4096, 128, 304, 0, 0, 1)]
    out = geo(["G " + " ".join(map(str, c)) for c in cases])
    nseg = 0
    for (nx, ny, bw, slots, _, _, lane), (bands, wout, chunks, rows, seg, blocks) in zip(cases, out):
        assert 1 <= wout <= bw - 2
        assert bands * wout >= nx and (bands - 1) * wout < nx    # every column, no empty band
        assert rows * chunks >= ny and (chunks - 1) * rows < ny  # every row, no empty chunk
        if seg == 0:
            assert blocks == bands * chunks
        else:                                                     # every band-row, no empty block
            nseg += 1
            assert blocks * seg >= bands * ny and (blocks - 1) * seg < bands * ny
            # chosen only where it is 2 % cheaper: pieces of seg rows + 1.5 against chunks
            pieces = 1 + math.ceil((seg - 1) / ny)
            assert seg + 1.5 * pieces < 0.98 * (rows + 1.5)
        if bands <= slots:
            assert blocks <= slots                               # one wave of blocks
        if not lane:
            assert bands <= math.ceil(nx / (bw - 2)) and wout >= min(nx, bw - 2) // 2
    assert nseg > 0


def test_lane_aware_bands(geo):
    # 2048 columns: 22 bands of 94 columns (96 lanes each) rather than 17 of 121 (128 lanes)
    (l22,), (l17,) = geo(["L 2048 22", "L 2048 17"])
    assert (l22, l17) == (22 * 96, 17 * 128)
    out = geo(["G 2048 2048 128 304 0 0 1", "G 2048 2048 128 304 0 0 0",
               "G 1024 1024 128 304 0 0 1", "G 1024 1024 128 304 0 0 0"])
    assert out[0][:2] == [22, 94] and out[1][:2] == [17, 121]
    assert out[2][:2] == [11, 94] and out[3][:2] == [9, 114]
    # one wave on 304 slots: 22 bands of 2048 rows in 303 segments of 149 band-rows (22 x 13 =
    # 286 chunks of 158 rows would leave 18 slots empty); 11 x 27 = 297 chunks of 38 rows
    assert out[0][4:] == [149, 303] and out[0][0] * out[0][2] == 286
    assert out[2][4:] == [0, 297] and out[2][0] * out[2][2] == 297
    # FP32-bulk 2048^2 in 192-thread blocks, two per SM: 11 bands of 187 columns (189 of the 192
    # lanes) in 27 chunks of 76 rows (segments of 75 band-rows in up to two pieces would not be
    # 2 % cheaper)
    (g192,) = geo(["G 2048 2048 192 304 0 0 0"])
    assert g192 == [11, 187, 27, 76, 0, 297]
    # the lane-aware choice is taken only when it saves lanes
    rng = np.random.default_rng(3)
    nxs = [int(v) for v in rng.integers(1, 6000, size=200)]
    lanes_aw = geo([f"G {n} 64 128 304 0 0 1" for n in nxs])
    lanes_pl = geo([f"G {n} 64 128 304 0 0 0" for n in nxs])
    q = []
    for n, a, p in zip(nxs, lanes_aw, lanes_pl):
        q += [f"L {n} {a[0]}", f"L {n} {p[0]}"]
    lz = geo(q)
    for k in range(len(nxs)):
        assert lz[2 * k][0] <= lz[2 * k + 1][0]


def test_fixed_tile_shapes(geo):
    out = geo(["G 2048 2048 128 304 32 0 1",    # rows fixed
               "G 2048 2048 128 304 0 4 1",     # too few bands: raised to the 126-column bound
               "G 2048 2048 128 304 0 40 0",    # more bands than the default
               "G 100 50 128 304 500 0 0",      # rows above ny: one chunk
               "G 300 37 96 304 -7 0 1",        # segments of 7 band-rows
               "G 300 37 96 304 -100000 0 1"])  # a segment longer than all bands: one block
    assert out[0][3] == 32 and out[0][2] == 64 and out[0][4] == 0
    assert out[1][0] == 17 and out[1][1] == 121
    assert out[2][0] == 40 and out[2][1] == 52
    assert out[3][2:4] == [1, 50] and out[3][4] == 0
    assert out[4][0] == 5 and out[4][4:] == [7, math.ceil(5 * 37 / 7)]   # 5 bands of 60
    assert out[5][4:] == [5 * 37, 1]


def test_batched_rows_minimise_the_waves(geo):
    rng = np.random.default_rng(11)
    classes = [([11], [1024], 304), ([9], [1024], 456), ([11, 9, 6], [1024, 768, 512], 304),
               ([3, 5], [256, 384], 304), ([2], [128], 304), ([22], [2048], 304),
               ([1], [2], 304), ([1], [4], 304)]
    for _ in range(60):
        m = int(rng.integers(1, 12))
        nys = [int(v) for v in rng.choice([64, 128, 256, 384, 512, 768, 1024], size=m)]
        bands = [math.ceil(y / 94) for y in nys]
        classes.append((bands, nys, int(rng.choice([152, 304, 456]))))
    lines = ["R %d %d %s" % (slots, len(b), " ".join(f"{x} {y}" for x, y in zip(b, ny)))
             for b, ny, slots in classes]
    got = [r[0] for r in geo(lines)]
    for (bands, nys, slots), r in zip(classes, got):
        assert 4 <= r <= max(4, max(nys))
        cost, items = _waves_cost(bands, nys, slots, r)
        brute = min(_waves_cost(bands, nys, slots, q)[0] for q in range(4, max(4, max(nys)) + 1))
        assert cost == brute
        # the smallest rows of least cost (the most items)
        assert all(_waves_cost(bands, nys, slots, q)[0] > cost for q in range(4, r))
    # a lone 1024^2 FP64 solve: 38 rows, 297 items in one wave (37 rows would need 308)
    assert got[0] == 38 and _waves_cost([11], [1024], 304, 38)[1] == 297
    # degenerate inputs
    assert geo(["R 304 0", "R 0 1 3 100"]) == [[32], [32]]
