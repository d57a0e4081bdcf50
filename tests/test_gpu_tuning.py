"""Autotuner and numeric helpers on the GPU."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_keeps_results_and_roundtrips(tmp_path):
    w = I.quadrant_vortex_2d(4, 256)
    p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=256, ny=256, x0=0, x1=1, y0=0, y1=1,
                       bc=w.bc)
    eng = H.hweno_create()
    try:
        sid = H.hweno_open(eng, p, w.U0)
        H.hweno_advance(eng, sid, 1.0, max_steps=3)
        ref, _ = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
        H.hweno_close(eng, sid)
        rows, bands, ms = H.hweno_autotune(eng, p, w.U0)
        assert rows in (0, 8, 16, 32, 64, 128, 256) and ms > 0
        # 256 columns: the widest bands are 2 (192-thread blocks), 3 (96 and 128 threads) or
        # 5 (64 threads)
        assert bands in (0, 3, 4, 5, 6, 7, 8, 10)
        tq = H.hweno_tuning_query(p)
        assert tq is not None and tq["width"] in (64, 96, 128, 192) and tq["lanes"] == 0
        sid = H.hweno_open(eng, p, w.U0)
        H.hweno_advance(eng, sid, 1.0, max_steps=3)
        got, _ = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    if tq["width"] == 96:
        # the default kernel's arithmetic: the tile decomposition does not change any bit
        np.testing.assert_array_equal(got, ref)
    else:
        # 64 / 128 / 192 threads form the coefficients from the projected stencil: equal within
        # rounding to the 96-thread kernel, which projects the conserved coefficients
        S = np.abs(ref[:, 0]).max(axis=(1, 2)).reshape(-1, 1, 1, 1)
        assert float((np.abs(got - ref) / np.maximum(np.abs(ref), S)).max()) <= 1e-13
    path = str(tmp_path / "tuning.txt")
    H.hweno_tuning_save(path)
    text = open(path).read()
    assert " 2 1 0 256 256 " in text
    assert H.hweno_tuning_load(path) >= 1


RCP_TEST = r"""
#include <cstdio>
#include <cmath>
#include <cstring>
#include "hweno_device.cuh"
__global__ void k(const double* x, double* a, double* b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { a[i] = hw::rcp_nr(x[i]); b[i] = 1.0 / x[i]; }
}
int main() {
  const int n = 1 << 20;
  double *x, *a, *b;
  cudaMallocManaged(&x, n * 8); cudaMallocManaged(&a, n * 8); cudaMallocManaged(&b, n * 8);
  unsigned long long s = 88172645463325252ULL;
  for (int i = 0; i < n; ++i) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    double m = 1.0 + (double)(s >> 11) / 9007199254740992.0;      // [1, 2)
    int e = (int)((s >> 3) % 2098) - 1074;                         // 2^-1074 .. 2^1023
    x[i] = ldexp(m, e) * ((s & 1) ? -1.0 : 1.0);
    if (i % 1024 == 0) x[i] = (i % 2048 == 0) ? 0.0 : INFINITY;    // division branch
    if (i % 1024 == 1) x[i] = ldexp(m, -1030);                     // subnormal
  }
  k<<<(n + 255) / 256, 256>>>(x, a, b, n);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
  long long maxulp = 0;
  for (int i = 0; i < n; ++i) {
    long long ua, ub; memcpy(&ua, &a[i], 8); memcpy(&ub, &b[i], 8);
    if ((ua < 0) != (ub < 0)) { maxulp = 1LL << 60; break; }     // sign mismatch
    long long d = ua > ub ? ua - ub : ub - ua;
    if (d > maxulp) maxulp = d;
  }
  printf("%lld\n", maxulp);
  return 0;
}
"""


def test_refined_reciprocal_within_one_ulp_of_division():
    """rcp_nr (the FP32 reciprocal of the significand refined by one third-order step, the
    exponent negated on the integer bits; the division for zeros, subnormals, infinities and
    the largest exponents) against CUDA's correctly rounded 1/x on 2^20 values over the whole
    double range 2^-1074 .. 2^1024, both signs."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "rcp.cu")
        open(src, "w").write(RCP_TEST)
        exe = os.path.join(d, "rcp")
        subprocess.run(["nvcc", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-I", os.path.join(ROOT, "paper_2402_03074_gb300", "csrc"), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    assert int(out.strip()) <= 1


CVT_TEST = r"""
#include <cstdio>
#include <cmath>
#include <cstring>
#include "hweno_device.cuh"
__global__ void k(const double* x, double* a, double* b, float* c, float* d, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float f = (float)x[i];
    a[i] = hw::f2d_bits(f);      b[i] = (double)f;
    c[i] = hw::d2f_bits(x[i]);   d[i] = f;
  }
}
int main() {
  const int n = 1 << 20;
  double *x, *a, *b; float *c, *d;
  cudaMallocManaged(&x, n * 8); cudaMallocManaged(&a, n * 8); cudaMallocManaged(&b, n * 8);
  cudaMallocManaged(&c, n * 4); cudaMallocManaged(&d, n * 4);
  unsigned long long s = 88172645463325252ULL;
  for (int i = 0; i < n; ++i) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    double m = 1.0 + (double)(s >> 11) / 9007199254740992.0;      // [1, 2)
    int e = (int)((s >> 3) % 240) - 120;                           // 2^-120 .. 2^119
    x[i] = ldexp(m, e) * ((s & 1) ? -1.0 : 1.0);
    if (i % 4096 == 0) x[i] = 0.0;
    if (i % 4096 == 1) x[i] = -0.0;
    if (i % 4096 == 2) x[i] = 1.0 + ldexp(1.0, -24);               // a tie
  }
  k<<<(n + 255) / 256, 256>>>(x, a, b, c, d, n);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
  long long bad = 0;
  for (int i = 0; i < n; ++i) {
    if (memcmp(&a[i], &b[i], 8) != 0) ++bad;
    if (memcmp(&c[i], &d[i], 4) != 0) ++bad;
  }
  printf("%lld\n", bad);
  return 0;
}
"""


def test_integer_bit_conversions_equal_the_hardware_conversions():
    """f2d_bits / d2f_bits (float <-> double on the integer pipe, used by the FP32-bulk path)
    against the hardware conversions, bit for bit, on 2^20 values over 2^-120 .. 2^119 (the
    normal float range), zeros of both signs and rounding ties."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "cvt.cu")
        open(src, "w").write(CVT_TEST)
        exe = os.path.join(d, "cvt")
        subprocess.run(["nvcc", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                        "-I", os.path.join(ROOT, "paper_2402_03074_gb300", "csrc"), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    assert int(out.strip()) == 0


# ------------------------------------------------------------------------------------------
# 1D Euler with the characteristic decomposition: one lane per characteristic field
def _tuning_file(tmp_path, entries):
    import torch
    name = torch.cuda.get_device_name(0).replace(" ", "_")
    path = str(tmp_path / "t1d.txt")
    with open(path, "w") as f:
        for (mixed, nx, width, lanes) in entries:
            f.write(f"{name} 2 1 {mixed} {nx} 1 0 0 {width} {lanes}\n")
    return path


@pytest.mark.parametrize("width", [32, 64, 128])
def test_fields_layout_1d_matches_oracle(tmp_path, width):
    """The lanes-per-field layout (selected through the tuning table) against the oracle at
    1e-12 for every stage, on grids of one block, one block +- 1 cell, several blocks with a
    ragged tail, and all boundary conditions."""
    from gpu_helpers import problems
    from test_gpu_parity import _check_stage
    cells = {32: 6, 64: 14, 128: 30}[width]
    sizes = [2, cells - 1, cells, cells + 1, 3 * cells + 5, 997]
    sizes = sorted({n for n in sizes if n >= 2})
    path = _tuning_file(tmp_path, [(0, n, width, 4) for n in sizes])
    assert H.hweno_tuning_load(path) == len(sizes)
    try:
        for n in sizes:
            for bc in (0, 1, 2):
                op, hp = problems(1, "euler", n, bc=bc, characteristic=1)
                for k in (1, 2, 3):
                    _check_stage(op, hp, k, seed=31 * k + n)
    finally:
        H.hweno_tuning_load(_tuning_file(tmp_path, [(0, n, 0, 0) for n in sizes]))


def test_autotune_1d_picks_a_layout_and_the_run_matches_oracle():
    """hweno_autotune on a 1D Euler shock tube (4000 cells): it times the one-thread-per-cell
    blocks and the lanes-per-field blocks, keeps the fastest, and a run in the kept layout
    matches the oracle."""
    w = I.shock_tube_1d(3, n=4000, t_end=0.05)
    hp = H.make_problem(dim=1, equation=H.HWENO_EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    eng = H.hweno_create()
    try:
        width, lanes, ms = H.hweno_autotune(eng, hp, w.U0)
        assert width in (32, 64, 128) and lanes in (1, 4) and ms > 0.0
        sid = H.hweno_open(eng, hp, w.U0)
        ns = H.hweno_advance(eng, sid, 1e9, max_steps=20)
        got, t = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    import oracle as O
    op = O.Problem(dim=1, eq=O.EULER, nx=w.nx, x0=w.x0, x1=w.x1, bc=w.bc)
    U, to, nso, st = O.run(op, w.U0, 0.0, 1e9, max_steps=20)
    assert ns == nso == 20 and st == 0 and t == pytest.approx(to, rel=1e-13)
    S = np.abs(w.U0[:, 0]).max(axis=(1, 2)).reshape(-1, 1, 1, 1)
    assert float((np.abs(got - U) / np.maximum(np.abs(U), S)).max()) <= 20e-12


# ------------------------------------------------------------------------------------------
# 2D block widths (64, 96, 128, 192 threads), selected through the tuning table
def _tuning_file_2d(tmp_path, entries):
    import torch
    name = torch.cuda.get_device_name(0).replace(" ", "_")
    path = str(tmp_path / "t2d.txt")
    with open(path, "w") as f:
        for (eq, ch, mixed, nx, ny, width) in entries:
            rows = bands = -1 if width else 0
            f.write(f"{name} {eq} {ch} {mixed} {nx} {ny} {rows} {bands} {width} 0\n")
    return path


@pytest.mark.parametrize("width", [64, 96, 128, 192])
def test_block_widths_2d_match_oracle(tmp_path, width):
    """Characteristic FP64 2D Euler in every block width against the oracle at 1e-12 for every
    stage (the 96-thread kernel projects the conserved coefficients formed once per cell, the
    others form the coefficients from the projected stencil), on grids of one band less one
    column, one band, one band plus one column and several bands with a ragged tail, every
    boundary condition.  Each case takes the first seed from 13 k + nx whose stage the oracle
    finds physical and well conditioned (physical_seed)."""
    from gpu_helpers import problems
    from test_gpu_parity import _check_stage, physical_seed
    wb = width - 2
    sizes = [(wb - 1, 5), (wb, 7), (wb + 1, 3), (3 * wb + 5, 11)]
    path = _tuning_file_2d(tmp_path, [(2, 1, 0, nx, ny, width) for nx, ny in sizes])
    assert H.hweno_tuning_load(path) == len(sizes)
    try:
        for nx, ny in sizes:
            for bc in (0, 1, 2):
                op, hp = problems(2, "euler", nx, ny, bc=bc, characteristic=1)
                for k in (1, 2, 3):
                    _check_stage(op, hp, k, seed=physical_seed(op, k, 13 * k + nx))
    finally:
        H.hweno_tuning_load(_tuning_file_2d(tmp_path, [(2, 1, 0, nx, ny, 0) for nx, ny in sizes]))


def test_block_widths_2d_same_bits_where_the_arithmetic_is_the_same(tmp_path):
    """The block width changes the decomposition, not the arithmetic, of the FP32-bulk kernel,
    the component-wise FP64 kernel and the characteristic FP64 kernel in 64, 128 and 192
    threads: their stage outputs are bitwise equal across widths."""
    from gpu_helpers import gpu_problems_stage
    nx, ny = 211, 17
    cases = [(1, 0), (0, 0), (1, 1)]   # (characteristic, mixed)
    for ch, mixed in cases:
        outs = {}
        for width in (64, 96, 128, 192):
            path = _tuning_file_2d(tmp_path, [(2, ch, mixed, nx, ny, width)])
            assert H.hweno_tuning_load(path) == 1
            try:
                outs[width] = gpu_problems_stage(nx, ny, ch, mixed, seed=3)
            finally:
                H.hweno_tuning_load(_tuning_file_2d(tmp_path, [(2, ch, mixed, nx, ny, 0)]))
        np.testing.assert_array_equal(outs[64], outs[128])
        np.testing.assert_array_equal(outs[192], outs[128])
        if not (ch == 1 and mixed == 0):   # the 96-thread FP64 characteristic kernel differs
            np.testing.assert_array_equal(outs[96], outs[128])


@pytest.mark.parametrize("seg", [7, 23, 37, 41, 150])
def test_segment_layout_matches_oracle_and_the_chunk_layout(tmp_path, seg):
    """The segment layout (tuning entry rows = -seg): the bands' rows taken one after another
    and cut into segments of `seg` band-rows, one per block, a segment that crosses the end of
    a band swept in two or more pieces (seg = 150 > the 4 x 37 band-rows: one block sweeps all
    four bands).  Characteristic FP64 2D Euler on 200 x 37 cells (4 bands of 50 columns):
    every stage against the oracle at 1e-12 for every boundary condition, and bitwise the
    default chunk layout (the decomposition changes no cell's arithmetic).  Seeds whose stage
    the oracle finds physical and well conditioned (physical_seed)."""
    import torch
    from gpu_helpers import gpu_problems_stage, problems
    from test_gpu_parity import _check_stage, physical_seed
    name = torch.cuda.get_device_name(0).replace(" ", "_")
    nx, ny = 200, 37
    ref = {ch: gpu_problems_stage(nx, ny, ch, 0, seed=5) for ch in (1, 0)}
    path = str(tmp_path / "seg.txt")
    with open(path, "w") as f:
        f.write(f"{name} 2 1 0 {nx} {ny} {-seg} 0 0 0\n{name} 2 0 0 {nx} {ny} {-seg} 0 0 0\n")
    assert H.hweno_tuning_load(path) == 2
    try:
        q = H.hweno_tuning_query(H.make_problem(dim=2, equation=H.HWENO_EULER, nx=nx, ny=ny,
                                                x1=1.0, y1=ny / nx))
        assert q["rows"] == -seg
        for ch in (1, 0):
            np.testing.assert_array_equal(gpu_problems_stage(nx, ny, ch, 0, seed=5), ref[ch])
        for bc in (0, 1, 2):
            op, hp = problems(2, "euler", nx, ny, bc=bc, characteristic=1)
            for k in (1, 2, 3):
                _check_stage(op, hp, k, seed=physical_seed(op, k, 29 * k + seg))
    finally:
        with open(path, "w") as f:
            f.write(f"{name} 2 1 0 {nx} {ny} 0 0 0 0\n{name} 2 0 0 {nx} {ny} 0 0 0 0\n")
        H.hweno_tuning_load(path)
