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
        assert bands in (0, 4, 5, 6)            # 256 columns: 3 bands at the widest
        sid = H.hweno_open(eng, p, w.U0)
        H.hweno_advance(eng, sid, 1.0, max_steps=3)
        got, _ = H.hweno_get_state(eng, sid, np.empty_like(w.U0))
    finally:
        H.hweno_destroy(eng)
    np.testing.assert_array_equal(got, ref)   # the decomposition does not change any bit
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
    int e = (int)((s >> 3) % 400) - 200;                           // 2^-200 .. 2^199
    x[i] = ldexp(m, e) * ((s & 1) ? -1.0 : 1.0);
  }
  k<<<(n + 255) / 256, 256>>>(x, a, b, n);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("cuda error\n"); return 2; }
  long long maxulp = 0;
  for (int i = 0; i < n; ++i) {
    long long ua, ub; memcpy(&ua, &a[i], 8); memcpy(&ub, &b[i], 8);
    long long d = ua > ub ? ua - ub : ub - ua;
    if (d > maxulp) maxulp = d;
  }
  printf("%lld\n", maxulp);
  return 0;
}
"""


def test_refined_reciprocal_within_one_ulp_of_division():
    """rcp_nr (the FP32 reciprocal refined by one third-order step) against CUDA's
    correctly rounded 1/x on 2^20 values over 2^-200 .. 2^200, both signs."""
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
