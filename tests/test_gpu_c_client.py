"""The C ABI used from plain C: a small C program (compiled with gcc against include/hweno.h
and linked with libhweno.so) reads initial moments from a file, advances them with
hweno_open / hweno_advance, serves a second copy through hweno_submit / hweno_serve /
hweno_poll, and writes both results; the test checks them against the FP64 oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_CLIENT = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "hweno.h"

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  const int n = atoi(argv[1]);
  const double t_end = atof(argv[2]);
  hweno_problem p;
  memset(&p, 0, sizeof p);
  p.dim = 2; p.equation = HWENO_EULER; p.nx = n; p.ny = n;
  p.x0 = 0.0; p.x1 = 1.0; p.y0 = 0.0; p.y1 = 1.0; p.ax = 1.0; p.ay = 1.0; p.gamma = 1.4;
  for (int s = 0; s < 4; ++s) p.bc[s] = HWENO_BC_TRANSMISSIVE;
  p.cfl = 0.6; p.t_end = t_end; p.precision = HWENO_FP64; p.characteristic = 1;
  p.weights = HWENO_W_SCALE_INVARIANT; p.gamma_lo = 1.0 / 400.0; p.eps = 1e-10;
  const size_t count = (size_t)hweno_ncomp(&p) * hweno_nmom(&p) * n * n;
  double* u = malloc(sizeof(double) * count);
  double* v = malloc(sizeof(double) * count);
  FILE* f = fopen(argv[3], "rb");
  if (!f || fread(u, sizeof(double), count, f) != count) return 3;
  fclose(f);
  hweno_engine* eng = NULL;
  if (hweno_create(NULL, &eng) != HWENO_OK) return 4;
  uint64_t id = 0, ticket = 0;
  int64_t steps = 0;
  double t = 0.0;
  if (hweno_open(eng, &p, u, &id) != HWENO_OK) return 5;
  if (hweno_advance(eng, id, t_end, -1, &steps) != HWENO_OK) return 6;
  if (hweno_get_state(eng, id, v, &t) != HWENO_OK) return 7;
  hweno_close(eng, id);
  if (hweno_submit(eng, &p, u, &ticket) != HWENO_OK) return 8;
  hweno_result info;
  int rc = HWENO_PENDING, active = 0;
  for (int it = 0; it < 1000000 && rc == HWENO_PENDING; ++it) {
    if (hweno_serve(eng, 8, &active) != HWENO_OK) return 9;
    rc = hweno_poll(eng, ticket, u, &info);
  }
  if (rc != HWENO_OK) return 10;
  hweno_destroy(eng);
  f = fopen(argv[4], "wb");
  fwrite(v, sizeof(double), count, f);
  fwrite(u, sizeof(double), count, f);
  fclose(f);
  printf("%lld %.17g %lld %.17g\n", (long long)steps, t, (long long)info.steps, info.t);
  free(u);
  free(v);
  return 0;
}
"""


def test_c_program_uses_the_abi(tmp_path):
    from paper_2402_03074_gb300 import build as B
    lib = B.build()
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    n, T = 48, 0.02
    w = I.quadrant_vortex_2d(12, n)
    inp, outp = tmp_path / "in.bin", tmp_path / "out.bin"
    w.U0.astype(np.float64).tofile(inp)
    r = subprocess.run([str(exe), str(n), repr(T), str(inp), str(outp)], capture_output=True,
                       text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    steps, t, steps_s, t_s = r.stdout.split()
    res = np.fromfile(outp).reshape((2,) + w.U0.shape)
    op = O.Problem(dim=2, eq=O.EULER, nx=n, ny=n, x0=w.x0, x1=w.x1, y0=w.y0, y1=w.y1, bc=w.bc)
    ref, tr, ns, st = O.run(op, w.U0, 0.0, T)
    assert int(steps) == int(steps_s) == ns and float(t) == float(t_s) == tr == T
    S = np.abs(w.U0[:, 0]).max(axis=(1, 2))[:, None, None, None]
    for out in res:
        err = (np.abs(out - ref) / np.maximum(np.abs(ref), S)).max()
        assert err <= 1e-12 * ns, err
