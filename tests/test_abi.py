"""CPU-side checks of the C ABI library: it loads, exports every function include/hweno.h
declares, validates problems on the host, and refuses to run without a GPU (no fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    from paper_2402_03074_gb300 import build as B
    B.build()
    from paper_2402_03074_gb300 import _binding
    return _binding


def declared_functions():
    src = open(os.path.join(ROOT, "include", "hweno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hweno_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(H):
    lib = ctypes.CDLL(H.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi(H):
    for n in declared_functions():
        assert hasattr(H, n), n


def test_problem_validation_on_host(H):
    ok = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=8, ny=8)
    assert H.hweno_ncomp(ok) == 4 and H.hweno_nmom(ok) == 3
    assert H.hweno_ncomp(H.make_problem(dim=1, equation=H.HWENO_EULER, nx=8)) == 3
    assert H.hweno_nmom(H.make_problem(dim=1, equation=H.HWENO_BURGERS, nx=8)) == 2
    bad = [
        H.make_problem(dim=3),
        H.make_problem(dim=2, nx=8, ny=4, x1=1.0, y1=1.0),            # dx != dy
        H.make_problem(dim=2, nx=8, eps=0.0),
        H.make_problem(dim=2, nx=8, gamma_lo=0.3),                      # gamma_0 <= 0
        H.make_problem(dim=2, nx=8, bc=(0, 1, 0, 0)),                   # half-periodic
        H.make_problem(dim=1, nx=1),
        H.make_problem(dim=2, nx=8, precision=7),
        H.make_problem(dim=2, nx=8, cfl=0.0, dt_fixed=0.0),
        H.make_problem(dim=2, equation=H.HWENO_EULER, nx=8, gamma=1.0),
    ]
    for p in bad:
        assert H.hweno_ncomp(p) == 0


def test_create_without_gpu_fails_loudly(H):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(H.HwenoError) as ei:
        H.hweno_create()
    assert ei.value.code == H.HWENO_ERR_CUDA


def test_tuning_table_load_query_and_save_on_the_host(H, tmp_path):
    """The tuning table is host state: entries of this device (no GPU here: the name is
    "unknown") load, a single-solve problem finds its entry through hweno_tuning_query, other
    problems find none, entries of other devices are skipped, and a save writes them back."""
    path = str(tmp_path / "t.txt")
    with open(path, "w") as f:
        f.write("# comment\n")
        f.write("unknown 2 1 0 640 480 32 9 96 0\n")       # 2D Euler characteristic FP64
        f.write("unknown 0 0 0 200 1 0 0 32 1\n")          # 1D advection
        f.write("Some_Other_GPU 2 1 0 640 480 8 8 64 0\n")  # another device: skipped
    assert H.hweno_tuning_load(path) == 2
    p2 = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=640, ny=480, x1=4.0 / 3.0)
    assert H.hweno_tuning_query(p2) == {"rows": 32, "bands": 9, "width": 96, "lanes": 0}
    p1 = H.make_problem(dim=1, equation=H.HWENO_ADVECTION, nx=200)
    assert H.hweno_tuning_query(p1) == {"rows": 0, "bands": 0, "width": 32, "lanes": 1}
    assert H.hweno_tuning_query(H.make_problem(dim=2, equation=H.HWENO_EULER, nx=64)) is None
    out = str(tmp_path / "saved.txt")
    H.hweno_tuning_save(out)
    lines = [ln for ln in open(out) if not ln.startswith("#")]
    assert "unknown 2 1 0 640 480 32 9 96 0\n" in lines
    assert "unknown 0 0 0 200 1 0 0 32 1\n" in lines
    # clear the entries again (all zero = not tuned)
    with open(path, "w") as f:
        f.write("unknown 2 1 0 640 480 0 0 0 0\nunknown 0 0 0 200 1 0 0 0 0\n")
    assert H.hweno_tuning_load(path) == 2
    assert H.hweno_tuning_query(p2) is None and H.hweno_tuning_query(p1) is None
