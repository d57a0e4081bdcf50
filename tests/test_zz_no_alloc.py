"""The entry point that allocates nothing (hweno_stage_batch_static) against the existing
per-solve entry point (hweno_stage_device).

Callers that cannot allocate device memory -- applications whose device memory all comes from
a pool allocator of their own, and latency-critical loops that cannot afford cudaMalloc /
cudaFree -- run one batched stage of several solves with the work list in a static device
array of the library.  Two calls in a row (stage 1, then stage 2 on the first call's output)
must match hweno_stage_device on every solve within the parity tolerance of the tests (1e-12
of the component scale for FP64, 1e-5 for the FP32-bulk path), with the same wave speeds and
status words, and the second call must leave the device's free memory unchanged.  This file
is collected last so a failure here does not stop the other GPU tests; it also runs alone in
a fresh process (it creates every buffer it uses), and one test runs the entry point in a
process of its own where nothing else of the library has run.
"""
import numpy as np
import pytest

from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _setup(precision=H.HWENO_FP64):
    import torch
    dev = torch.device("cuda:0")
    sizes = [(40, 40, 1), (64, 48, 2), (100, 70, 3)]
    solves = []
    for nx, ny, seed in sizes:
        w = I.quadrant_vortex_2d(seed, 128, window=(10, 20, nx, ny))
        p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=nx, ny=ny, x0=w.x0, x1=w.x1,
                           y0=w.y0, y1=w.y1, bc=w.bc, precision=precision)
        U = torch.from_numpy(w.U0).to(dev)
        a = torch.zeros(2, dtype=torch.float64, device=dev)
        H.hweno_alpha_device(p, U, a, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        dt = torch.tensor([0.3 / (128.0 * float(a.sum()))], dtype=torch.float64, device=dev)
        solves.append(dict(p=p, U=U, a=a, dt=dt))
    return torch, dev, solves


def _scale(U):
    S = U[:, 0].abs().amax(dim=(1, 2)).reshape(-1, 1, 1, 1)
    return S


def _rel(x, ref, scale):
    return float(((x - ref).abs() / ref.abs().clamp_min(0).maximum(scale)).max())


def _per_solve(torch, solves, k, U_in, Vh):
    """Reference: hweno_stage_device, one launch per solve."""
    outs, vhs, aouts, sts = [], [], [], []
    st = torch.cuda.current_stream().cuda_stream
    for s, S in enumerate(solves):
        Uo = torch.full_like(S["U"], float("nan"))
        V = Vh[s].clone()
        ao = torch.zeros(2, dtype=torch.float64, device=S["U"].device)
        status = torch.zeros(1, dtype=torch.int32, device=S["U"].device)
        a_in = S["a"] if k == 1 else S["a_k"]
        H.hweno_stage_device(S["p"], k, U_in[s], S["U"], V, Uo, a_in, ao, S["dt"], status, st)
        outs.append(Uo)
        vhs.append(V)
        aouts.append(ao)
        sts.append(status)
    torch.cuda.synchronize()
    return outs, vhs, aouts, sts


def _static(torch, solves, k, U_in, Vh, memory=None):
    outs = [torch.full_like(S["U"], float("nan")) for S in solves]
    vhs = [v.clone() for v in Vh]
    aouts = [torch.zeros(2, dtype=torch.float64, device=S["U"].device) for S in solves]
    sts = [torch.zeros(1, dtype=torch.int32, device=S["U"].device) for S in solves]
    a_in = [S["a"] if k == 1 else S["a_k"] for S in solves]
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())
    H.hweno_stage_batch_static([S["p"] for S in solves], k, U_in, [S["U"] for S in solves], vhs,
                               outs, a_in, aouts, [S["dt"] for S in solves], sts,
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if memory is not None:
        memory.append((before, (torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved())))
    return outs, vhs, aouts, sts


@pytest.mark.parametrize("precision,tol", [(H.HWENO_FP64, TOL), (H.HWENO_MIXED32, 1e-5)])
def test_static_batch_matches_per_solve_entry_point_on_two_calls(precision, tol):
    """Both precision classes (FP32 bulk against its own per-solve launches: the parity bound
    of that path, 1e-5).  The second call allocates nothing: the device's free memory and
    PyTorch's reserved memory are the same before and after it."""
    torch, dev, solves = _setup(precision)
    Vh0 = [torch.zeros((4, 2, S["p"].ny, S["p"].nx), dtype=torch.float64, device=dev)
           for S in solves]
    # first call: stage 1 from U^n
    U_in = [S["U"] for S in solves]
    ref = _per_solve(torch, solves, 1, U_in, Vh0)
    got = _static(torch, solves, 1, U_in, Vh0)
    for s, S in enumerate(solves):
        sc = _scale(S["U"])
        assert _rel(got[0][s], ref[0][s], sc) <= tol
        assert _rel(got[1][s], ref[1][s], sc) <= tol      # v-hat^n, w-hat^n written by stage 1
        torch.testing.assert_close(got[2][s], ref[2][s], rtol=1e-13, atol=0)
        assert int(got[3][s].item()) == int(ref[3][s].item()) == 0
        S["a_k"] = got[2][s]
    # second call in a row: stage 2 on the first call's output (the scratch keeps the first
    # call's work list until this call rewrites it)
    U1 = got[0]
    Vh1 = got[1]
    ref2 = _per_solve(torch, solves, 2, U1, Vh1)
    memory = []
    got2 = _static(torch, solves, 2, U1, Vh1, memory)
    assert memory[0][0] == memory[0][1], memory          # no device allocation by the call
    for s, S in enumerate(solves):
        sc = _scale(S["U"])
        assert _rel(got2[0][s], ref2[0][s], sc) <= tol
        torch.testing.assert_close(got2[2][s], ref2[2][s], rtol=1e-13, atol=0)
        assert int(got2[3][s].item()) == int(ref2[3][s].item()) == 0


def test_static_batch_rejects_too_many_solves():
    torch, dev, solves = _setup()
    S = solves[0]
    n = H.HWENO_STATIC_BATCH_MAX + 1
    with pytest.raises(H.HwenoError) as ei:
        H.hweno_stage_batch_static([S["p"]] * n, 1, [S["U"]] * n, [S["U"]] * n, [S["U"]] * n,
                                   [S["U"]] * n, [S["a"]] * n, [S["a"]] * n, [S["dt"]] * n,
                                   [S["a"]] * n)
    assert ei.value.code == H.HWENO_ERR_ARG


def test_static_batch_rejects_buffers_shared_between_solves():
    """An output that is another solve's input (one launch reads and writes both) is refused."""
    torch, dev, solves = _setup()
    A, B = solves[0], solves[1]
    outs = [B["U"], torch.empty_like(B["U"])]          # solve 0 writes into solve 1's input
    Vh = [torch.zeros((4, 2, S["p"].ny, S["p"].nx), dtype=torch.float64, device=dev)
          for S in (A, B)]
    st = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(2)]
    with pytest.raises(H.HwenoError) as ei:
        H.hweno_stage_batch_static([A["p"], B["p"]], 1, [A["U"], B["U"]], [A["U"], B["U"]], Vh,
                                   outs, [A["a"], B["a"]], [A["a"].clone(), B["a"].clone()],
                                   [A["dt"], B["dt"]], st)
    assert ei.value.code == H.HWENO_ERR_ARG


ALONE = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
from paper_2402_03074_gb300 import _binding as H
from paper_2402_03074_gb300 import inputs as I
dev = torch.device("cuda:0")
w = I.quadrant_vortex_2d(1, 128, window=(10, 20, 48, 40))
p = H.make_problem(dim=2, equation=H.HWENO_EULER, nx=48, ny=40, x0=w.x0, x1=w.x1, y0=w.y0,
                   y1=w.y1, bc=w.bc)
U = torch.from_numpy(w.U0).to(dev)
Vh = torch.zeros((4, 2, 40, 48), dtype=torch.float64, device=dev)
Uo = torch.full_like(U, float("nan"))
a = torch.tensor([3.0, 3.0], dtype=torch.float64, device=dev)
ao = torch.zeros(2, dtype=torch.float64, device=dev)
dt = torch.tensor([1e-4], dtype=torch.float64, device=dev)
st = torch.zeros(1, dtype=torch.int32, device=dev)
H.hweno_stage_batch_static([p], 1, [U], [U], [Vh], [Uo], [a], [ao], [dt], [st])
torch.cuda.synchronize()
print(int(st.item()), bool(torch.isfinite(Uo).all().item()), float(ao.max().item()))
"""


def test_static_batch_runs_first_in_a_fresh_process():
    """The entry point used on its own, in a process where no other entry point of the library
    has run (nothing has raised the per-thread stack limit): the kernel's stack frame fits the
    CUDA default, so the call succeeds."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", ALONE, root], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    st, finite, amax = r.stdout.split()
    assert st == "0" and finite == "True" and float(amax) > 0.0
