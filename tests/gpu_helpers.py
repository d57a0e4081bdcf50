"""Helpers shared by the GPU tests: run one stage through the C ABI on torch buffers and
compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2402_03074_gb300 import _binding as H

EQ = {"adv": (O.ADVECTION, H.HWENO_ADVECTION), "burg": (O.BURGERS, H.HWENO_BURGERS),
      "euler": (O.EULER, H.HWENO_EULER)}


def problems(dim, eq, nx, ny=1, bc=0, characteristic=1, precision=0, L=None, weights=0):
    """Matching oracle and library problem descriptions (square cells in 2D)."""
    oeq, heq = EQ[eq]
    x1 = float(nx) / 64.0 if L is None else L
    y1 = x1 * ny / nx if dim == 2 else 1.0
    bcs = (bc,) * 4 if isinstance(bc, int) else tuple(bc)
    op = O.Problem(dim=dim, eq=oeq, nx=nx, ny=ny if dim == 2 else 1, x0=0.0, x1=x1, y0=0.0,
                   y1=y1, ax=1.0, ay=-0.7, bc=bcs, characteristic=characteristic, weights=weights)
    hp = H.make_problem(dim=dim, equation=heq, nx=nx, ny=ny if dim == 2 else 1, x0=0.0, x1=x1,
                        y0=0.0, y1=y1, ax=1.0, ay=-0.7, bc=bcs, characteristic=characteristic,
                        precision=precision, weights=weights)
    return op, hp


def gpu_stage(hp, k, Uin, Un, Vh, alpha, dt, device="cuda:0"):
    """One stage through hweno_stage_device; returns (Uout, Vh, alpha_out, status)."""
    import torch
    dev = torch.device(device)
    Ui = torch.from_numpy(np.ascontiguousarray(Uin)).to(dev)
    Unn = Ui if Un is Uin else torch.from_numpy(np.ascontiguousarray(Un)).to(dev)
    Vt = torch.from_numpy(np.ascontiguousarray(Vh)).to(dev)
    Uo = torch.full_like(Ui, float("nan"))
    a_in = torch.tensor(np.asarray(alpha, dtype=np.float64), device=dev)
    a_out = torch.zeros(2, dtype=torch.float64, device=dev)
    dtt = torch.tensor([dt], dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    H.hweno_stage_device(hp, k, Ui, Unn, Vt, Uo, a_in, a_out, dtt, st,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return Uo.cpu().numpy(), Vt.cpu().numpy(), a_out.cpu().numpy(), int(st.item())


def rel_err(got, ref, U_scale):
    """max |g - o| / max(|o|, S_c), S_c = max |average of component c| (per component)."""
    S = np.abs(U_scale[:, 0]).max(axis=(1, 2))
    S = S.reshape((-1,) + (1,) * (ref.ndim - 1))
    return float((np.abs(got - ref) / np.maximum(np.abs(ref), S)).max())


def gpu_problems_stage(nx, ny, characteristic, mixed, seed, k=2):
    """Stage k of 2D Euler on seeded smooth-plus-noise data (transmissive) through
    hweno_stage_device; returns the output moments."""
    rng = np.random.default_rng(seed)
    op, hp = problems(2, "euler", nx, ny, bc=1, characteristic=characteristic,
                      precision=H.HWENO_MIXED32 if mixed else H.HWENO_FP64)
    U = np.zeros((4, 3, ny, nx))
    U[0, 0] = 1.0 + 0.2 * rng.random((ny, nx))
    U[1, 0] = 0.3 * rng.standard_normal((ny, nx))
    U[2, 0] = 0.3 * rng.standard_normal((ny, nx))
    U[3, 0] = 2.5 + 0.5 * rng.random((ny, nx))
    U[:, 1:] = 0.01 * rng.standard_normal((4, 2, ny, nx))
    Un = U + 1e-3 * rng.standard_normal(U.shape)
    Vh = 0.01 * rng.standard_normal((4, 2, ny, nx))
    out, _, _, _ = gpu_stage(hp, k, U, Un, Vh, (2.0, 2.0), 1e-3)
    return out
