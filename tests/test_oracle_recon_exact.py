"""Pins of the oracle's whole reconstruction (Steps 1-3 and the reconstruction formula of
Sec. 2.1 / 2.2) against exact rational values computed from the definitions.

tests/golden/recon_exact.json is written by tests/golden/make_recon_exact.py, which imports
nothing from the oracle: it solves the moment conditions of Eq. 2.5 / 2.17 exactly (a KKT
system for the 2D least-squares reading), integrates the smoothness indicators from their
definitions Eq. 2.8 / 2.19 (not the closed forms Eq. 2.9 / 2.20 the oracle uses), forms tau,
u_ave and the weights of Eq. 2.10-2.11 / 2.21-2.22 with epsilon = 1e-10 as a rational, and
evaluates the combined polynomial (Eq. 2.12 / 2.23) at the Gauss(-Lobatto) points exactly.

The 2D stencils are chosen so that the plausible slips in Step 3 fail here:
  * "corner" (only cell 1 non-zero): u_ave over cells 2, 4, 5, 6, 8 is 0, so omega = gamma;
    an u_ave over all nine cells gives omega_0 ~ 1e-9 instead;
  * "ridge", "step in x / y", "generic": tau's divisor (4) and the square in u_ave each move
    omega by O(1) relative; "step in x" vs "step in y" tell the x and y labels (v vs w,
    S_1..S_4) apart;
  * "zero averages": omega = gamma exactly (u_ave = 0), v-hat / w-hat from p_0 alone.
The 1D stencils include six hand-worked cases (linear, quadratic, step, zero averages, the
step scaled by 2^-20, the step with the original weights), whose 16-digit values are also
checked here against the script's exact results.
"""
import json
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "recon_exact.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _fr(s):
    a, b = s.split("/")
    return float(int(a)) / float(int(b)) if b != "1" else float(int(a))


def _close(o, g, rel, floor, what):
    o, g = np.asarray(o, dtype=np.float64), np.asarray(g, dtype=np.float64)
    err = np.abs(o - g)
    bound = rel * np.abs(g) + floor
    assert (err <= bound).all(), (what, o, g, err / np.maximum(np.abs(g), 1e-300))


def test_golden_file_is_the_scripts_output():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_recon_exact", os.path.join(HERE, "golden", "make_recon_exact.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    g = _golden()
    for case, (name, ub, vb, orig) in zip(g["recon1d"], mod.cases_1d()):
        assert case["name"] == name
        r = mod.recon_1d(ub, vb, orig)
        for k, v in r.items():
            assert case[k] == v, (name, k)
    for case, (name, ub, vb, wb, orig) in zip(g["recon2d"], mod.cases_2d()):
        assert case["name"] == name
        r = mod.recon_2d(ub, vb, wb, orig)
        for k, v in r.items():
            assert case[k] == v, (name, k)


def _check(o, g, scale):
    _close(o["c0"], g["c0"], 1e-14, 1e-15 * scale, "c0")
    _close(o["beta"], g["beta"], 1e-13, 1e-15 * scale * scale, "beta")
    _close(o["tau"], g["tau"], 1e-12, 1e-15 * scale ** 4, "tau")
    _close(o["uave"], g["uave"], 1e-14, 1e-300, "uave")
    _close(o["omega"], g["omega"], 1e-12, 1e-300, "omega")
    _close(o["pts"], g["pts"], 1e-12, 1e-16 * scale, "pts")
    _close(o["vhat"], g["vhat"], 1e-12, 1e-16 * scale, "vhat")


@pytest.mark.parametrize("idx", range(7))
def test_recon1d_matches_exact_values(idx):
    g = _golden()["recon1d"][idx]
    ub = [_fr(x) for x in g["ub"]]
    vb = [_fr(x) for x in g["vb"]]
    wm = O.W_ORIGINAL if g["original"] else O.W_SCALE_INVARIANT
    o = O.recon1d(ub, vb, weights=wm)
    _check(o, g, max(1e-300, max(abs(x) for x in ub + vb)))


@pytest.mark.parametrize("idx", range(8))
def test_recon2d_matches_exact_values(idx):
    g = _golden()["recon2d"][idx]
    ub = [_fr(x) for x in g["ub"]]
    vb = [_fr(x) for x in g["vb"]]
    wb = [_fr(x) for x in g["wb"]]
    wm = O.W_ORIGINAL if g["original"] else O.W_SCALE_INVARIANT
    o = O.recon2d(ub, vb, wb, weights=wm)
    _check(o, g, max(abs(x) for x in ub + vb + wb))
    _close(o["what"], g["what"], 1e-12, 1e-16 * max(abs(x) for x in ub + vb + wb), "what")


# Hand-worked values (exact rational arithmetic on Eq. 2.9 with the corrected first term and
# Eq. 2.10-2.12, gamma = (0.995, 1/400, 1/400), epsilon = 1e-10), rounded to 16 digits.
HAND_1D = {
    "linear u = xi": dict(beta=[1, 1, 1], tau=0.0, omega=[0.995, 0.0025, 0.0025],
                          ends=[-0.5, 0.5], vhat=1.0 / 12.0),
    "quadratic u = xi^2": dict(beta=[4.333333333333333, 1, 1], tau=11.11111111111111,
                               uave=0.5625,
                               omega=[0.9815835159303118, 0.009208242034844102,
                                      0.009208242034844102],
                               ends=[0.2477526827353956, 0.2477526827353956], vhat=0.0,
                               interior=0.05044946345292089),
    "step": dict(beta=[252.9347690772985, 0, 1], tau=63723.31263910903, uave=1.0 / 9.0,
                 omega=[1.416799980709750e-09, 0.9999999976831985, 9.000015663892666e-10],
                 ends=[-6.949087054529991e-10, 1.288208529870818e-09],
                 vhat=1.683824002651487e-10),
    "zero averages": dict(beta=[35397.32142857143, 0, 0], uave=0.0,
                          omega=[0.995, 0.0025, 0.0025], ends=[1.5, 1.5], vhat=0.0),
    "step scaled by 2^-20": dict(omega=[0.995, 0.0025, 0.0025],
                                 ends=[-1.652198925352933e-07, 5.625841910378975e-07],
                                 vhat=6.274173134251644e-08),
    "step, original weights": dict(omega=[1.579773983486057e-10, 0.999999999742021,
                                          1.000015692485946e-10]),
}


def test_exact_script_reproduces_the_hand_worked_values():
    """Two independent derivations of the same quantities: the hand-worked 16-digit values
    and the script's exact rationals agree to 1e-15 relative."""
    by_name = {c["name"]: c for c in _golden()["recon1d"]}
    for name, h in HAND_1D.items():
        g = by_name[name]
        rel = lambda a, b: abs(a - b) <= 1e-15 * abs(b) + 1e-300
        for k in ("beta", "omega"):
            if k in h:
                assert all(rel(a, b) for a, b in zip(g[k], h[k])), (name, k)
        for k in ("tau", "uave", "vhat"):
            if k in h:
                assert rel(g[k], h[k]), (name, k)
        if "ends" in h:
            assert rel(g["pts"][0], h["ends"][0]) and rel(g["pts"][3], h["ends"][1]), name
        if "interior" in h:
            assert rel(g["pts"][1], h["interior"]) and rel(g["pts"][2], h["interior"]), name
