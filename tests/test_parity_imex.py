"""Parity of the CUDA library's first-order semi-implicit scheme (Sec. 3.3,
Eq. ImpSchemeDD) with the oracle's, in the stiff regime dt/tau0 > 5 where the
explicit scheme is unstable.  GPU only.

Tolerances: FP64 state within 1e-12 of the largest value; FP32 moments within
1e-5 (relative per field; velocities relative to max(|u|, 1)).
"""
import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def moments_err(cfg, Fo, s):
    mo = oracle.moments(cfg, Fo)
    mg = s.moments()
    live = mo["rho"] > 0
    errs = {}
    keys = ("rho", "ux", "uy", "uz", "T") if cfg.get("dim", 2) == 3 else ("rho", "ux", "uy", "T")
    for k in keys:
        ref = mo[k][live]
        scale = np.abs(ref).max()
        if k.startswith("u"):
            scale = max(scale, 1.0)
        errs[k] = np.abs(mg[k][live] - ref).max() / scale
    return errs


def run_pair(cfg, steps, prec):
    F0 = oracle.initial_state(cfg)
    s = dvm.Solver(cfg, prec)
    assert s.dt / s.tau0 > 5          # stiff: the explicit scheme would need dt < tau
    s.set_state(F0)
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, steps)
    assert h["status"] == 0
    s.step(steps)
    return s, Fo, h


def check(cfg, s, Fo, prec):
    if prec == dvm.FP64:
        Fg = s.get_state()
        assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < (1e-12 if prec == dvm.FP64 else 1e-5), errs


def stiff(cfg, Kn=1e-3):
    cfg = dict(cfg)
    cfg.update(Kn=Kn, time_scheme=1)
    return cfg


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_imex_cylinder(prec):
    """Fixed cylinder, MUSCL, Mach 2: cut cells, merged control volumes, the
    diffuse wall and Maxwellian / zero-gradient sides."""
    cfg = stiff(W.cylinder_mach2(nx=48, nv=16))
    s, Fo, h = run_pair(cfg, 20, prec)
    check(cfg, s, Fo, prec)
    hg = s.history(20)["Fx"]
    tol = 1e-10 if prec == dvm.FP64 else 1e-4
    assert np.abs(hg - h["Fx"]).max() <= tol * np.abs(h["Fx"]).max()
    s.close()


def test_imex_moving_ellipse_fp64():
    """Rotating ellipse: geometry rebuilt each step, appearing and vanishing
    cells, area ratios S^n/S^{n+1}; the body's angle follows the oracle's."""
    cfg = stiff(W.rotating_ellipse(nx=64, nv=12, scheme=1), Kn=5e-4)
    s, Fo, h = run_pair(cfg, 15, dvm.FP64)
    check(cfg, s, Fo, dvm.FP64)
    th, om = s.body_state()
    assert abs(th - h["theta"]) <= 1e-12 and abs(om - h["omega"]) <= 1e-10 * max(abs(h["omega"]), 1.0)
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_imex_periodic_bump(prec):
    cfg = stiff(W.periodic_bump(nx=32, nv=16), Kn=1e-4)
    s, Fo, _ = run_pair(cfg, 20, prec)
    check(cfg, s, Fo, prec)
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_imex_sphere(prec):
    cfg = stiff(W.sphere_mach15(n=16, nv=8), Kn=1e-3)
    s, Fo, _ = run_pair(cfg, 6, prec)
    check(cfg, s, Fo, prec)
    s.close()


def test_imex_graph_replays_bitwise():
    cfg = stiff(W.cylinder_mach2(nx=48, nv=16))
    out = []
    for graphs in (False, True):
        s = dvm.Solver(cfg, dvm.FP32)
        s.graphs(graphs)
        s.init_maxwellian()
        s.step(21)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])


def test_imex_adjoint_refused():
    cfg = stiff(W.cylinder_mach2(nx=32, nv=8))
    s = dvm.Solver(cfg, dvm.FP32)
    s.init_maxwellian()
    with pytest.raises(dvm.DVMError):
        s.drag_adjoint(4, checkpoint_every=2)
    s.close()


def test_time_scheme_argument_checked():
    s = dvm.Solver(W.cylinder_mach2(nx=32, nv=8), dvm.FP32)
    with pytest.raises(dvm.DVMError):
        s.set_time_scheme(2)
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64])
def test_scheme_switch_mid_run(prec):
    """5 explicit, 5 semi-implicit, 5 explicit steps: the explicit step after
    the semi-implicit ones starts from the partial sums the relaxation kernel
    wrote (those of the relaxed state); the oracle runs the same sequence."""
    base = W.cylinder_mach2(nx=48, nv=16)
    base.update(Kn=0.05)
    ce, ci = dict(base, time_scheme=0), dict(base, time_scheme=1)
    F0 = oracle.initial_state(ce)
    Fo = F0.copy()
    for cfg in (ce, ci, ce):
        assert oracle.run(cfg, Fo, 5)["status"] == 0
    s = dvm.Solver(ce, prec)
    s.set_state(F0)
    for scheme in (0, 1, 0):
        s.set_time_scheme(scheme)
        s.step(5)
    Fg = s.get_state()
    assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    s.close()
