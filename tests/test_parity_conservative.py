"""Parity of the conservative discrete equilibrium on the GPU
(dvm_set_equilibrium(DVM_EQ_CONSERVATIVE), Sec. 3.1: the equilibrium's
(rho, u, T) by Newton's method so that its discrete moments equal the
state's) with the oracle's, and exact discrete conservation on a coarse
velocity grid.  GPU only.

Tolerances: FP64 state within 1e-12 of the largest value; FP32 moments within
1e-5 (relative per field; velocities relative to max(|u|, 1)).  The cases use
coarse velocity grids, where the conservative parameters differ from the
direct moments (a GPU path that ignored the mode would fail the FP64 state
check).
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
    s.set_state(F0)
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, steps)
    assert h["status"] == 0
    s.step(steps)
    return s, Fo, h


def check(cfg, s, Fo, prec):
    if prec == dvm.FP64:
        Fg = s.get_state()
        assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max(), np.abs(Fg - Fo).max() / np.abs(Fo).max()
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < (1e-12 if prec == dvm.FP64 else 1e-5), errs


def cons(cfg, **kw):
    cfg = dict(cfg)
    cfg.update(conservative=1, **kw)
    return cfg


def test_conservative_differs_from_direct_here():
    """The cases below are meaningful: on the coarse grid the two modes give
    states that differ by far more than the parity tolerance."""
    cfg = W.cylinder_mach2(nx=32, nv=10, scheme=1)
    a = oracle.initial_state(cfg)
    b = a.copy()
    oracle.run(cfg, a, 5)
    oracle.run(cons(cfg), b, 5)
    assert np.abs(a - b).max() > 1e-6 * np.abs(a).max()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_conservative_cylinder(prec, scheme):
    """Fixed cylinder, Mach 2, 10^2 velocities on [-8, 8)^2 (dv = 1.6): cut
    cells, merged control volumes, diffuse wall, Maxwellian and zero-gradient
    sides; 12 steps (the graph replays included)."""
    cfg = cons(W.cylinder_mach2(nx=40, nv=10, scheme=scheme))
    s, Fo, h = run_pair(cfg, 12, prec)
    check(cfg, s, Fo, prec)
    hg = s.history(12)["Fx"]
    tol = 1e-10 if prec == dvm.FP64 else 1e-4
    assert np.abs(hg - h["Fx"]).max() <= tol * np.abs(h["Fx"]).max()
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_conservative_semi_implicit_stiff(prec):
    """The semi-implicit scheme (Eq. ImpSchemeDD) at dt/tau0 > 5, with the
    conservative parameters of the transported state."""
    cfg = cons(W.cylinder_mach2(nx=40, nv=10, scheme=1), Kn=1e-3, time_scheme=1)
    s, Fo, h = run_pair(cfg, 12, prec)
    assert s.dt / s.tau0 > 5
    check(cfg, s, Fo, prec)
    s.close()


def test_conservative_moving_ellipse_fp64():
    """Rotating ellipse (geometry rebuilt every step, fusion each step)."""
    cfg = cons(W.rotating_ellipse(nx=48, nv=10, scheme=1))
    s, Fo, h = run_pair(cfg, 10, dvm.FP64)
    check(cfg, s, Fo, dvm.FP64)
    s.close()


@pytest.mark.parametrize("bc", [[0, 0, 0, 0, 0, 0], [2, 2, 2, 2, 0, 0]])
def test_conservative_ragged_box(bc):
    """No obstacle, ragged 37 x 29 grid (several tiles and a ragged tail),
    drifting non-uniform gas, periodic or zero-gradient sides, FP64 and FP32."""
    nx, ny = 37, 29
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    init = dict(rho=(1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).ravel(),
                ux=(0.6 + 0.3 * np.cos(2 * np.pi * Y)).ravel(), uy=(0.2 * np.sin(2 * np.pi * X)).ravel(),
                uz=0.0, T=(1.0 + 0.3 * np.cos(2 * np.pi * X)).ravel())
    cfg = W.base2d(nx, ny, 10, 5.0, Kn=0.02, Lref=1.0, scheme=1, bc=bc, init=init, conservative=1)
    for prec in (dvm.FP64, dvm.FP32):
        s, Fo, _ = run_pair(cfg, 15, prec)
        check(cfg, s, Fo, prec)
        s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_conservative_sphere(prec):
    """3D sphere, 8^3 velocities on [-5, 5)^3, MUSCL, Mach 1.5: the full F
    with five unknowns per cell."""
    cfg = cons(W.sphere_mach15(n=16, nv=8, scheme=1))
    cfg["ra"] = 0.23
    s, Fo, h = run_pair(cfg, 5, prec)
    check(cfg, s, Fo, prec)
    s.close()


def test_conservative_sphere_semi_implicit_fp64():
    cfg = cons(W.sphere_mach15(n=16, nv=8, scheme=1), Kn=1e-3, time_scheme=1)
    cfg["ra"] = 0.23
    s, Fo, h = run_pair(cfg, 5, dvm.FP64)
    check(cfg, s, Fo, dvm.FP64)
    s.close()


def _totals2(cfg, F):
    nc = cfg["nx"] * cfg["ny"]
    dvx = (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]
    dvy = (cfg["vymax"] - cfg["vymin"]) / cfg["nvy"]
    VX, VY = np.meshgrid(cfg["vxmin"] + np.arange(cfg["nvx"]) * dvx, cfg["vymin"] + np.arange(cfg["nvy"]) * dvy)
    VX, VY = VX.ravel(), VY.ravel()
    Fv = F.reshape(nc, 2, VX.size).astype(np.float64)
    f, g = Fv[:, 0], Fv[:, 1]
    dv = dvx * dvy
    return np.array([f.sum(), (f * VX).sum(), (f * VY).sum(), (0.5 * (VX ** 2 + VY ** 2) * f + g).sum()]) * dv


@pytest.mark.parametrize("time_scheme", [0, 1])
def test_gpu_conserves_mass_momentum_energy(time_scheme):
    """Periodic 48^2 box, 10^2 velocities on [-5, 5)^2, FP64: with the
    conservative equilibrium the totals stay at their initial values to
    round-off over 100 steps; with the direct moments momentum and energy
    drift by far more (the same run on the GPU)."""
    n = 48
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    init = dict(rho=(1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).ravel(),
                ux=(0.5 + 0.3 * np.cos(2 * np.pi * Y)).ravel(), uy=(0.2 * np.sin(2 * np.pi * X)).ravel(),
                uz=0.0, T=(1.0 + 0.3 * np.cos(2 * np.pi * X)).ravel())
    drift = {}
    for mode in (1, 0):
        cfg = W.base2d(n, n, 10, 5.0, Kn=0.02 if time_scheme == 0 else 1e-3, Lref=1.0, scheme=1, init=init,
                       conservative=mode, time_scheme=time_scheme)
        s = dvm.Solver(cfg, dvm.FP64)
        s.init_maxwellian()
        t0 = _totals2(cfg, s.get_state())
        s.step(100)
        t1 = _totals2(cfg, s.get_state())
        s.close()
        scale = np.array([t0[0], t0[0], t0[0], t0[3]])
        drift[mode] = np.abs(t1 - t0) / scale
    assert drift[1].max() <= 1e-13, drift[1]
    assert drift[0][1:].max() > 1e-7, drift[0]


def test_conservative_mode_errors():
    cfg = W.cylinder_mach2(nx=32, nv=8)
    s = dvm.Solver(cfg, dvm.FP64)
    with pytest.raises(dvm.DVMError) as e:
        s.set_equilibrium(7)
    assert e.value.code == dvm.ERR_ARG
    s.set_equilibrium(1)
    with pytest.raises(dvm.DVMError) as e:
        s.set_collision_model(1, 2.0 / 3.0)            # Shakhov with the conservative mode
    assert e.value.code == dvm.ERR_UNSUPPORTED
    s.init_maxwellian()
    with pytest.raises(dvm.DVMError) as e:
        s.drag_adjoint(3, 2)
    assert e.value.code == dvm.ERR_UNSUPPORTED
    s.close()
    s = dvm.Solver(cfg, dvm.FP64)
    s.set_collision_model(1, 2.0 / 3.0)
    with pytest.raises(dvm.DVMError) as e:
        s.set_equilibrium(1)
    assert e.value.code == dvm.ERR_UNSUPPORTED
    s.close()
