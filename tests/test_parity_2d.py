"""Parity of the CUDA library (through the C-ABI) with the FP64 CPU oracle,
2D reduced (f, g) model.  GPU only.

Tolerances (relative, per moment field: ||m_gpu - m_ref||_inf / ||m_ref||_inf):
FP64 path 1e-12, FP32 path 1e-5; geometry bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {dvm.FP64: 1e-12, dvm.FP32: 1e-5}
# Velocities are in units of sqrt(R T0) = 1: a velocity error is relative to
# max(||u||_inf, 1), so that a flow near rest is not measured by the ratio of
# two round-off-sized numbers.
GEO_KEYS = ("type", "cgas", "lx", "ly", "lw", "nwx", "nwy", "rwx", "rwy", "sbar")


def rel_inf(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()
    s = np.abs(np.asarray(b, np.float64)).max()
    return d / s if s > 0 else d


def moments_err(cfg, Fo, s):
    mo = oracle.moments(cfg, Fo)
    mg = s.moments()
    live = mo["rho"] > 0
    errs = {}
    for k in ("rho", "ux", "uy", "T"):
        ref = mo[k][live]
        scale = np.abs(ref).max()
        if k in ("ux", "uy"):
            scale = max(scale, 1.0)
        errs[k] = np.abs(mg[k][live] - ref).max() / scale
    return errs


def run_pair(cfg, steps, prec, init_from_oracle=True):
    F0 = oracle.initial_state(cfg)
    s = dvm.Solver(cfg, prec)
    if init_from_oracle:
        s.set_state(F0)
    else:
        s.init_maxwellian()
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, steps)
    assert h["status"] == 0
    s.step(steps)
    return s, Fo, h


# ------------------------------------------------------------------ geometry
@pytest.mark.parametrize("shape,kw", [
    (1, dict(ra=0.1)), (1, dict(ra=0.2371, cx=0.4987, cy=0.5123)),
    (2, dict(ra=0.12, rb=0.04, theta=0.0)), (2, dict(ra=0.12, rb=0.04, theta=0.7345)),
    (2, dict(ra=0.3, rb=0.05, theta=2.1))])
@pytest.mark.parametrize("nx", [64, 256, 129])
def test_geometry_bit_exact(shape, kw, nx):
    """Appendix A geometry: cell types, edge lengths, wall edges, areas and
    masters equal the oracle's bit for bit for the same (cos, sin)."""
    cfg = W.base2d(nx, nx, 4, 4.0, shape=shape, **kw)
    th = kw.get("theta", 0.0)
    ct, st = math.cos(th), math.sin(th)
    s = dvm.Solver(cfg, dvm.FP64)
    s.geometry2d_at(ct, st)
    gg = s.geometry2d()
    go = oracle.geometry2d(cfg, ct, st)
    for k in GEO_KEYS:
        assert np.array_equal(gg[k], go[k]), k
    mo, rc = oracle.masters2d(cfg, go)
    assert rc == 0
    assert np.array_equal(gg["master"], mo)
    s.close()


# ------------------------------------------------------------------ initial state
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_init_maxwellian(prec):
    cfg = W.cylinder_mach2(nx=48, nv=16)
    s = dvm.Solver(cfg, prec)
    s.init_maxwellian()
    Fo = oracle.initial_state(cfg)
    Fg = s.get_state()
    tol = 1e-15 if prec == dvm.FP64 else 1e-7
    assert rel_inf(Fg, Fo) < tol
    s.close()


# ------------------------------------------------------------------ no obstacle
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_periodic_bump_full_config(prec):
    """2D reduced BGK, periodic 32x32, 16x16 velocities, upwind, 20 steps
    (the FP64 correctness configuration) and its FP32 counterpart."""
    cfg = W.periodic_bump()
    s, Fo, h = run_pair(cfg, 20, prec, init_from_oracle=False)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(s.get_state(), Fo) < 1e-12
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("nx,ny,nv,bc", [
    (37, 29, 12, [0, 0, 0, 0]),            # ragged grid, vector width 2
    (33, 17, 9, [1, 2, 2, 2]),             # odd velocity count, vector width 1
    (40, 24, 16, [2, 2, 1, 1]),            # Maxwellian y sides
])
def test_ragged_grids_no_body(prec, scheme, nx, ny, nv, bc):
    rng = np.random.default_rng(nx * 7 + ny)
    u = 0.6
    st = [None] * 6
    for sd in range(4):
        if bc[sd] == 1:
            n = ny if sd < 2 else nx
            a = np.zeros((n, 5))
            a[:, 0] = 1.0 + 0.1 * rng.uniform(-1, 1, n)
            a[:, 1] = u
            a[:, 2] = 0.2 * rng.uniform(-1, 1, n)
            a[:, 4] = 1.0 + 0.2 * rng.uniform(-1, 1, n)
            st[sd] = a
    X = (np.arange(nx) + 0.5) / nx
    Y = (np.arange(ny) + 0.5) / ny
    XX, YY = np.meshgrid(X, Y)
    cfg = W.base2d(nx, ny, nv, 7.0, Kn=0.05, scheme=scheme, bc=bc + [0, 0], bc_state=st,
                   init=dict(rho=(1 + 0.3 * np.sin(2 * np.pi * XX) * np.cos(2 * np.pi * YY)).ravel(),
                             ux=u, uy=(0.2 * np.sin(2 * np.pi * YY)).ravel(), uz=0.0,
                             T=(1 + 0.2 * np.cos(2 * np.pi * XX)).ravel()))
    s, Fo, h = run_pair(cfg, 25, prec)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(s.get_state(), Fo) < 1e-12
    s.close()


# ------------------------------------------------------------------ fixed obstacle
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_cylinder_small(prec, scheme):
    """Mach-2 cylinder (cut cells, merged control volumes, diffuse wall,
    inflow/outflow) at reduced size: state, moments and drag history."""
    cfg = W.cylinder_mach2(nx=64, nv=16, scheme=scheme)
    steps = 120
    s, Fo, h = run_pair(cfg, steps, prec)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < TOL[prec], errs
    hg = s.history(steps)
    assert len(hg["Fx"]) == steps
    assert rel_inf(hg["Fx"], h["Fx"]) < TOL[prec]
    # the lift is round-off noise around zero: compare on the drag scale
    assert np.abs(hg["Fy"] - h["Fy"]).max() < TOL[prec] * np.abs(h["Fx"]).max()
    if prec == dvm.FP64:
        assert rel_inf(s.get_state(), Fo) < 1e-12
    assert s.get_state().min() >= 0
    s.close()


def test_cylinder_segmented_wall_temperatures():
    cfg = W.cylinder_adjoint(nx=64, nv=16)
    s, Fo, h = run_pair(cfg, 40, dvm.FP64)
    assert rel_inf(s.get_state(), Fo) < 1e-12
    assert rel_inf(s.history(40)["Fx"], h["Fx"]) < 1e-12
    s.close()


# ------------------------------------------------------------------ moving obstacle
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_rotating_ellipse_small(prec):
    """Freely rotating ellipse in shear flow: geometry rebuilt every step on
    the device, fusion, appearing/disappearing cells, FP64 torque and ODE."""
    cfg = W.rotating_ellipse(nx=64, nv=16)
    cfg.update(omega=3.0, inertia=1e-3)
    steps = 100
    s, Fo, h = run_pair(cfg, steps, prec)
    th, om = s.body_state()
    hg = s.history(steps)
    tol = TOL[prec]
    assert abs(th - h["theta"]) < 1e-10 * max(1.0, abs(h["theta"])) if prec == dvm.FP64 else abs(th - h["theta"]) < 1e-6
    assert rel_inf(hg["torque"], h["torque"]) < (1e-9 if prec == dvm.FP64 else 1e-4)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < (1e-10 if prec == dvm.FP64 else tol), errs
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_mass_conservation_gpu(prec):
    """Eq. def-masse on the device: closed periodic box, hot rotating body."""
    cfg = W.base2d(48, 48, 32, 10.0, shape=2, ra=0.2, rb=0.06, theta=0.3, omega=4.0,
                   movable=1, inertia=1e-2, Tw=1.3, Kn=0.1,
                   init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0))
    s = dvm.Solver(cfg, prec)
    s.init_maxwellian()
    m0 = s.mass()
    s.step(120)
    m1 = s.mass()
    drift = abs(m1 - m0) / m0
    assert drift < (1e-13 if prec == dvm.FP64 else 1e-5), drift
    s.close()


# ------------------------------------------------------------------ error paths
def test_errors_are_reported_not_raised_on_device():
    cfg = W.base2d(16, 16, 8, 4.0)
    s = dvm.Solver(cfg, dvm.FP64)
    with pytest.raises(dvm.DVMError) as e:
        s.step(1)                                  # no state yet
    assert e.value.code == dvm.ERR_STATE
    with pytest.raises(dvm.DVMError) as e:
        s.set_state(np.zeros(5))
    assert e.value.code == dvm.ERR_ARG
    s.init_maxwellian()
    s.step(0)
    # a vacuum state is non-physical: detected by the moment kernel, reported
    s.set_state(np.zeros(s.state_size))
    with pytest.raises(dvm.DVMError) as e:
        s.step(1)
    assert e.value.code == dvm.ERR_NONPHYSICAL
    s.close()
