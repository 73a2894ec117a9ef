"""Parity of the Shakhov collision model of the CUDA library with the FP64
CPU oracle: the reduced 2D (f, g) model of Eq. ShakhovDD and the full 3D F
of Sec. 2.1, under the explicit scheme (fixed and rotating obstacles) and the
semi-implicit one.  GPU only.

Tolerances as for BGK: FP64 state within 1e-12 of the largest value, FP32
moments within 1e-5 (relative; velocities on the scale max(|u|, 1)).
"""
import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {dvm.FP64: 1e-12, dvm.FP32: 1e-5}
PR = 2.0 / 3.0


def rel_inf(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()
    s = np.abs(np.asarray(b, np.float64)).max()
    return d / s if s > 0 else d


def moments_err(cfg, Fo, Fg):
    mo = oracle.moments(cfg, Fo)
    mg = oracle.moments(cfg, np.asarray(Fg, np.float64))
    live = mo["rho"] > 0
    errs = {}
    keys = ("rho", "ux", "uy", "uz", "T") if cfg.get("dim", 2) == 3 else ("rho", "ux", "uy", "T")
    for k in keys:
        ref = mo[k][live]
        scale = np.abs(ref).max()
        if k in ("ux", "uy", "uz"):
            scale = max(scale, 1.0)
        errs[k] = np.abs(mg[k][live] - ref).max() / scale
    return errs


def shakhov(cfg, Pr=PR):
    return dict(cfg, model=dvm.SHAKHOV, Pr=Pr)


def run_pair(cfg, steps, prec, F0=None):
    F0 = oracle.initial_state(cfg) if F0 is None else F0
    s = dvm.Solver(cfg, prec)
    s.set_state(F0)
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, steps)
    assert h["status"] == 0
    s.step(steps)
    return s, Fo, h


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_cylinder_small(prec, scheme):
    """Mach-2 cylinder (cut cells, merged control volumes, diffuse wall)."""
    cfg = shakhov(W.cylinder_mach2(nx=64, nv=16, scheme=scheme))
    steps = 60
    s, Fo, h = run_pair(cfg, steps, prec)
    Fg = s.get_state()
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) < TOL[prec]
    assert rel_inf(s.history(steps)["Fx"], h["Fx"]) < TOL[prec]
    # the heat flux term is not negligible here: BGK lands elsewhere
    Fb = oracle.initial_state(cfg)
    oracle.run(dict(cfg, model=0), Fb, steps)
    assert rel_inf(Fb, Fo) > 1e3 * TOL[dvm.FP32]
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_ragged_no_body(prec, scheme):
    """A grid that is not a multiple of the tiles, Maxwellian, zero-gradient
    and periodic sides, a hot spot whose heat flux the model relaxes."""
    nx, ny, nv = 37, 21, 12
    cfg = W.base2d(nx, ny, nv, 5.0, Kn=0.3, scheme=scheme, bc=[1, 2, 0, 0, 0, 0])
    side = np.zeros((ny, 5))
    side[:, 0] = 1.0
    side[:, 1] = 0.3
    side[:, 4] = 1.0
    cfg["bc_state"] = [side, None, None, None, None, None]
    xc = (np.arange(nx) + 0.5) / nx
    yc = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(xc, yc)
    bump = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / 0.02).ravel()
    cfg["init"] = dict(rho=1.0 + 0.3 * bump, ux=0.1, uy=-0.05, uz=0.0, T=1.0 + 0.5 * bump)
    cfg = shakhov(cfg, Pr=0.5)
    s, Fo, _ = run_pair(cfg, 25, prec)
    Fg = s.get_state()
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) < TOL[prec]
    s.close()


@pytest.mark.parametrize("Pr", [PR, 0.2])
def test_heat_flux_relaxes_at_rate_pr(Pr):
    """Homogeneous periodic gas with a heat flux: each explicit step
    multiplies it by 1 - Pr dt/tau and leaves rho, u, T fixed."""
    n, nv, win = 4, 64, 12.0
    cfg = shakhov(W.base2d(n, n, nv, win, Kn=0.5, bc=[0] * 6), Pr=Pr)
    rho, u, T, q = 1.2, (0.4, -0.3), 1.3, (0.2, -0.15)
    start = oracle.equilibrium(dict(cfg, model=1, Pr=0.0), rho, u, T, q)
    s = dvm.Solver(cfg, dvm.FP64)
    s.set_state(np.tile(start, n * n))
    steps = 16
    s.step(steps)
    Fg = s.get_state()
    cell = Fg[: start.size]
    q0, _ = oracle.heat_flux(cfg, start)
    qn, _ = oracle.heat_flux(cfg, cell)
    r = s.dt * rho / s.tau0
    assert np.allclose(qn, (1.0 - Pr * r) ** steps * q0, rtol=0, atol=1e-10 * np.abs(q0).max())
    m = oracle.moments(cfg, Fg)
    assert np.allclose(m["rho"], rho, rtol=1e-12) and np.allclose(m["T"], T, rtol=1e-12)
    s.close()


def test_unsupported_combinations_are_reported():
    cyl = W.cylinder_mach2(nx=32, nv=8)
    s = dvm.Solver(cyl, dvm.FP32)
    with pytest.raises(dvm.DVMError) as e:
        s.set_collision_model(dvm.SHAKHOV, -0.1)
    assert e.value.code == dvm.ERR_ARG
    s.set_collision_model(dvm.SHAKHOV, PR)
    s.init_maxwellian()
    with pytest.raises(dvm.DVMError) as e:
        s.drag_adjoint(4, 2)
    assert e.value.code == dvm.ERR_UNSUPPORTED
    with pytest.raises(dvm.DVMError) as e:
        s.set_equilibrium(1)                   # the conservative equilibrium is BGK
    assert e.value.code == dvm.ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_moving_ellipse(prec):
    """Rotating ellipse: the geometry is rebuilt every step, control volumes
    merge, appear and vanish, and the Shakhov term of a merged control volume
    carries its area ratio S^n / S^{n+1,*} (Eq. ExSchemeDD); the torque and
    the body angle follow the oracle's."""
    cfg = shakhov(W.rotating_ellipse(nx=64, nv=12, scheme=1))
    s, Fo, h = run_pair(cfg, 12, prec)
    Fg = s.get_state()
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) <= 1e-12, rel_inf(Fg, Fo)
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    th, om = s.body_state()
    assert abs(th - h["theta"]) <= (1e-12 if prec == dvm.FP64 else 1e-8)
    assert rel_inf(s.history(12)["torque"], h["torque"]) <= (1e-10 if prec == dvm.FP64 else 1e-4)
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_semi_implicit_stiff(prec):
    """The semi-implicit scheme (Eq. ImpSchemeDD) with the Shakhov
    equilibrium at dt/tau0 > 5, heat flux q_T / (1 + nu Pr): cylinder, MUSCL,
    and a rotating ellipse in FP64."""
    cfg = shakhov(dict(W.cylinder_mach2(nx=40, nv=12), Kn=1e-3, time_scheme=1))
    s, Fo, _ = run_pair(cfg, 12, prec)
    assert s.dt / s.tau0 > 5
    Fg = s.get_state()
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) <= 1e-12, rel_inf(Fg, Fo)
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    s.close()
    if prec == dvm.FP64:
        cfg = shakhov(dict(W.rotating_ellipse(nx=48, nv=12, scheme=1), Kn=5e-4, time_scheme=1))
        s, Fo, _ = run_pair(cfg, 10, prec)
        assert rel_inf(s.get_state(), Fo) <= 1e-12
        s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_semi_implicit_sphere_3d(prec):
    cfg = shakhov(dict(W.sphere_mach15(n=16, nv=8, scheme=1), Kn=1e-3, time_scheme=1))
    cfg["ra"] = 0.23
    s, Fo, _ = run_pair(cfg, 5, prec)
    Fg = s.get_state()
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) <= 1e-12, rel_inf(Fg, Fo)
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    s.close()


# ------------------------------------------------------------------ 3D
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_sphere_small_3d(prec, scheme):
    """Mach-1.5 sphere, 20^3 cells x 8^3 velocities: state, moments, drag."""
    cfg = W.sphere_mach15(n=20, nv=8, scheme=scheme)
    cfg["ra"] = 0.23
    cfg = shakhov(cfg)
    steps = 10
    F0 = oracle.initial_state(cfg)
    Fo = F0.copy()
    h = oracle.run3d(cfg, Fo, steps)
    assert h["status"] == 0
    s = dvm.Solver(cfg, prec)
    s.set_state(F0)
    s.step(steps)
    Fg = s.get_state()
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) < TOL[prec]
    fs = np.abs(h["Fx"]).max()
    assert np.abs(s.history(steps)["Fx"] - h["Fx"]).max() <= 10 * TOL[prec] * fs
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("dims,nvs,bc", [((12, 10, 9), (6, 5, 4), [0] * 6),
                                         ((9, 7, 11), (6, 6, 5), [2] * 6)])
def test_ragged_no_body_3d(prec, dims, nvs, bc):
    nx, ny, nz = dims
    cfg = W.base3d(nx, nvs[0], 5.0, ny=ny, nz=nz, nvy=nvs[1], nvz=nvs[2], scheme=1, Kn=0.2, cfl=0.45, bc=list(bc))
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    bump = np.exp(-((X - 0.5) ** 2 + (Y - 0.4) ** 2 + (Z - 0.6) ** 2) / 0.03).ravel()
    cfg["init"] = dict(rho=1.0 + 0.3 * bump, ux=0.1, uy=-0.05, uz=0.05, T=1.0 + 0.5 * bump)
    cfg = shakhov(cfg, Pr=0.5)
    F0 = oracle.initial_state(cfg)
    Fo = F0.copy()
    assert oracle.run3d(cfg, Fo, 8)["status"] == 0
    s = dvm.Solver(cfg, prec)
    s.set_state(F0)
    s.step(8)
    Fg = s.get_state()
    errs = moments_err(cfg, Fo, Fg)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        assert rel_inf(Fg, Fo) < TOL[prec]
    s.close()


def test_heat_flux_relaxes_at_rate_pr_3d():
    n, nv, win, Pr = 4, 40, 11.0, PR
    cfg = shakhov(W.base3d(n, nv, win, Kn=0.5, bc=[0] * 6), Pr=Pr)
    rho, u, T, q = 1.2, (0.4, -0.3, 0.2), 1.3, (0.2, -0.15, 0.1)
    start = oracle.equilibrium(dict(cfg, model=1, Pr=0.0), rho, u, T, q)
    s = dvm.Solver(cfg, dvm.FP64)
    s.set_state(np.tile(start, n ** 3))
    steps = 12
    s.step(steps)
    cell = s.get_state()[: start.size]
    q0, _ = oracle.heat_flux(cfg, start)
    qn, _ = oracle.heat_flux(cfg, cell)
    r = s.dt * rho / s.tau0
    assert np.allclose(qn, (1.0 - Pr * r) ** steps * q0, rtol=0, atol=1e-10 * np.abs(q0).max())
    s.close()
