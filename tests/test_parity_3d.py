"""Parity of the CUDA library (through the C-ABI) with the FP64 CPU oracle,
3D full-F model (Sec. 5).  GPU only.

Tolerances: FP64 path 1e-12 relative, FP32 path 1e-5 relative on the
moments (velocities relative to max(||u||_inf, 1)); geometry bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {dvm.FP64: 1e-12, dvm.FP32: 1e-5}
GEO_KEYS = ("type", "cgas", "ax", "ay", "az", "sw", "nwx", "nwy", "nwz", "rwx", "rwy", "rwz", "vol")


def moments_err(cfg, Fo, s):
    mo = oracle.moments(cfg, Fo)
    mg = s.moments()
    live = mo["rho"] > 0
    errs = {}
    for k in ("rho", "ux", "uy", "uz", "T"):
        ref = mo[k][live]
        scale = np.abs(ref).max()
        if k in ("ux", "uy", "uz"):
            scale = max(scale, 1.0)
        errs[k] = np.abs(mg[k][live] - ref).max() / scale
    return errs


def bump_init(cfg, seed=0):
    """Smooth nonuniform macroscopic fields (density bump, swirl, hot spot)."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r2 = (X - 0.45) ** 2 + (Y - 0.55) ** 2 + (Z - 0.5) ** 2
    rho = 1.0 + 0.3 * np.exp(-r2 / 0.02)
    ux = 0.3 * np.sin(2 * np.pi * Y)
    uy = -0.2 * np.sin(2 * np.pi * Z)
    uz = 0.25 * np.cos(2 * np.pi * X)
    T = 1.0 + 0.2 * np.exp(-r2 / 0.05)
    return dict(rho=rho.ravel(), ux=ux.ravel(), uy=uy.ravel(), uz=uz.ravel(), T=T.ravel())


def run_pair(cfg, steps, prec):
    F0 = oracle.initial_state(cfg)
    s = dvm.Solver(cfg, prec)
    s.set_state(F0)
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, steps)
    assert h["status"] == 0
    s.step(steps)
    return s, Fo, h


# ------------------------------------------------------------------ geometry
@pytest.mark.parametrize("n,kw", [
    (20, dict(ra=0.15)), (20, dict(ra=0.2371, cx=0.4987, cy=0.5123, cz=0.4711)),
    (33, dict(ra=0.31, cx=0.503, cy=0.49, cz=0.512)), (48, dict(ra=0.15))])
def test_geometry3d_bit_exact(n, kw):
    """Seven-face virtual cells: types, face areas, wall faces, volumes and
    masters equal the oracle's bit for bit."""
    cfg = W.base3d(n, 4, 4.0, shape=3, **kw)
    s = dvm.Solver(cfg, dvm.FP64)
    gg = s.geometry3d()
    go = oracle.geometry3d(cfg)
    assert go["status"] == 0
    for k in GEO_KEYS:
        assert np.array_equal(gg[k], go[k]), k
    mo, rc = oracle.masters3d(cfg, go)
    assert rc == 0
    assert np.array_equal(gg["master"], mo)
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_init_maxwellian3d(prec):
    cfg = W.base3d(12, 6, 5.0, ny=10, nz=9, nvy=5, nvz=7, shape=3, ra=0.3,
                   init=None)
    cfg["init"] = bump_init(cfg)
    s = dvm.Solver(cfg, prec)
    s.init_maxwellian()
    Fg = s.get_state().astype(np.float64)
    Fo = oracle.initial_state(cfg)
    tol = 1e-14 if prec == dvm.FP64 else 1e-7
    assert np.abs(Fg - Fo).max() <= tol * np.abs(Fo).max()
    s.close()


# ------------------------------------------------------------------ no obstacle
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("dims,nvs,bc", [
    ((12, 10, 9), (6, 5, 4), [0] * 6),
    ((37, 9, 6), (8, 6, 6), [1, 2, 2, 2, 0, 0]),
    ((8, 17, 5), (5, 4, 6), [2, 2, 0, 0, 1, 1]),
])
def test_ragged_no_body_3d(prec, scheme, dims, nvs, bc):
    """Ragged grids (x not a multiple of the warp, y of the block rows, z of
    the z-column, v_x of the velocity group), periodic, Maxwellian and
    zero-gradient sides, both schemes: state and moments after 8 steps."""
    nx, ny, nz = dims
    cfg = W.base3d(nx, nvs[0], 5.0, ny=ny, nz=nz, nvy=nvs[1], nvz=nvs[2], scheme=scheme,
                   Kn=0.2, Lref=1.0, cfl=0.45, bc=list(bc))
    sides = [None] * 6
    for sd in range(6):
        if bc[sd] == 1:
            n = (ny * nz) if sd < 2 else ((nx * nz) if sd < 4 else nx * ny)
            st = np.zeros((n, 5))
            st[:, 0] = 1.1
            st[:, 1] = 0.4 if sd == 0 else -0.1
            st[:, 2] = 0.05
            st[:, 3] = -0.1 if sd == 4 else 0.1
            st[:, 4] = 1.05
            sides[sd] = st
    cfg["bc_state"] = sides
    cfg["init"] = bump_init(cfg)
    s, Fo, _ = run_pair(cfg, 8, prec)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < TOL[prec], errs
    if prec == dvm.FP64:
        Fg = s.get_state()
        assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    s.close()


# ------------------------------------------------------------------ sphere
@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
@pytest.mark.parametrize("scheme", [0, 1])
def test_sphere_small(prec, scheme):
    """The 3D sphere problem (Mach-1.5 Maxwellian inflow on x-, zero-gradient
    elsewhere, diffuse wall at T0) on a 20^3 grid with 8^3 velocities:
    moments, state and the drag history after 10 steps."""
    cfg = W.sphere_mach15(n=20, nv=8, scheme=scheme)
    cfg["ra"] = 0.23
    s, Fo, h = run_pair(cfg, 10, prec)
    errs = moments_err(cfg, Fo, s)
    assert max(errs.values()) < TOL[prec], errs
    hg = s.history(10)
    fs = np.abs(h["Fx"]).max()
    assert fs > 0
    for k in ("Fx", "Fy", "Fz"):
        assert np.abs(hg[k] - h[k]).max() <= TOL[prec] * 10 * fs, (k, hg[k], h[k])
    if prec == dvm.FP64:
        Fg = s.get_state()
        assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    cc = s.cell_counts()
    assert cc["walls"] > 0 and cc["cvs"] > 0
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_sphere_rotating_wall_torque(prec):
    """Wall velocity of a spinning (fixed-centre) sphere, u_w = omega e_z x
    (r - c): torque about z against the oracle."""
    cfg = W.base3d(16, 8, 6.0, shape=3, ra=0.27, omega=1.5, Tw=1.2, scheme=1, Kn=0.1,
                   init=dict(rho=1.0, ux=0.3, uy=-0.1, uz=0.2, T=1.0))
    s, Fo, h = run_pair(cfg, 6, prec)
    hg = s.history(6)
    fs = np.abs(np.stack([h["Fx"], h["Fy"], h["Fz"]])).max()
    assert np.abs(h["torque"]).max() > 1e-6 * fs
    assert np.abs(hg["torque"] - h["torque"]).max() <= TOL[prec] * 10 * fs * cfg["ra"]
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_mass_conservation_gpu_3d(prec):
    """Periodic box, hot sphere, drifting gas: dvm_mass constant in time.
    dv = 0.8 makes the discrete moments of the direct Maxwellian exact to
    ~1e-14, so the relaxation conserves mass too (as in the oracle pin)."""
    cfg = W.base3d(16, 20, 8.0, shape=3, ra=0.25, Tw=1.3, Kn=0.1, scheme=1,
                   init=dict(rho=1.0, ux=0.4, uy=0.1, uz=-0.2, T=1.0))
    s = dvm.Solver(cfg, prec)
    s.set_state(oracle.initial_state(cfg))
    m0 = s.mass()
    s.step(20)
    drift = abs(s.mass() - m0) / m0
    assert drift < (1e-12 if prec == dvm.FP64 else 2e-6), drift
    s.close()


def test_errors_3d():
    cfg = W.base3d(8, 4, 4.0, nz=3)
    with pytest.raises(dvm.DVMError) as e:
        dvm.Solver(cfg, dvm.FP64)
    assert e.value.code == dvm.ERR_ARG
    cfg = W.base3d(8, 4, 4.0, shape=3, ra=0.2, movable=1, inertia=1.0)
    with pytest.raises(dvm.DVMError) as e:
        dvm.Solver(cfg, dvm.FP64)
    assert e.value.code == dvm.ERR_UNSUPPORTED
    cfg = W.base3d(8, 4, 4.0, shape=2, ra=0.2, rb=0.1)
    with pytest.raises(dvm.DVMError) as e:
        dvm.Solver(cfg, dvm.FP64)
    assert e.value.code == dvm.ERR_UNSUPPORTED
