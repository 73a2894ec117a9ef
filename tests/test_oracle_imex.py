"""Pins of the oracle's first-order semi-implicit scheme (Sec. 3.3,
Eq. ImpSchemeDD): transport explicit, relaxation implicit with the moments of
the new time level, which are those of the transported values because the
collision term sums to zero over the velocities.  CPU only.

Each test names the fact it pins and the mistake it would catch.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import workloads as W


def _maxw2d(rho, ux, uy, T, vx, vy):
    # textbook 2D Gaussian used only to build inputs and closed forms
    return rho / (2 * np.pi * T) * np.exp(-((vx - ux) ** 2 + (vy - uy) ** 2) / (2 * T))


def _maxw3d(rho, u, T, VX, VY, VZ):
    # textbook 3D Gaussian used only to build inputs and closed forms
    return rho / (2 * np.pi * T) ** 1.5 * np.exp(
        -((VX - u[0]) ** 2 + (VY - u[1]) ** 2 + (VZ - u[2]) ** 2) / (2 * T))


def _vgrid(cfg):
    dvx = (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]
    dvy = (cfg["vymax"] - cfg["vymin"]) / cfg["nvy"]
    vx = cfg["vxmin"] + np.arange(cfg["nvx"]) * dvx
    vy = cfg["vymin"] + np.arange(cfg["nvy"]) * dvy
    VX, VY = np.meshgrid(vx, vy)          # p = p2*nvx + p1
    return VX.ravel(), VY.ravel(), dvx * dvy


def _tau(cfg, rho):
    # tau = tau0 / rho with tau0 = sqrt(pi)/2 Kn Lref / sqrt(2) (Sec. 2.1)
    return math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2) / rho


def test_imex_space_homogeneous_closed_form():
    """No transport in a uniform state: f^{n+1} = (f^n + nu M)/(1 + nu), so
    f^n = M + (1 + nu)^-n (f^0 - M), here with dt/tau = 3.5, far beyond the
    explicit scheme's dt < tau.  Catches an explicit (1 - nu) factor, a wrong
    nu = dt rho/tau0, and a wrong reduced equilibrium g_eq = T/2 M."""
    cfg = W.base2d(2, 1, 32, 10.0, Kn=0.05, Lref=1.0, dt=0.1, time_scheme=1)
    VX, VY, dv = _vgrid(cfg)
    r1, u1, T1 = 0.6, (0.3, 0.1), 0.8
    r2, u2, T2 = 0.5, (-0.3, 0.2), 1.0
    f0 = _maxw2d(r1, *u1, T1, VX, VY) + _maxw2d(r2, *u2, T2, VX, VY)
    g0 = T1 / 2 * _maxw2d(r1, *u1, T1, VX, VY) + T2 / 2 * _maxw2d(r2, *u2, T2, VX, VY)
    rho = r1 + r2
    ux = (r1 * u1[0] + r2 * u2[0]) / rho
    uy = (r1 * u1[1] + r2 * u2[1]) / rho
    E = sum(r * (0.5 * (u[0] ** 2 + u[1] ** 2) + 1.5 * T) for r, u, T in ((r1, u1, T1), (r2, u2, T2)))
    T = (2 * E / rho - ux ** 2 - uy ** 2) / 3
    M = _maxw2d(rho, ux, uy, T, VX, VY)
    G = T / 2 * M
    cell = np.concatenate([f0, g0])
    F = np.concatenate([cell, cell])
    n = 10
    h = oracle.run(cfg, F, n)
    assert h["status"] == 0
    nu = cfg["dt"] / _tau(cfg, rho)
    assert nu > 3
    lam = (1 + nu) ** -n
    nv = VX.size
    for c in range(2):
        got = F[c * 2 * nv: (c + 1) * 2 * nv]
        np.testing.assert_allclose(got[:nv], M + lam * (f0 - M), rtol=0, atol=1e-13 * f0.max())
        np.testing.assert_allclose(got[nv:], G + lam * (g0 - G), rtol=0, atol=1e-13 * g0.max())


def _bump_row(time_scheme, Kn):
    nx = 16
    x = (np.arange(nx) + 0.5) / nx
    return W.base2d(nx, 1, 24, 8.0, Kn=Kn, Lref=1.0, cfl=0.5, scheme=1, time_scheme=time_scheme,
                    init=dict(rho=1.0 + 0.3 * np.sin(2 * np.pi * x), ux=0.2, uy=0.0, uz=0.0,
                              T=1.0 + 0.2 * np.cos(2 * np.pi * x)))


def test_imex_stiff_limit_is_maxwellian_of_transported_moments():
    """nu -> infinity: one step gives, in every cell, the Maxwellian of the
    moments of the transported values (pure transport: the explicit scheme
    with tau = infinity, pinned by the transport tests), built here from the
    textbook moment formulas.  Catches moments taken at t^n instead of
    t^{n+1}: in this non-uniform row transport changes them by about 1e-2."""
    Ft = oracle.initial_state(_bump_row(0, 1e30))
    F0 = Ft.copy()
    assert oracle.run(_bump_row(0, 1e30), Ft, 1)["status"] == 0
    cfg = _bump_row(1, 1e-13)
    F = F0.copy()
    assert oracle.run(cfg, F, 1)["status"] == 0
    VX, VY, dv = _vgrid(cfg)
    nv = VX.size
    moved = 0.0
    for k in range(cfg["nx"]):
        f, g = Ft[(2 * k) * nv:(2 * k + 1) * nv], Ft[(2 * k + 1) * nv:(2 * k + 2) * nv]
        rho = f.sum() * dv
        ux, uy = (VX * f).sum() * dv / rho, (VY * f).sum() * dv / rho
        E = ((0.5 * (VX ** 2 + VY ** 2) * f).sum() + g.sum()) * dv
        T = (2 * E / rho - ux ** 2 - uy ** 2) / 3
        M = _maxw2d(rho, ux, uy, T, VX, VY)
        np.testing.assert_allclose(F[(2 * k) * nv:(2 * k + 1) * nv], M, rtol=0, atol=1e-10 * M.max())
        np.testing.assert_allclose(F[(2 * k + 1) * nv:(2 * k + 2) * nv], T / 2 * M, rtol=0,
                                   atol=1e-10 * M.max())
        rho0 = F0[(2 * k) * nv:(2 * k + 1) * nv].sum() * dv
        moved = max(moved, abs(rho - rho0) / rho0)
    assert moved > 1e-3      # the transported moments differ from those at t^n


@pytest.mark.parametrize("moving", [False, True])
def test_imex_without_collisions_is_transport(moving):
    """tau = infinity: nu = 0 and the semi-implicit scheme is the explicit
    transport with the area ratio S^n/S^{n+1} of a moving body (the first two
    terms of Eq. ImpSchemeDD equal those of Eq. ExSchemeDD).  Catches a
    dropped or changed transport term in the semi-implicit branch."""
    kw = dict(Kn=1e30, Lref=1.0, cfl=0.5, scheme=1, Tw=1.2,
              init=dict(rho=1.0, ux=0.3, uy=0.1, uz=0.0, T=1.0))
    if moving:
        kw.update(shape=2, ra=0.2, rb=0.06, theta=0.3, omega=4.0, movable=1, inertia=1e-2)
    else:
        kw.update(shape=1, ra=0.15)
    ce = W.base2d(32, 32, 12, 6.0, time_scheme=0, **kw)
    ci = W.base2d(32, 32, 12, 6.0, time_scheme=1, **kw)
    Fe = oracle.initial_state(ce)
    Fi = Fe.copy()
    assert oracle.run(ce, Fe, 6)["status"] == 0
    assert oracle.run(ci, Fi, 6)["status"] == 0
    np.testing.assert_allclose(Fi, Fe, rtol=0, atol=1e-14 * np.abs(Fe).max())


def test_imex_mass_conservation_closed_box():
    """Sec. 3.4.2 (Eq. def-masse) for the semi-implicit scheme: periodic box,
    hot diffuse wall, drifting gas, dt/tau about 4.  The velocity grid
    (dv = 0.625 on [-10, 10)) makes the discrete moments of the Maxwellian
    exact to round-off, so the implicit relaxation conserves mass too."""
    cfg = W.base2d(48, 48, 32, 10.0, shape=1, ra=0.15, Tw=1.3, Kn=2e-4, scheme=1, time_scheme=1,
                   init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0))
    F = oracle.initial_state(cfg)
    M0 = oracle.mass2d(cfg, F)
    h = oracle.run(cfg, F, 60)
    assert h["status"] == 0
    assert oracle.time_step(cfg) / oracle.tau0(cfg) > 3
    drift = np.abs(h["mass"] - M0).max() / M0
    assert drift < 1e-13, drift


def test_imex_3d_space_homogeneous_closed_form():
    """Full F in 3D: f^n = M + (1 + nu)^-n (f^0 - M) with the 3D Maxwellian
    of the conserved moments, dt/tau = 3.5."""
    cfg = W.base3d(2, 40, 10.0, nx=2, ny=1, nz=1, Kn=0.05, Lref=1.0, dt=0.1, time_scheme=1)
    n1 = cfg["nvx"]
    v = cfg["vxmin"] + np.arange(n1) * (cfg["vxmax"] - cfg["vxmin"]) / n1
    VZ, VY, VX = np.meshgrid(v, v, v, indexing="ij")
    VX, VY, VZ = VX.ravel(), VY.ravel(), VZ.ravel()
    r1, u1, T1 = 0.6, (0.3, 0.1, -0.2), 0.8
    r2, u2, T2 = 0.5, (-0.3, 0.2, 0.1), 1.1
    f0 = _maxw3d(r1, u1, T1, VX, VY, VZ) + _maxw3d(r2, u2, T2, VX, VY, VZ)
    rho = r1 + r2
    u = (r1 * np.array(u1) + r2 * np.array(u2)) / rho
    E = sum(r * (0.5 * np.dot(uu, uu) + 1.5 * T) for r, uu, T in ((r1, u1, T1), (r2, u2, T2)))
    T = (2 * E / rho - u @ u) / 3
    M = _maxw3d(rho, u, T, VX, VY, VZ)
    F = np.concatenate([f0, f0])
    n = 8
    assert oracle.run(cfg, F, n)["status"] == 0
    lam = (1 + cfg["dt"] / _tau(cfg, rho)) ** -n
    for c in range(2):
        np.testing.assert_allclose(F[c * VX.size:(c + 1) * VX.size], M + lam * (f0 - M), rtol=0,
                                   atol=3e-13 * f0.max())
