"""Pins of the oracle's conservative discrete equilibrium (Sec. 3.1, the
paragraph after Eq. MacroscopicDDv: the (rho, u, T) of the equilibrium are
obtained by Newton's method so that the collision term keeps the discrete
conservation).  CPU only.

The defining property is that the discrete moments of the discrete
equilibrium equal those of the state.  The tests below check it with
moments summed here in numpy (independent of the oracle's loops), and its
consequences: a discrete Maxwellian is its own equilibrium, the parameters
tend to the direct moments on wide fine grids, and a periodic box conserves
mass, momentum and energy to round-off on a coarse velocity grid, where the
direct moments visibly do not.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import workloads as W


def _grid2(cfg):
    dvx = (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]
    dvy = (cfg["vymax"] - cfg["vymin"]) / cfg["nvy"]
    vx = cfg["vxmin"] + np.arange(cfg["nvx"]) * dvx
    vy = cfg["vymin"] + np.arange(cfg["nvy"]) * dvy
    VX, VY = np.meshgrid(vx, vy)
    return VX.ravel(), VY.ravel(), dvx * dvy


def _grid3(cfg):
    d = [(cfg[f"v{a}max"] - cfg[f"v{a}min"]) / cfg[f"nv{a}"] for a in "xyz"]
    ax = [cfg[f"v{a}min"] + np.arange(cfg[f"nv{a}"]) * d[k] for k, a in enumerate("xyz")]
    VZ, VY, VX = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")   # p = (p3 nvy + p2) nvx + p1
    return VX.ravel(), VY.ravel(), VZ.ravel(), d[0] * d[1] * d[2]


def _m2(r, ux, uy, T, VX, VY):
    return r / (2 * np.pi * T) * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2) / (2 * T))


def _m3(r, ux, uy, uz, T, VX, VY, VZ):
    return r / (2 * np.pi * T) ** 1.5 * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2 + (VZ - uz) ** 2) / (2 * T))


def _moments2(f, g, VX, VY, dv):
    return np.array([f.sum() * dv, (VX * f).sum() * dv, (VY * f).sum() * dv,
                     (0.5 * (VX ** 2 + VY ** 2) * f + g).sum() * dv])


def _moments3(F, VX, VY, VZ, dv):
    return np.array([F.sum() * dv, (VX * F).sum() * dv, (VY * F).sum() * dv, (VZ * F).sum() * dv,
                     (0.5 * (VX ** 2 + VY ** 2 + VZ ** 2) * F).sum() * dv])


def _mixture2(VX, VY):
    f = _m2(0.7, 0.6, -0.3, 0.9, VX, VY) + _m2(0.5, -0.4, 0.5, 1.4, VX, VY)
    g = 0.45 * _m2(0.7, 0.6, -0.3, 0.9, VX, VY) + 0.7 * _m2(0.5, -0.4, 0.5, 1.4, VX, VY)
    return f, g


COARSE2 = dict(nvx=8, nvy=8, vxmin=-4.0, vxmax=4.0, vymin=-4.0, vymax=4.0)


def test_discrete_moments_of_the_equilibrium_equal_the_state_2d():
    """The defining equations: moments 1, v, |v|^2/2 (+ g) of the discrete
    equilibrium M, T/2 M at the returned parameters equal the state's, on a
    coarse 8^2 grid on [-4, 4)^2 (dv = 1) where the direct moments miss by
    more than 1e-3.  Catches a dropped g term, a wrong energy weight or a
    wrong Jacobian that stops Newton short."""
    cfg = W.base2d(1, 1, 8, 4.0, conservative=1)
    VX, VY, dv = _grid2(cfg)
    f, g = _mixture2(VX, VY)
    par, it, rc = oracle.equilibrium_params(cfg, np.concatenate([f, g]))
    assert rc == 0 and 2 <= it <= 12, (rc, it)
    r, ux, uy, _, T = par
    M = _m2(r, ux, uy, T, VX, VY)
    want = _moments2(f, g, VX, VY, dv)
    got = _moments2(M, T / 2 * M, VX, VY, dv)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), (got, want)
    # the direct moments' Maxwellian does not conserve on this grid
    dpar, _, _ = oracle.equilibrium_params(dict(cfg, conservative=0), np.concatenate([f, g]))
    Md = _m2(dpar[0], dpar[1], dpar[2], dpar[4], VX, VY)
    miss = np.abs(_moments2(Md, dpar[4] / 2 * Md, VX, VY, dv) - want).max() / np.abs(want).max()
    assert miss > 1e-3, miss


def test_discrete_moments_of_the_equilibrium_equal_the_state_3d():
    cfg = W.base3d(1, 6, 3.0, conservative=1)
    VX, VY, VZ, dv = _grid3(cfg)
    F = _m3(0.8, 0.5, -0.2, 0.3, 0.9, VX, VY, VZ) + _m3(0.4, -0.6, 0.4, 0.0, 1.3, VX, VY, VZ)
    par, it, rc = oracle.equilibrium_params(cfg, F)
    assert rc == 0 and it >= 2
    M = _m3(par[0], par[1], par[2], par[3], par[4], VX, VY, VZ)
    want = _moments3(F, VX, VY, VZ, dv)
    got = _moments3(M, VX, VY, VZ, dv)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), (got, want)


@pytest.mark.parametrize("dim", [2, 3])
def test_discrete_maxwellian_is_its_own_equilibrium(dim):
    """A state that is itself a discrete Maxwellian M[rho, u, T] on a coarse
    grid has the conservative parameters (rho, u, T) exactly (the root is
    unique), while its direct moments differ."""
    rho, u, T = 1.3, (0.4, -0.25, 0.15), 1.1
    if dim == 2:
        cfg = W.base2d(1, 1, 8, 4.0, conservative=1)
        VX, VY, dv = _grid2(cfg)
        M = _m2(rho, u[0], u[1], T, VX, VY)
        fk = np.concatenate([M, T / 2 * M])
        want = np.array([rho, u[0], u[1], 0.0, T])
    else:
        cfg = W.base3d(1, 6, 3.0, conservative=1)
        VX, VY, VZ, dv = _grid3(cfg)
        fk = _m3(rho, *u, T, VX, VY, VZ)
        want = np.array([rho, *u, T])
    par, _, rc = oracle.equilibrium_params(cfg, fk)
    assert rc == 0
    assert np.abs(par - want).max() <= 1e-13, par - want
    dpar, _, _ = oracle.equilibrium_params(dict(cfg, conservative=0), fk)
    assert np.abs(dpar - want).max() > 1e-4


def test_wide_fine_grid_gives_the_direct_moments():
    """On a wide fine grid the discrete moments of a Maxwellian are exact to
    round-off, so the conservative parameters equal the direct moments."""
    cfg = W.base2d(1, 1, 64, 10.0, conservative=1)
    VX, VY, dv = _grid2(cfg)
    f, g = _mixture2(VX, VY)
    fk = np.concatenate([f, g])
    par, _, rc = oracle.equilibrium_params(cfg, fk)
    dpar, _, _ = oracle.equilibrium_params(dict(cfg, conservative=0), fk)
    assert rc == 0
    assert np.abs(par - dpar).max() <= 1e-12


def _periodic_box(cons, time_scheme=0, dim=2):
    """A periodic box with a drifting, non-uniform gas on a coarse velocity
    grid, no obstacle."""
    if dim == 2:
        n = 12
        x = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(x, x)
        init = dict(rho=(1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)).ravel(),
                    ux=(0.5 + 0.3 * np.cos(2 * np.pi * Y)).ravel(), uy=(0.2 * np.sin(2 * np.pi * X)).ravel(),
                    uz=0.0, T=(1.0 + 0.3 * np.cos(2 * np.pi * X)).ravel())
        return W.base2d(n, n, 10, 5.0, Kn=0.02, Lref=1.0, cfl=0.5, scheme=1, init=init,
                        conservative=cons, time_scheme=time_scheme)
    n = 6
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    init = dict(rho=(1.0 + 0.3 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Z)).ravel(),
                ux=(0.4 + 0.2 * np.cos(2 * np.pi * Y)).ravel(), uy=0.0, uz=(0.2 * np.sin(2 * np.pi * X)).ravel(),
                T=(1.0 + 0.2 * np.cos(2 * np.pi * Y)).ravel())
    return W.base3d(n, 8, 4.0, Kn=0.02, Lref=1.0, cfl=0.5, scheme=1, init=init, conservative=cons,
                    time_scheme=time_scheme)


def _totals(cfg, F):
    dim = cfg.get("dim", 2)
    nc = oracle.ncells(cfg)
    if dim == 2:
        VX, VY, dv = _grid2(cfg)
        nv = VX.size
        Fv = F.reshape(nc, 2, nv)
        return sum(_moments2(Fv[k, 0], Fv[k, 1], VX, VY, dv) for k in range(nc))
    VX, VY, VZ, dv = _grid3(cfg)
    Fv = F.reshape(nc, VX.size)
    return sum(_moments3(Fv[k], VX, VY, VZ, dv) for k in range(nc))


@pytest.mark.parametrize("time_scheme", [0, 1])
@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_box_conserves_mass_momentum_energy(dim, time_scheme):
    """Periodic box, coarse velocity grid: with the conservative equilibrium
    the totals of mass, momentum and energy stay at their initial values to
    round-off over 40 steps (explicit, Eq. ExSchemeDD, and semi-implicit,
    Eq. ImpSchemeDD); with the direct moments momentum or energy drift by
    far more.  Transport is conservative by the flux form, so this pins the
    collision term."""
    drift = {}
    for cons in (1, 0):
        cfg = _periodic_box(cons, time_scheme, dim)
        F = oracle.initial_state(cfg)
        t0 = _totals(cfg, F)
        h = oracle.run(cfg, F, 40)
        assert h["status"] == 0
        t1 = _totals(cfg, F)
        scale = np.array([abs(t0[0])] + [abs(t0[0])] * dim + [abs(t0[-1])])
        drift[cons] = np.abs(t1 - t0) / scale
    assert drift[1].max() <= 2e-14, drift[1]
    assert drift[0][1:].max() > 1e-6, drift[0]


def test_homogeneous_relaxation_to_the_conservative_maxwellian():
    """Space-homogeneous explicit relaxation (Eq. ExSchemeDD): the moments
    are invariant, so the equilibrium is a fixed discrete Maxwellian M* and
    f^n = M* + (1 - dt/tau)^n (f^0 - M*), with tau from the direct density
    (the density is conserved, so it is the same at every step)."""
    cfg = W.base2d(2, 1, 8, 4.0, Kn=0.05, Lref=1.0, dt=2e-3, conservative=1)
    VX, VY, dv = _grid2(cfg)
    f, g = _mixture2(VX, VY)
    cell = np.concatenate([f, g])
    par, _, _ = oracle.equilibrium_params(cfg, cell)
    M = _m2(par[0], par[1], par[2], par[4], VX, VY)
    G = par[4] / 2 * M
    rho_direct = f.sum() * dv
    F = np.concatenate([cell, cell])
    n = 50
    h = oracle.run(cfg, F, n)
    assert h["status"] == 0
    tau = math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2) / rho_direct
    lam = (1 - cfg["dt"] / tau) ** n
    nv = VX.size
    np.testing.assert_allclose(F[:nv], M + lam * (f - M), rtol=0, atol=1e-13 * f.max())
    np.testing.assert_allclose(F[nv:2 * nv], G + lam * (g - G), rtol=0, atol=1e-13 * g.max())


def test_conservative_equilibrium_is_bgk_only():
    """The conservative parameters are defined here for the BGK model; the
    oracle refuses the Shakhov model with them, and the adjoint."""
    cfg = _periodic_box(1)
    cfg.update(model=1, Pr=2.0 / 3.0)
    F = oracle.initial_state(cfg)
    assert oracle.run(cfg, F, 1)["status"] != 0
