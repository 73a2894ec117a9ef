"""Oracle pins of the closed containers (2D, the gas inside a disk or a box):
the Appendix A geometry of a boundary whose gas side is its inside, the
steady state of a uniform rest gas at the wall temperature, and exact mass
conservation with a hot diffuse wall (Sec. 3.4.2, Eq. def-masse).  CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import workloads as W

GAS, CUT, SOLID = 0, 1, 2


def _shoelace(pts):
    a = 0.0
    for q in range(len(pts)):
        (x0, y0), (x1, y1) = pts[q], pts[(q + 1) % len(pts)]
        a += x0 * y1 - x1 * y0
    return 0.5 * a


def _check_identities(cfg):
    """Full gas cells: full edges, no wall, area dx dy; solid cells: all
    zero; cut cells: the wall edge closes the polygon, the Green-formula
    area equals the shoelace area of the polygon cut by the interpolated
    boundary, and n_w points into the solid.  Returns the number of cut
    cells."""
    nx = cfg["nx"]
    g = oracle.geometry2d(cfg)
    assert g["status"] == 0
    dx = dy = 1.0 / nx
    lx = g["lx"].reshape(nx, nx + 1)
    ly = g["ly"].reshape(nx + 1, nx)
    phi = g["phi"].reshape(nx + 1, nx + 1)
    t = g["type"].reshape(nx, nx)
    ncut = 0
    for j in range(nx):
        for i in range(nx):
            k = j * nx + i
            L = (lx[j, i], lx[j, i + 1], ly[j, i], ly[j + 1, i])
            if t[j, i] == GAS:
                assert L == (dy, dy, dx, dx) and g["lw"][k] == 0 and g["sbar"][k] == dx * dy
            elif t[j, i] == SOLID:
                assert L == (0, 0, 0, 0) and g["lw"][k] == 0 and g["sbar"][k] == 0
            else:
                ncut += 1
                lw, nw = g["lw"][k], np.array([g["nwx"][k], g["nwy"][k]])
                clos = np.array([L[1] - L[0], L[3] - L[2]]) + lw * nw
                assert np.abs(clos).max() < 1e-15
                corners = [((0, 0), phi[j, i]), ((dx, 0), phi[j, i + 1]),
                           ((dx, dy), phi[j + 1, i + 1]), ((0, dy), phi[j + 1, i])]
                pts = []
                for q in range(4):
                    (p0, a), (p1, b) = corners[q], corners[(q + 1) % 4]
                    if a > 0:
                        pts.append(p0)
                    if (a > 0) != (b > 0):
                        s = a / (a - b)
                        pts.append((p0[0] + s * (p1[0] - p0[0]), p0[1] + s * (p1[1] - p0[1])))
                assert abs(_shoelace(pts) - g["sbar"][k]) < 1e-12 * dx * dy
                gx = 0.5 * ((phi[j, i + 1] + phi[j + 1, i + 1]) - (phi[j, i] + phi[j + 1, i])) / dx
                gy = 0.5 * ((phi[j + 1, i] + phi[j + 1, i + 1]) - (phi[j, i] + phi[j, i + 1])) / dy
                assert nw @ np.array([gx, gy]) < 0
    return g, ncut


@pytest.mark.parametrize("shape,kw", [(4, dict(ra=0.4312, cx=0.503, cy=0.49)),
                                      (5, dict(ra=0.41, rb=0.33, cx=0.5013, cy=0.4987))])
def test_container_geometry_identities(shape, kw):
    """Appendix A with the gas inside: the per-cell identities hold, the
    cells at the domain's corners are solid and the centre is gas."""
    cfg = W.base2d(96, 96, 4, 4.0, shape=shape, **kw)
    g, ncut = _check_identities(cfg)
    t = g["type"].reshape(96, 96)
    assert t[0, 0] == SOLID and t[95, 95] == SOLID and t[48, 48] == GAS
    assert ncut > 40


def test_container_areas():
    """The gas area of the disk container converges to pi r^2 at second
    order; the box container's is exact but for its four corner cells (the
    interpolated level set is exact along the straight sides)."""
    errs = []
    for nx in (32, 64, 128, 256):
        cfg = W.base2d(nx, nx, 4, 4.0, shape=4, ra=0.37, cx=0.51, cy=0.48)
        g = oracle.geometry2d(cfg)
        errs.append(abs(g["sbar"].sum() - math.pi * 0.37 ** 2))
    orders = [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]
    assert min(orders) > 1.6, orders
    nx = 128
    cfg = W.base2d(nx, nx, 4, 4.0, shape=5, ra=0.41, rb=0.33, cx=0.5013, cy=0.4987)
    g = oracle.geometry2d(cfg)
    assert abs(g["sbar"].sum() - 4 * 0.41 * 0.33) < 4 * (1.0 / nx) ** 2


@pytest.mark.parametrize("shape,kw", [(4, dict(ra=0.45)), (5, dict(ra=0.41, rb=0.33))])
def test_container_masters(shape, kw):
    """Sec. 3.2.3: one master per non-solid cell, a gas-centred master that is
    its own master, control volumes of area >= dx dy / 2."""
    nx = 128
    cfg = W.base2d(nx, nx, 4, 4.0, shape=shape, **kw)
    g = oracle.geometry2d(cfg)
    master, rc = oracle.masters2d(cfg, g)
    assert rc == 0
    nonsolid = g["type"] != SOLID
    assert np.all(master[nonsolid] >= 0) and np.all(master[~nonsolid] == -1)
    ms = np.unique(master[nonsolid])
    assert np.all(g["cgas"][ms] == 1) and np.all(master[ms] == ms)
    S = np.zeros(nx * nx)
    np.add.at(S, master[nonsolid], g["sbar"][nonsolid])
    assert S[ms].min() >= 0.5 / nx ** 2


@pytest.mark.parametrize("shape,kw", [(4, dict(ra=0.45)), (5, dict(ra=0.41, rb=0.33))])
def test_container_uniform_equilibrium_preserved(shape, kw):
    """A uniform rest Maxwellian at T = T_w in a closed container is a steady
    state of the scheme (phi = rho on the symmetric velocity grid, the
    virtual cells close, relaxation vanishes), and the net force on the
    closed wall vanishes."""
    rho, T = 1.7, 1.2
    cfg = W.base2d(48, 48, 24, 10.0, shape=shape, Tw=T, Kn=0.1, scheme=1,
                   init=dict(rho=rho, ux=0.0, uy=0.0, uz=0.0, T=T), **kw)
    F0 = oracle.initial_state(cfg)
    F = F0.copy()
    h = oracle.run(cfg, F, 5)
    assert h["status"] == 0
    assert np.abs(F - F0).max() <= 1e-14 * F0.max() * 5
    assert abs(h["Fx"][0]) < 1e-13 and abs(h["Fy"][0]) < 1e-13


@pytest.mark.parametrize("which", ["disk", "box"])
def test_container_mass_conservation(which):
    """Sec. 3.4.2 (Eq. def-masse): with a hot diffuse wall (T_w = 1.3) the
    explicit scheme keeps the total mass in the container exactly; the gas
    moves (a density bump, and a drift in the box).  The velocity grid
    (dv = 0.625 on [-10, 10)) makes the direct Maxwellian's discrete mass
    exact to round-off."""
    mk = W.disk_container if which == "disk" else W.box_container
    cfg = mk(nx=48, nv=32)
    cfg.update(vxmin=-10.0, vxmax=10.0, vymin=-10.0, vymax=10.0)
    F = oracle.initial_state(cfg)
    M0 = oracle.mass2d(cfg, F)
    h = oracle.run(cfg, F, 150)
    assert h["status"] == 0
    drift = np.abs(h["mass"] - M0).max() / M0
    assert drift < 1e-13, drift
    # the gas did change: the wall heats it
    m = oracle.moments(cfg, F)
    live = m["rho"] > 0
    assert m["T"][live].max() > 1.01
