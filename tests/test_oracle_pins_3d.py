"""Pins of the 3D part of the FP64 CPU oracle (Sec. 5: full distribution F,
seven-face virtual cells) against facts fixed by the paper and by
mathematics, independent of the oracle's own code.  CPU only.

The strongest pin ties the 3D oracle to the (separately pinned) 2D reduced
one: a cylinder extruded along one axis, with periodic data along it, must
reproduce the 2D reduced-model run once F is reduced over the extruded
velocity component (Sec. 2.2 defines the reduced pair f, g exactly that
way).
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_1503_04544_gb300 import workloads as W

GAS, CUT, SOLID = 0, 1, 2


def _axis(cfg, d):
    n = cfg["nv" + d]
    dv = (cfg["v%smax" % d] - cfg["v%smin" % d]) / n
    return cfg["v%smin" % d] + np.arange(n) * dv, dv


def _vgrid3(cfg):
    vx, dx = _axis(cfg, "x")
    vy, dy = _axis(cfg, "y")
    vz, dz = _axis(cfg, "z")
    VZ, VY, VX = np.meshgrid(vz, vy, vx, indexing="ij")   # p = (p3*nvy + p2)*nvx + p1
    return VX.ravel(), VY.ravel(), VZ.ravel(), dx * dy * dz


def _maxw3d(rho, u, T, VX, VY, VZ):
    # textbook 3D Gaussian used only to build inputs and closed forms
    return rho / (2 * np.pi * T) ** 1.5 * np.exp(
        -((VX - u[0]) ** 2 + (VY - u[1]) ** 2 + (VZ - u[2]) ** 2) / (2 * T))


def _shoelace(pts):
    x, y = np.array(pts).T
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def _face_polygon_area(p, h1, h2):
    """Gas area of a face with nodal values p = (p00, p10, p11, p01) in
    counter-clockwise order, the boundary interpolated linearly on the
    edges: the shoelace area of the clipped square."""
    corners = [(0.0, 0.0), (h1, 0.0), (h1, h2), (0.0, h2)]
    pts = []
    for q in range(4):
        a, b = p[q], p[(q + 1) % 4]
        p0, p1 = corners[q], corners[(q + 1) % 4]
        if a > 0:
            pts.append(p0)
        if (a > 0) != (b > 0):
            s = a / (a - b)
            pts.append((p0[0] + s * (p1[0] - p0[0]), p0[1] + s * (p1[1] - p0[1])))
    return _shoelace(pts) if len(pts) >= 3 else 0.0


# ------------------------------------------------------------ geometry
def test_3d_geometry_identities_sphere():
    """Seven-face virtual cells (Sec. 5, built from Appendix A face by face):
    gas cells have full faces and volume dx dy dz exactly, solid cells have
    nothing; on cut cells every face area equals the shoelace area of the
    face square clipped by the linearly interpolated boundary, the wall face
    closes the polyhedron (sum_f A_f n_f + S_w n_w = 0), n_w points into the
    solid (the level set decreases along it) and the volume lies in
    (0, dx dy dz]."""
    n = 20
    cfg = W.base3d(n, 4, 4.0, shape=3, ra=0.31, cx=0.503, cy=0.49, cz=0.512)
    g = oracle.geometry3d(cfg)
    assert g["status"] == 0
    h = 1.0 / n
    phi = g["phi"].reshape(n + 1, n + 1, n + 1)        # [c][b][a]
    ax = g["ax"].reshape(n, n, n + 1)                  # [k][j][a]
    ay = g["ay"].reshape(n, n + 1, n)                  # [k][b][i]
    az = g["az"].reshape(n + 1, n, n)                  # [c][j][i]
    t = g["type"].reshape(n, n, n)
    ncut = 0
    for k in range(n):
        for j in range(n):
            for i in range(n):
                q = (k * n + j) * n + i
                A = (ax[k, j, i], ax[k, j, i + 1], ay[k, j, i], ay[k, j + 1, i], az[k, j, i], az[k + 1, j, i])
                if t[k, j, i] == GAS:
                    assert A == (h * h,) * 6 and g["sw"][q] == 0 and g["vol"][q] == h * h * h
                    continue
                if t[k, j, i] == SOLID:
                    assert A == (0.0,) * 6 and g["sw"][q] == 0 and g["vol"][q] == 0
                    continue
                ncut += 1
                P = lambda a, b, c: phi[k + c, j + b, i + a]
                faces = [
                    (A[0], (P(0, 0, 0), P(0, 1, 0), P(0, 1, 1), P(0, 0, 1))),
                    (A[1], (P(1, 0, 0), P(1, 1, 0), P(1, 1, 1), P(1, 0, 1))),
                    (A[2], (P(0, 0, 0), P(1, 0, 0), P(1, 0, 1), P(0, 0, 1))),
                    (A[3], (P(0, 1, 0), P(1, 1, 0), P(1, 1, 1), P(0, 1, 1))),
                    (A[4], (P(0, 0, 0), P(1, 0, 0), P(1, 1, 0), P(0, 1, 0))),
                    (A[5], (P(0, 0, 1), P(1, 0, 1), P(1, 1, 1), P(0, 1, 1))),
                ]
                for area, p in faces:
                    assert abs(area - _face_polygon_area(p, h, h)) < 1e-13 * h * h
                nw = np.array([g["nwx"][q], g["nwy"][q], g["nwz"][q]])
                clos = np.array([A[1] - A[0], A[3] - A[2], A[5] - A[4]]) + g["sw"][q] * nw
                assert np.abs(clos).max() < 1e-15
                grad = np.array([
                    (P(1, 0, 0) + P(1, 1, 0) + P(1, 0, 1) + P(1, 1, 1)) - (P(0, 0, 0) + P(0, 1, 0) + P(0, 0, 1) + P(0, 1, 1)),
                    (P(0, 1, 0) + P(1, 1, 0) + P(0, 1, 1) + P(1, 1, 1)) - (P(0, 0, 0) + P(1, 0, 0) + P(0, 0, 1) + P(1, 0, 1)),
                    (P(0, 0, 1) + P(1, 0, 1) + P(0, 1, 1) + P(1, 1, 1)) - (P(0, 0, 0) + P(1, 0, 0) + P(0, 1, 0) + P(1, 1, 0))])
                if g["sw"][q] > 0:
                    assert abs(np.linalg.norm(nw) - 1) < 1e-14
                    assert nw @ grad < 0
                assert 0 < g["vol"][q] <= h ** 3 * (1 + 1e-14)
    assert ncut > 100


def test_3d_volume_and_wall_area_converge_second_order():
    """Sum of virtual-cell volumes -> 1 - 4/3 pi r^3 and sum of wall areas
    -> 4 pi r^2, both at O(h^2) (the boundary is the linear interpolant of
    an exact signed distance).  A dropped term of the divergence-theorem
    volume or a wrong wall centre would leave an O(1) or O(h) error."""
    ev, ea = [], []
    r = 0.27
    for n in (16, 32, 64):
        cfg = W.base3d(n, 2, 2.0, shape=3, ra=r, cx=0.51, cy=0.48, cz=0.505)
        g = oracle.geometry3d(cfg)
        assert g["status"] == 0
        ev.append(abs(g["vol"].sum() - (1 - 4 / 3 * math.pi * r ** 3)))
        ea.append(abs(g["sw"].sum() - 4 * math.pi * r ** 2))
    ov = [math.log2(a / b) for a, b in zip(ev[:-1], ev[1:])]
    oa = [math.log2(a / b) for a, b in zip(ea[:-1], ea[1:])]
    assert min(ov) > 1.6 and min(oa) > 1.6, (ov, oa)
    assert ev[-1] < 5e-3 * 4 / 3 * math.pi * r ** 3


def test_3d_masters_unique_and_cv_volume():
    """Sec. 3.2.3 with six faces: every non-solid cell has one master whose
    centre is in the gas and which is its own master; solid cells have none;
    merging happens; every control volume keeps a sizeable volume."""
    n = 32
    cfg = W.base3d(n, 2, 2.0, shape=3, ra=0.23, cx=0.497, cy=0.52, cz=0.49)
    g = oracle.geometry3d(cfg)
    master, rc = oracle.masters3d(cfg, g)
    assert rc == 0
    nonsolid = g["type"] != SOLID
    assert np.all(master[nonsolid] >= 0) and np.all(master[~nonsolid] == -1)
    ms = np.unique(master[nonsolid])
    assert np.all(g["cgas"][ms] == 1) and np.all(master[ms] == ms)
    S = np.zeros(n ** 3)
    np.add.at(S, master[nonsolid], g["vol"][nonsolid])
    assert S[ms].min() >= 0.3 / n ** 3
    assert np.sum(master[nonsolid] != np.nonzero(nonsolid)[0]) > 0


# ------------------------------------------------------------ relaxation, transport
def test_3d_space_homogeneous_relaxation_closed_form():
    """Full-F BGK (Sec. 2.1, Eq. eq-schema3D with no transport): a uniform
    state follows f^n = M + (1 - dt/tau)^n (f^0 - M), M the 3D Maxwellian
    rho/(2 pi T)^{3/2} exp(-|v-u|^2/2T) of the conserved moments with
    T = (2E/rho - |u|^2)/3.  Catches a wrong normalisation power, energy or
    temperature in 3D."""
    cfg = W.base3d(2, 40, 10.0, nx=2, ny=1, nz=1, Kn=0.05, Lref=1.0, dt=2e-3)
    VX, VY, VZ, dv = _vgrid3(cfg)
    r1, u1, T1 = 0.6, (0.3, 0.1, -0.2), 0.8
    r2, u2, T2 = 0.5, (-0.3, 0.2, 0.1), 1.1
    f0 = _maxw3d(r1, u1, T1, VX, VY, VZ) + _maxw3d(r2, u2, T2, VX, VY, VZ)
    rho = r1 + r2
    u = (r1 * np.array(u1) + r2 * np.array(u2)) / rho
    E = sum(r * (0.5 * np.dot(uu, uu) + 1.5 * T) for r, uu, T in ((r1, u1, T1), (r2, u2, T2)))
    T = (2 * E / rho - u @ u) / 3
    M = _maxw3d(rho, u, T, VX, VY, VZ)
    F = np.concatenate([f0, f0])
    n = 40
    h = oracle.run(cfg, F, n)
    assert h["status"] == 0
    tau = math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2) / rho
    exp = M + (1 - cfg["dt"] / tau) ** n * (f0 - M)
    for c in range(2):
        np.testing.assert_allclose(F[c * VX.size:(c + 1) * VX.size], exp, rtol=0, atol=3e-13 * f0.max())


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_3d_free_transport_exact_shift(scheme, axis):
    """Eq. eq-schema3D fluxes at CFL 1 along each axis: the velocity with
    |v_d| dt/dx_d = 1 shifts its column by one cell per step (the limited
    correction carries 1 - nu), and n steps on n periodic cells give the
    data back.  With one velocity on the other axes the step is exactly the
    CFL 1 step of that axis.  Catches a wrong velocity component per
    direction or a wrong neighbour along z."""
    n = 12
    kw = dict(nx=1, ny=1, nz=1, nvx=1, nvy=1, nvz=1, vxmin=0.0, vxmax=1.0, vymin=0.0,
              vymax=1.0, vzmin=0.0, vzmax=1.0)
    d = "xyz"[axis]
    kw["n" + d] = n
    kw["nv" + d] = 4
    kw["v%smin" % d] = -2.0
    kw["v%smax" % d] = 2.0
    cfg = W.base3d(n, 4, 2.0, Kn=1e30, cfl=1.0, scheme=scheme, **kw)
    assert abs(oracle.time_step(cfg) - (1.0 / n) / 2.0) < 1e-18
    F0 = W.uniform_random(n * 4, seed=5 + axis, lo=0.1, hi=1.0)
    F = F0.copy()
    assert oracle.run(cfg, F, 1)["status"] == 0
    # v = -2 (p = 0): cell c takes the value of cell c+1
    np.testing.assert_allclose(F.reshape(n, 4)[:, 0], np.roll(F0.reshape(n, 4)[:, 0], -1), rtol=1e-15, atol=0)
    assert oracle.run(cfg, F, n - 1)["status"] == 0
    np.testing.assert_allclose(F.reshape(n, 4)[:, 0], F0.reshape(n, 4)[:, 0], rtol=64 * 2.3e-16, atol=0)


def test_3d_upwind_difference_form_brute_force():
    """Eq. eq-schema3D on gas cells of a periodic grid equals the textbook
    upwind difference form in three directions plus dt/tau (M - F),
    evaluated here by brute force on a tiny 3 x 4 x 5 grid.  Catches swapped
    v^+/v^-, a wrong direction's velocity (the printed fluxes all use
    v_{p1}) or a missing dt in the relaxation term."""
    nx, ny, nz = 3, 4, 5
    cfg = W.base3d(nx, 6, 4.0, ny=ny, nz=nz, Kn=0.3, Lref=1.0, cfl=0.4)
    VX, VY, VZ, dv = _vgrid3(cfg)
    nv = VX.size
    rng = np.random.default_rng(8)
    base = _maxw3d(1.0, (0.2, -0.1, 0.15), 1.1, VX, VY, VZ)
    F0 = base[None, None, None, :] * (1 + 0.2 * rng.uniform(-1, 1, (nz, ny, nx, nv)))
    Fl = F0.ravel().copy()
    dt = oracle.time_step(cfg)
    assert oracle.run(cfg, Fl, 1)["status"] == 0
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    tau0 = math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2)
    exp = np.zeros_like(F0)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                f = F0[k, j, i]
                rho = f.sum() * dv
                u = np.array([(VX * f).sum(), (VY * f).sum(), (VZ * f).sum()]) * dv / rho
                E = (0.5 * (VX ** 2 + VY ** 2 + VZ ** 2) * f).sum() * dv
                T = (2 * E / rho - u @ u) / 3
                M = _maxw3d(rho, u, T, VX, VY, VZ)
                out = f.copy()
                for V, h, fm, fp in ((VX, dx, F0[k, j, (i - 1) % nx], F0[k, j, (i + 1) % nx]),
                                     (VY, dy, F0[k, (j - 1) % ny, i], F0[k, (j + 1) % ny, i]),
                                     (VZ, dz, F0[(k - 1) % nz, j, i], F0[(k + 1) % nz, j, i])):
                    out -= dt / h * (np.maximum(V, 0) * (f - fm) + np.minimum(V, 0) * (fp - f))
                exp[k, j, i] = out + dt * rho / tau0 * (M - f)
    np.testing.assert_allclose(Fl.reshape(exp.shape), exp, rtol=1e-13, atol=1e-16)


# ------------------------------------------------------------ 3D <-> 2D
def _reduce(F3, nc, nvx3, nvy3, nvz3, axis, vline, dline):
    """Reduce F over the extruded velocity component (Sec. 2.2):
    f = sum F dv_e, g = sum v_e^2/2 F dv_e, returned in the 2D layout."""
    F = F3.reshape(nc, nvz3, nvy3, nvx3)
    w = np.ones_like(vline) * dline
    w2 = 0.5 * vline ** 2 * dline
    if axis == 2:       # remaining (vx, vy): 2D p = p2*nvx + p1
        f = np.einsum("czyx,z->cyx", F, w)
        g = np.einsum("czyx,z->cyx", F, w2)
    else:               # axis x: remaining (vy, vz) become the 2D (vx, vy)
        f = np.einsum("czyx,x->czy", F, w)
        g = np.einsum("czyx,x->czy", F, w2)
    return np.stack([f.reshape(nc, -1), g.reshape(nc, -1)], axis=1).ravel()


@pytest.mark.parametrize("axis", [2, 0])
@pytest.mark.parametrize("case", ["upwind_bgk", "muscl_collisionless"])
def test_3d_extruded_cylinder_equals_2d_reduced(axis, case):
    """A cylinder extruded along z (or x), one periodic cell along the axis,
    data uniform along it: the 3D run reduced over the extruded velocity
    equals the 2D reduced-model run (Sec. 2.2) to v-quadrature error, cut
    cells, wall reflection included; so do the force and, about the z axis,
    the torque with a rotating wall.  Ties every 3D routine to the pinned 2D
    ones.

    The reduction commutes with a linear scheme, so the first-order scheme
    is compared with relaxation and a hot wall.  The limiter is nonlinear:
    it commutes with the reduction only while F stays a product
    f(x, v_2D) h(v_e) with a fixed h > 0, which holds without collisions when
    the wall and the gas have the same temperature; that case checks the
    limited fluxes and their gas masks."""
    n, nv, vw = 24, 12, 6.0
    omega = 0.7 if axis == 2 else 0.0
    if case == "upwind_bgk":
        common = dict(Kn=0.2, Lref=0.2, dt=4e-4, scheme=0, Tw=1.3, omega=omega)
    else:
        common = dict(Kn=1e30, Lref=0.2, dt=4e-4, scheme=1, Tw=1.0, omega=omega)
    c2 = W.base2d(n, n, nv, vw, shape=1, cx=0.47, cy=0.52, ra=0.17,
                  init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0), **common)
    # 3D: the extruded axis has one periodic cell and a fine velocity line
    nve, vwe = 26, 10.0
    if axis == 2:
        c3 = W.base3d(n, nv, vw, nz=1, nvz=nve, vzmin=-vwe, vzmax=vwe, shape=1, axis=2,
                      cx=0.47, cy=0.52, cz=0.5, ra=0.17,
                      init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0), **common)
    else:
        c3 = W.base3d(n, nv, vw, nx=1, nvx=nve, vxmin=-vwe, vxmax=vwe, shape=1, axis=0,
                      cx=0.5, cy=0.47, cz=0.52, ra=0.17,
                      init=dict(rho=1.0, ux=0.0, uy=0.4, uz=0.1, T=1.0), **common)
    F2 = oracle.initial_state(c2)
    F3 = oracle.initial_state(c3)
    steps = 30
    h2 = oracle.run(c2, F2, steps)
    h3 = oracle.run(c3, F3, steps)
    assert h2["status"] == 0 and h3["status"] == 0
    vline, dline = _axis(c3, "xyz"[axis])
    R = _reduce(F3, n * n, c3["nvx"], c3["nvy"], c3["nvz"], axis, vline, dline)
    m2 = oracle.moments(c2, F2)
    m2r = oracle.moments(c2, R)
    assert np.abs(R - F2).max() < 1e-11 * F2.max()
    assert np.abs(F2 - oracle.initial_state(c2)).max() > 1e-3 * F2.max()   # the flow did evolve
    for key in ("rho", "ux", "uy", "T"):
        np.testing.assert_allclose(m2r[key], m2[key], rtol=0, atol=1e-11)
    fs = np.abs(h2["Fx"]).max()
    if axis == 2:
        np.testing.assert_allclose(h3["Fx"], h2["Fx"], rtol=0, atol=1e-11 * fs)
        np.testing.assert_allclose(h3["Fy"], h2["Fy"], rtol=0, atol=1e-11 * fs)
        np.testing.assert_allclose(h3["torque"], h2["torque"], rtol=0, atol=1e-11 * fs * 0.17)
        assert np.abs(h3["Fz"]).max() < 1e-13 * fs
    else:
        np.testing.assert_allclose(h3["Fy"], h2["Fx"], rtol=0, atol=1e-11 * fs)
        np.testing.assert_allclose(h3["Fz"], h2["Fy"], rtol=0, atol=1e-11 * fs)
        assert np.abs(h3["Fx"]).max() < 1e-13 * fs


def test_3d_muscl_second_order_along_z():
    """The limited z-fluxes of Eq. eq-schema3D are second order on a smooth
    profile while the first-order ones are first order (one velocity column
    v_z = 1, collisionless).  Catches a wrong stencil or (1 - nu) factor in
    the z direction that the x/y-extruded checks cannot see."""
    def err(n, scheme):
        cfg = W.base3d(n, 1, 1.0, nx=1, ny=1, nz=n, nvx=1, nvy=1, nvz=4, vxmin=0.0, vxmax=1.0,
                       vymin=0.0, vymax=1.0, vzmin=-2.0, vzmax=2.0, Kn=1e30, scheme=scheme,
                       dt=0.4 / n)
        z = (np.arange(n) + 0.5) / n
        prof = 1.5 + np.sin(2 * np.pi * z)
        F = np.ones((n, 4))
        F[:, 3] = prof                          # v_z = -2 + 3 = 1
        F = F.ravel()
        steps = n // 2
        assert oracle.run(cfg, F, steps)["status"] == 0
        exact = 1.5 + np.sin(2 * np.pi * (z - steps * 0.4 / n))
        return np.abs(F.reshape(n, 4)[:, 3] - exact).mean()

    e1 = [err(n, 0) for n in (40, 80, 160)]
    e2 = [err(n, 1) for n in (40, 80, 160)]
    assert 0.8 < math.log2(e1[1] / e1[2]) < 1.2
    assert math.log2(e2[1] / e2[2]) > 1.6


# ------------------------------------------------------------ walls, conservation
def test_3d_free_molecular_sphere_closed_form():
    """First-step force and torque on a sphere in a uniform drifting gas
    (3D forms of Eqs. BoundaryDDv, StressTensorDD, eq-force, eq-torque, with
    a rotating wall u_w = omega e_z x (r - c)) equal the continuous
    free-molecular closed form summed over the wall facets, up to the
    velocity-quadrature error.  Per facet with unit normal n into the body:
    phi = rho I1 / sqrt(Tw / 2 pi), force = (rho I2 + phi Tw/2) n + rho I1 U_t,
    I1, I2 the first and second half-range moments of the normal velocity."""
    Phi = lambda x: 0.5 * (1 + erf(x / math.sqrt(2)))
    pdf = lambda x: math.exp(-x * x / 2) / math.sqrt(2 * math.pi)
    U, rho, T, om, Tw = np.array([0.7, -0.2, 0.3]), 1.3, 0.9, 0.4, 1.5
    cfg = W.base3d(16, 32, 8.0, shape=3, ra=0.3, Tw=Tw, Kn=1e6, dt=1e-9, omega=om,
                   init=dict(rho=rho, ux=U[0], uy=U[1], uz=U[2], T=T))
    g = oracle.geometry3d(cfg)
    F0 = oracle.initial_state(cfg)
    h = oracle.run(cfg, F0, 1)
    assert h["status"] == 0
    s = math.sqrt(T)
    Fc = np.zeros(3)
    tc = 0.0
    for q in np.nonzero((g["type"] == CUT) & (g["sw"] > 0))[0]:
        nn = np.array([g["nwx"][q], g["nwy"][q], g["nwz"][q]])
        r = np.array([g["rwx"][q] - cfg["cx"], g["rwy"][q] - cfg["cy"]])
        uw = np.array([-r[1] * om, r[0] * om, 0.0])
        Ur = U - uw
        Un = Ur @ nn
        Ut = Ur - Un * nn
        I1 = Un * Phi(Un / s) + s * pdf(Un / s)
        I2 = (Un ** 2 + T) * Phi(Un / s) + Un * s * pdf(Un / s)
        phiw = rho * I1 / math.sqrt(Tw / (2 * math.pi))
        f = ((rho * I2 + phiw * Tw / 2) * nn + rho * I1 * Ut) * g["sw"][q]
        Fc += f
        tc += r[0] * f[1] - r[1] * f[0]
    got = np.array([h["Fx"][0], h["Fy"][0], h["Fz"][0]])
    assert got[0] > 0
    assert np.abs(got - Fc).max() < 2e-3 * np.abs(Fc).max(), (got, Fc)
    assert abs(h["torque"][0] - tc) < 2e-3 * np.abs(Fc).max() * cfg["ra"]
    assert np.sign(h["torque"][0]) == np.sign(tc)


def test_3d_uniform_equilibrium_preserved_and_zero_drag():
    """A rest Maxwellian with T_w = T around a sphere is a steady state
    (phi = rho, the virtual cells close, relaxation vanishes) with zero net
    force.  Catches non-closure of the seven-face flux balance."""
    rho, T = 1.4, 1.2
    cfg = W.base3d(12, 24, 10.0, shape=3, ra=0.27, Tw=T, Kn=0.1, scheme=1,
                   init=dict(rho=rho, ux=0.0, uy=0.0, uz=0.0, T=T))
    F0 = oracle.initial_state(cfg)
    F = F0.copy()
    h = oracle.run(cfg, F, 3)
    assert h["status"] == 0
    assert np.abs(F - F0).max() <= 1e-13 * F0.max()
    assert max(abs(h["Fx"][0]), abs(h["Fy"][0]), abs(h["Fz"][0])) < 1e-12


def test_3d_mass_conservation_closed_box():
    """Sec. 3.4.2 in 3D: with diffuse walls and periodic sides the total mass
    is conserved to round-off (drifting gas, hot sphere, MUSCL, merged
    control volumes); dv = 0.8 makes the discrete moments of the direct
    Maxwellian exact to ~1e-14, so relaxation conserves mass too."""
    cfg = W.base3d(12, 20, 8.0, shape=3, ra=0.25, Tw=1.3, Kn=0.1, scheme=1,
                   init=dict(rho=1.0, ux=0.4, uy=0.1, uz=-0.2, T=1.0))
    F = oracle.initial_state(cfg)
    M0 = oracle.mass3d(cfg, F)
    h = oracle.run(cfg, F, 12)
    assert h["status"] == 0
    assert np.abs(h["mass"] - M0).max() / M0 < 1e-13
    assert F.min() >= 0.0
