"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code.  CPU only.

Each test names the passage or the closed form it pins and the kind of
mistake it would catch.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_1503_04544_gb300 import workloads as W

GAS, CUT, SOLID = 0, 1, 2


def _maxw2d(rho, ux, uy, T, vx, vy):
    # textbook 2D Gaussian used only to build inputs and closed forms
    return rho / (2 * np.pi * T) * np.exp(-((vx - ux) ** 2 + (vy - uy) ** 2) / (2 * T))


def _vgrid(cfg):
    dvx = (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]
    dvy = (cfg["vymax"] - cfg["vymin"]) / cfg["nvy"]
    vx = cfg["vxmin"] + np.arange(cfg["nvx"]) * dvx
    vy = cfg["vymin"] + np.arange(cfg["nvy"]) * dvy
    VX, VY = np.meshgrid(vx, vy)          # p = p2*nvx + p1
    return VX.ravel(), VY.ravel(), dvx * dvy


# ------------------------------------------------------------ relaxation
def test_space_homogeneous_relaxation_closed_form():
    """BGK relaxation (Sec. 2.1, Eq. BGKDD, Eq. ExSchemeDD): in a uniform
    state the scheme reduces to f^{n+1} = f^n + dt/tau (M - f^n), whose
    solution is f^n = M + (1 - dt/tau)^n (f^0 - M) with M the Maxwellian of
    the (conserved) moments.  Catches errors in the moments, T, tau(rho),
    the reduced equilibria f_eq = M, g_eq = T/2 M and the update."""
    cfg = W.base2d(2, 1, 32, 10.0, Kn=0.05, Lref=1.0, dt=2e-3)
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
    n = 60
    h = oracle.run(cfg, F, n)
    assert h["status"] == 0
    tau = math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2) / rho
    lam = (1 - cfg["dt"] / tau) ** n
    fexp = M + lam * (f0 - M)
    gexp = G + lam * (g0 - G)
    nv = VX.size
    for c in range(2):
        got = F[c * 2 * nv: (c + 1) * 2 * nv]
        np.testing.assert_allclose(got[:nv], fexp, rtol=0, atol=1e-13 * f0.max())
        np.testing.assert_allclose(got[nv:], gexp, rtol=0, atol=1e-13 * g0.max())


# ------------------------------------------------------------ transport
@pytest.mark.parametrize("scheme", [0, 1])
def test_free_transport_exact_shift(scheme):
    """Upwind flux (Eq. FluxDD) at CFL 1: the column with nu = |v| dt/dx = 1
    shifts by exactly one cell per step (also for the limited scheme, whose
    correction carries a factor 1 - nu).  32 steps on 32 periodic cells give
    back the initial data.  Catches a wrong upwind side or neighbour index."""
    nx = 32
    cfg = W.base2d(nx, 1, 16, 8.0, Kn=1e30, dt=(1.0 / nx) / 8.0, scheme=scheme)
    VX, VY, dv = _vgrid(cfg)
    nv = VX.size
    F0 = W.uniform_random(nx * 2 * nv, seed=7, lo=0.1, hi=1.0)
    F = F0.copy()
    h = oracle.run(cfg, F, 1)
    assert h["status"] == 0
    col = np.nonzero(VX == -8.0)[0]
    F0v = F0.reshape(nx, 2, nv)
    F1v = F.reshape(nx, 2, nv)
    # one step: cell i takes the value of cell i+1 for v_x = -8
    np.testing.assert_allclose(F1v[:, :, col], np.roll(F0v, -1, axis=0)[:, :, col], rtol=4e-16 * 8, atol=0)
    oracle.run(cfg, F, nx - 1)
    np.testing.assert_allclose(F.reshape(nx, 2, nv)[:, :, col], F0v[:, :, col], rtol=64 * 2.3e-16, atol=0)


def test_upwind_difference_form_brute_force():
    """Eqs. ExSchemeDD + FluxDD on gas cells of a periodic grid equal the
    textbook upwind difference form
      f_i - dt/dx [v^+ (f_i - f_{i-1}) + v^- (f_{i+1} - f_i)] - (y terms)
          + dt/tau (M - f_i),
    evaluated here by brute force on a tiny grid.  Catches swapped v^+/v^-
    or neighbour indices and a wrong area factor."""
    nx, ny = 5, 4
    cfg = W.base2d(nx, ny, 6, 4.0, Kn=0.3, Lref=1.0, cfl=0.4)
    VX, VY, dv = _vgrid(cfg)
    nv = VX.size
    rng = np.random.default_rng(3)
    # random but positive cell states near a Maxwellian
    base = _maxw2d(1.0, 0.2, -0.1, 1.1, VX, VY)
    F = np.zeros((ny, nx, 2, nv))
    for j in range(ny):
        for i in range(nx):
            F[j, i, 0] = base * (1 + 0.2 * rng.uniform(-1, 1, nv))
            F[j, i, 1] = 0.55 * base * (1 + 0.2 * rng.uniform(-1, 1, nv))
    F0 = F.copy()
    Fl = F.ravel().copy()
    dt = oracle.time_step(cfg)
    assert oracle.run(cfg, Fl, 1)["status"] == 0
    dx, dy = 1.0 / nx, 1.0 / ny
    tau0 = math.sqrt(math.pi) / 2 * cfg["Kn"] * cfg["Lref"] / math.sqrt(2)
    vp, vm = np.maximum(VX, 0), np.minimum(VX, 0)
    wp, wm = np.maximum(VY, 0), np.minimum(VY, 0)
    exp = np.zeros_like(F0)
    for j in range(ny):
        for i in range(nx):
            f = F0[j, i]
            rho = f[0].sum() * dv
            ux = (VX * f[0]).sum() * dv / rho
            uy = (VY * f[0]).sum() * dv / rho
            E = (0.5 * (VX ** 2 + VY ** 2) * f[0] + f[1]).sum() * dv
            T = (2 * E / rho - ux ** 2 - uy ** 2) / 3
            M = _maxw2d(rho, ux, uy, T, VX, VY)
            eq = np.stack([M, T / 2 * M])
            fl, fr = F0[j, (i - 1) % nx], F0[j, (i + 1) % nx]
            fd, fu = F0[(j - 1) % ny, i], F0[(j + 1) % ny, i]
            exp[j, i] = (f - dt / dx * (vp * (f - fl) + vm * (fr - f))
                         - dt / dy * (wp * (f - fd) + wm * (fu - f))
                         + dt * rho / tau0 * (eq - f))
    np.testing.assert_allclose(Fl.reshape(exp.shape), exp, rtol=1e-13, atol=1e-15)


def _tv(a):
    return np.abs(np.diff(np.concatenate([a, a[:1]]))).sum()


def test_muscl_tvd_and_second_order():
    """Limited scheme (reading of the second-order extension): for linear
    advection it is total-variation diminishing on random data and
    second-order accurate on a smooth profile, while first-order upwind is
    first order.  Catches a wrong sign of the (1 - nu) correction, a
    misplaced minmod argument or an upwind-side error."""
    # TVD on random data, a few velocity columns, collisionless
    nx = 40
    cfg = W.base2d(nx, 1, 8, 4.0, Kn=1e30, cfl=0.5, scheme=1)
    VX, VY, dv = _vgrid(cfg)
    nv = VX.size
    F = W.uniform_random(nx * 2 * nv, seed=11, lo=0.0, hi=1.0)
    Fv = F.reshape(nx, 2, nv)
    tv0 = [_tv(Fv[:, 0, p].copy()) for p in range(nv)]
    for _ in range(10):
        oracle.run(cfg, F, 1)
        Fv = F.reshape(nx, 2, nv)
        tv1 = [_tv(Fv[:, 0, p].copy()) for p in range(nv)]
        assert all(b <= a * (1 + 1e-12) for a, b in zip(tv0, tv1))
        tv0 = tv1
        assert F.min() >= 0.0

    # order of accuracy on a smooth periodic profile, one velocity column
    def err(nx, scheme):
        cfg = W.base2d(nx, 1, 4, 2.0, Kn=1e30, scheme=scheme, dt=0.4 / nx)  # v = 1 -> nu = 0.4
        VX, VY, dv = _vgrid(cfg)
        nv = VX.size
        x = (np.arange(nx) + 0.5) / nx
        prof = 1.5 + np.sin(2 * np.pi * x)
        F = np.ones((nx, 2, nv))
        F[:, 0, :] = prof[:, None]
        F = F.ravel()
        nsteps = nx // 2                      # t = 0.2
        oracle.run(cfg, F, nsteps)
        col = np.nonzero(VX == 1.0)[0][0]
        exact = 1.5 + np.sin(2 * np.pi * (x - nsteps * 0.4 / nx))
        return np.abs(F.reshape(nx, 2, nv)[:, 0, col] - exact).mean()

    e1 = [err(n, 0) for n in (40, 80, 160)]
    e2 = [err(n, 1) for n in (40, 80, 160)]
    o1 = math.log2(e1[1] / e1[2])
    o2 = math.log2(e2[1] / e2[2])
    assert 0.8 < o1 < 1.2
    assert o2 > 1.6


# ------------------------------------------------------------ geometry
def _shoelace(pts):
    x, y = np.array(pts).T
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_geometry_identities_circle_and_ellipse():
    """Appendix A / Sec. 3.2.2 parameter table: gas cells have full edges,
    zero wall and area dx dy exactly; solid cells have everything zero.  Cut
    cells: the wall edge closes the polygon (sum |L_e| n_e = 0), the
    Green-formula area equals the shoelace area of the polygon cut by the
    linearly interpolated boundary, and n_w points into the solid (the
    level set decreases along n_w)."""
    for shape, kw in ((1, dict(ra=0.23)), (2, dict(ra=0.12, rb=0.04, theta=0.7))):
        nx = 96
        cfg = W.base2d(nx, nx, 4, 4.0, shape=shape, cx=0.503, cy=0.49, **kw)
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
                    # polygon: gas nodes and crossings in counter-clockwise order
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
                    # n_w points into the solid: phi decreases along it
                    gx = 0.5 * ((phi[j, i + 1] + phi[j + 1, i + 1]) - (phi[j, i] + phi[j + 1, i])) / dx
                    gy = 0.5 * ((phi[j + 1, i] + phi[j + 1, i + 1]) - (phi[j, i] + phi[j, i + 1])) / dy
                    assert nw @ np.array([gx, gy]) < 0
        assert ncut > 20


def test_gas_area_converges_second_order():
    """Sum of virtual-cell areas -> exact gas area 1 - pi r^2 at O(dx^2)
    (linear interpolation of an exact signed distance, Appendix A)."""
    errs = []
    for nx in (32, 64, 128, 256):
        cfg = W.base2d(nx, nx, 4, 4.0, shape=1, ra=0.27, cx=0.51, cy=0.48)
        g = oracle.geometry2d(cfg)
        errs.append(abs(g["sbar"].sum() - (1 - math.pi * 0.27 ** 2)))
    orders = [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]
    assert min(orders) > 1.6, orders


def test_masters_unique_and_cv_area():
    """Sec. 3.2.3 and Eq. (ii): every non-solid cell has exactly one master,
    the master's centre is in the gas, it is its own master, and every
    control volume has area >= dx dy / 2."""
    for shape, kw in ((1, dict(ra=0.1)), (2, dict(ra=0.12, rb=0.04, theta=0.3)),
                      (2, dict(ra=0.12, rb=0.04, theta=1.9))):
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
        assert np.sum(master[nonsolid] != np.nonzero(nonsolid)[0]) > 0   # some merging happens


# ------------------------------------------------------------ walls
def _free_molecular(cfg, g, U, rho, T, omega, Tw):
    """Closed-form half-range integrals of a drifting Maxwellian hitting a
    diffusely reflecting flat element (Sec. 2.1 Eq. BoundaryTD, Eq.
    StressTensorDD with continuous velocities), summed over wall edges."""
    Phi = lambda x: 0.5 * (1 + erf(x / math.sqrt(2)))
    pdf = lambda x: math.exp(-x * x / 2) / math.sqrt(2 * math.pi)
    F = np.zeros(2)
    tq = 0.0
    s = math.sqrt(T)
    for k in np.nonzero((g["type"] == CUT) & (g["lw"] > 0))[0]:
        n = np.array([g["nwx"][k], g["nwy"][k]])
        lwn = g["lw"][k] * np.linalg.norm(n)
        nn = n / np.linalg.norm(n)
        t = np.array([-nn[1], nn[0]])
        r = np.array([g["rwx"][k] - cfg["cx"], g["rwy"][k] - cfg["cy"]])
        uw = np.array([-r[1] * omega, r[0] * omega])
        Ur = np.asarray(U) - uw
        Un, Ut = Ur @ nn, Ur @ t
        I1 = Un * Phi(Un / s) + s * pdf(Un / s)
        I2 = (Un ** 2 + T) * Phi(Un / s) + Un * s * pdf(Un / s)
        phiw = rho * I1 / math.sqrt(Tw / (2 * math.pi))
        f = ((rho * I2 + phiw * Tw / 2) * nn + (rho * Ut * I1) * t) * lwn
        F += f
        tq += r[0] * f[1] - r[1] * f[0]
    return F, tq


@pytest.mark.parametrize("shape", [1, 2])
def test_wall_stress_free_molecular_closed_form(shape):
    """First-step force and torque (Eqs. BoundaryDDv, StressTensorDD,
    eq-force, eq-torque, uwDD) on a body in a uniform drifting gas equal the
    continuous free-molecular closed form up to the O(dv^2) error of the
    velocity quadrature.  Catches a wrong normal orientation, wrong in/out
    sets, a wrong wall velocity sign or a wrong torque arm."""
    kw = dict(ra=0.2) if shape == 1 else dict(ra=0.2, rb=0.08, theta=0.4)
    U, rho, T, om, Tw = (0.7, -0.2), 1.3, 0.9, 0.3, 1.5
    cfg = W.base2d(64, 64, 64, 10.0, shape=shape, Tw=Tw, Kn=1e6, dt=1e-9, omega=om,
                   init=dict(rho=rho, ux=U[0], uy=U[1], uz=0.0, T=T), **kw)
    g = oracle.geometry2d(cfg)
    F0 = oracle.initial_state(cfg)
    h = oracle.run(cfg, F0, 1)
    Fc, tc = _free_molecular(cfg, g, U, rho, T, om, Tw)
    assert h["Fx"][0] > 0
    assert abs(h["Fx"][0] - Fc[0]) < 5e-4 * abs(Fc[0])
    assert abs(h["Fy"][0] - Fc[1]) < 5e-4 * np.abs(Fc).max()
    # the torque is a small difference of large moments: scale by |F| * size
    assert abs(h["torque"][0] - tc) < 2e-4 * np.abs(Fc).max() * cfg["ra"]
    assert np.sign(h["torque"][0]) == np.sign(tc)


def test_uniform_equilibrium_preserved_and_zero_drag():
    """A uniform rest Maxwellian with T_w = T around a fixed body is a
    steady state of the discrete scheme (Eq. BoundaryDDv gives phi = rho on a
    symmetric velocity grid, the virtual cell closes, relaxation vanishes),
    and the net force vanishes.  Catches any non-closure of the cut-cell
    fluxes or a wall density not equal to rho."""
    rho, T = 1.7, 1.2
    cfg = W.base2d(48, 48, 24, 10.0, shape=1, ra=0.2, Tw=T, Kn=0.1, scheme=1,
                   init=dict(rho=rho, ux=0.0, uy=0.0, uz=0.0, T=T))
    F0 = oracle.initial_state(cfg)
    F = F0.copy()
    h = oracle.run(cfg, F, 5)
    assert np.abs(F - F0).max() <= 1e-14 * F0.max() * 5
    assert abs(h["Fx"][0]) < 1e-13 and abs(h["Fy"][0]) < 1e-13


# ------------------------------------------------------------ conservation
@pytest.mark.parametrize("moving", [0, 1])
def test_mass_conservation_closed_box(moving):
    """Sec. 3.4.2 (Eq. def-masse): the explicit scheme with diffuse walls
    conserves the total mass exactly, also with a moving body whose cells
    merge, appear and disappear.  Periodic box (no in/outflow), hot wall,
    drifting gas.  The velocity grid (dv = 0.625 on [-10, 10)) makes the
    discrete moments of the direct Maxwellian exact to ~1e-20, so the
    relaxation term conserves mass too (Sec. 3.1 uses a conservative
    Maxwellian for coarser grids)."""
    if moving:
        cfg = W.base2d(48, 48, 32, 10.0, shape=2, ra=0.2, rb=0.06, theta=0.3, omega=4.0,
                       movable=1, inertia=1e-2, Tw=1.3, Kn=0.1, cfl=0.5,
                       init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0))
        steps = 120
    else:
        cfg = W.base2d(48, 48, 32, 10.0, shape=1, ra=0.15, Tw=1.3, Kn=0.1, scheme=1,
                       init=dict(rho=1.0, ux=0.4, uy=0.1, uz=0.0, T=1.0))
        steps = 200
    F = oracle.initial_state(cfg)
    M0 = oracle.mass2d(cfg, F)
    h = oracle.run(cfg, F, steps)
    assert h["status"] == 0
    drift = np.abs(h["mass"] - M0).max() / M0
    assert drift < 1e-13, drift
    if moving:
        assert abs(h["theta"] - cfg["theta"]) > 0.05        # the body really turned


def test_rigid_rotation_kinematics():
    """Eq. motionDD_posit with a huge inertia (Eq. motionDD_vit gives a
    constant angular velocity): theta^n = theta^0 + n dt omega."""
    cfg = W.base2d(48, 48, 8, 6.0, shape=2, ra=0.2, rb=0.06, theta=0.1, omega=2.0,
                   movable=1, inertia=1e30, Kn=0.1)
    F = oracle.initial_state(cfg)
    h = oracle.run(cfg, F, 30)
    dt = oracle.time_step(cfg)
    exp = 0.1 + dt * 2.0 * np.arange(1, 31)
    np.testing.assert_allclose(h["theta_hist"], exp, rtol=1e-14)
    np.testing.assert_allclose(h["omega_hist"], 2.0, rtol=1e-15)


def test_rigid_rotation_ode_finite_inertia():
    """Eqs. motionDD_vit and motionDD_posit with a finite moment of inertia
    J: an ellipse that turns in a uniform drifting gas at Kn -> infinity and
    dt -> 0, where the torque of the first step is the continuous
    free-molecular torque (closed form, the pin of
    test_wall_stress_free_molecular_closed_form).  Then
      omega^1 = omega^0 + dt T^0 / J     (torque at t^n, divided by J),
      theta^1 = theta^0 + dt omega^0     (explicit Euler, the old omega),
    and every later step follows the same recurrence with the torque the
    step reports.  dt / J = 20, so the first step changes omega by more than
    its initial value: a sign flip of the torque term, J swapped with the
    mass (m = 1 here), the torque of t^{n+1} or theta advanced with the new
    omega all fail.  (The torque falls as omega grows, dT/domega ~ -0.02, so
    the explicit recurrence converges towards the omega of zero torque.)"""
    U, rho, T, Tw = (0.7, -0.2), 1.3, 0.9, 1.5
    om0, th0, dt = 0.05, 0.4, 1e-9
    J = dt / 20.0
    cfg = W.base2d(64, 64, 64, 10.0, shape=2, ra=0.2, rb=0.08, theta=th0, omega=om0, movable=1,
                   mass=1.0, inertia=J, Tw=Tw, Kn=1e6, dt=dt,
                   init=dict(rho=rho, ux=U[0], uy=U[1], uz=0.0, T=T))
    _, tc = _free_molecular(cfg, oracle.geometry2d(cfg), U, rho, T, om0, Tw)
    F = oracle.initial_state(cfg)
    n = 6
    h = oracle.run(cfg, F, n)
    assert h["status"] == 0
    om, th, tq = h["omega_hist"], h["theta_hist"], h["torque"]
    # first step against the closed-form torque, within its O(dv^2)
    # quadrature bound (2e-4 |F| size) scaled by dt / J
    tol = dt / J * 2e-4 * 0.9 * cfg["ra"]
    assert abs(om[0] - (om0 + dt * tc / J)) < tol, (om[0], om0 + dt * tc / J)
    assert om[0] - om0 > 0.06
    assert th[0] == th0 + dt * om0
    # the recurrence over the following steps, with the torque each reports
    for k in range(1, n):
        assert abs(om[k] - (om[k - 1] + dt * tq[k] / J)) <= 1e-14 * abs(om[k]), k
        assert th[k] == th[k - 1] + dt * om[k - 1], k
    # omega changes at every step (the torque term is live)
    assert np.abs(np.diff(om)).min() > 0.005


def test_positivity_under_cfl():
    """Sec. 3.4.1: the explicit scheme keeps f >= 0 under the CFL condition,
    including cut and merged cells (Mach-2 cylinder, strong gradients)."""
    cfg = W.cylinder_mach2(nx=48, nv=16)
    F = oracle.initial_state(cfg)
    for _ in range(4):
        assert oracle.run(cfg, F, 10)["status"] == 0
        assert F.min() >= 0.0
