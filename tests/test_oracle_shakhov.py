"""Pins of the oracle's Shakhov collision model (Eq. ShakhovDD for the
reduced 2D (f, g) model; the 3D form of Sec. 2.1), against facts that do not
come from the oracle's own formulas:

- the defining moments of the Shakhov equilibrium: the mass, momentum and
  energy of the Maxwellian, and the heat flux (1 - Pr) q (2D and 3D), met by
  the discrete equilibrium on a wide, fine velocity grid to quadrature error;
- the reduction of the 3D equilibrium: integrating it over v_z (and v_z^2/2
  times it) gives the reduced f and g of Eq. ShakhovDD, which fixes the
  constants -4 and -2 and the factor T/2 independently of the 2D formula;
- Pr = 1 is the BGK model bit for bit (2D cylinder, 3D sphere);
- in a homogeneous gas the explicit scheme (Eq. ExSchemeDD) leaves rho, u
  and T fixed and multiplies the heat flux by 1 - Pr dt/tau each step
  (the Prandtl number of the model); BGK gives 1 - dt/tau;
- under the semi-implicit scheme (Eq. ImpSchemeDD) the heat flux is divided
  by 1 + Pr dt/tau each step (the reading q^{n+1} = q_T / (1 + nu Pr)), Pr = 1
  is the semi-implicit BGK scheme bit for bit, and a very stiff step lands on
  the Maxwellian of the transported moments.
"""
import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import workloads as W

CASES = [(1.2, (0.4, -0.3, 0.2), 1.3, (0.2, -0.15, 0.1)),
         (0.7, (-0.5, 0.1, -0.2), 0.8, (-0.05, 0.12, 0.03))]


def one_cell(dim, nv, win, **kw):
    if dim == 2:
        return W.base2d(1, 1, nv, win, **kw)
    return W.base3d(1, nv, win, **kw)


def velocity_axis(cfg, ax):
    n = cfg["nv" + ax]
    lo, hi = cfg["v" + ax + "min"], cfg["v" + ax + "max"]
    return lo + np.arange(n) * ((hi - lo) / n)


@pytest.mark.parametrize("dim,nv,win", [(2, 112, 12.0), (3, 56, 11.0)])
@pytest.mark.parametrize("Pr", [2.0 / 3.0, 0.3])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_equilibrium_moments(dim, nv, win, Pr, case):
    rho, u, T, q = CASES[case]
    u, q = u[:dim], q[:dim]
    cfg = one_cell(dim, nv, win, model=1, Pr=Pr)
    fk = oracle.equilibrium(cfg, rho, u, T, q)
    m = oracle.moments(cfg, fk)
    assert abs(m["rho"][0] - rho) < 1e-12 * rho
    got_u = [m["ux"][0], m["uy"][0], m["uz"][0]][:dim]
    assert np.allclose(got_u, u, rtol=0, atol=1e-12)
    assert abs(m["T"][0] - T) < 1e-12 * T
    qe, rc = oracle.heat_flux(cfg, fk)
    assert rc == 0
    assert np.allclose(qe[:dim], (1.0 - Pr) * np.asarray(q), rtol=0, atol=1e-12)
    # BGK: no heat flux at equilibrium
    qb, _ = oracle.heat_flux(cfg, oracle.equilibrium(dict(cfg, model=0), rho, u, T, q))
    assert np.abs(qb).max() < 1e-12


@pytest.mark.parametrize("case", range(len(CASES)))
def test_reduced_equilibrium_is_the_3d_one_integrated_over_vz(case):
    rho, u, T, q = CASES[case]
    u2, q2 = (u[0], u[1]), (q[0], q[1])
    nv, win = 40, 8.0
    c2 = one_cell(2, nv, win, model=1, Pr=2.0 / 3.0)
    c3 = one_cell(3, nv, win, model=1, Pr=2.0 / 3.0, nvz=72, vzmin=-9.0, vzmax=9.0)
    F = oracle.equilibrium(c3, rho, (u[0], u[1], 0.0), T, (q[0], q[1], 0.0)).reshape(72, nv, nv)
    vz = velocity_axis(c3, "z")
    dvz = vz[1] - vz[0]
    f = (F * dvz).sum(axis=0)
    g = (F * (0.5 * vz ** 2 * dvz)[:, None, None]).sum(axis=0)
    e2 = oracle.equilibrium(c2, rho, u2, T, q2)
    f2, g2 = e2[: nv * nv].reshape(nv, nv), e2[nv * nv:].reshape(nv, nv)
    assert np.abs(f - f2).max() < 1e-12 * np.abs(f2).max()
    assert np.abs(g - g2).max() < 1e-12 * np.abs(g2).max()


def test_pr_one_is_bgk_2d():
    cfg = W.cylinder_mach2(nx=32, nv=12)
    F0 = oracle.initial_state(cfg)
    a, b = F0.copy(), F0.copy()
    ha = oracle.run(cfg, a, 6)
    hb = oracle.run(dict(cfg, model=1, Pr=1.0), b, 6)
    assert ha["status"] == 0 and hb["status"] == 0
    assert np.array_equal(a, b)
    assert np.array_equal(ha["Fx"], hb["Fx"])


def test_pr_one_is_bgk_3d():
    cfg = W.sphere_mach15(n=12, nv=6)
    F0 = oracle.initial_state(cfg)
    a, b = F0.copy(), F0.copy()
    assert oracle.run3d(cfg, a, 3)["status"] == 0
    assert oracle.run3d(dict(cfg, model=1, Pr=1.0), b, 3)["status"] == 0
    assert np.array_equal(a, b)


def homogeneous(dim, Pr, model):
    """A periodic box of 2^dim cells holding one state with a heat flux."""
    nv, win = (80, 12.0) if dim == 2 else (40, 11.0)
    n = 2
    if dim == 2:
        cfg = W.base2d(n, n, nv, win, Kn=0.5, bc=[0] * 6, model=model, Pr=Pr)
    else:
        cfg = W.base3d(n, nv, win, Kn=0.5, bc=[0] * 6, model=model, Pr=Pr)
    rho, u, T, q = CASES[0]
    # the initial state: a Shakhov equilibrium of Pr = 0, whose heat flux is q
    start = oracle.equilibrium(dict(cfg, model=1, Pr=0.0), rho, u[:dim], T, q[:dim])
    F = np.tile(start, n ** dim)
    return cfg, F, start, rho


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("model,Pr", [(1, 2.0 / 3.0), (1, 0.3), (0, 1.0)])
def test_heat_flux_relaxes_at_rate_pr(dim, model, Pr):
    cfg, F, start, rho = homogeneous(dim, Pr, model)
    q0, _ = oracle.heat_flux(cfg, start)
    m0 = oracle.moments(cfg, F)
    r = oracle.time_step(cfg) * rho / oracle.tau0(cfg)     # dt / tau
    assert 0.01 < r < 0.5
    n = 12
    run = oracle.run if dim == 2 else oracle.run3d
    assert run(cfg, F, n)["status"] == 0
    nvs = F.size // (2 ** dim)
    cell0 = F[:nvs]
    assert np.array_equal(F, np.tile(cell0, 2 ** dim))        # still homogeneous
    qn, _ = oracle.heat_flux(cfg, cell0)
    expect = (1.0 - Pr * r) ** n * q0
    assert np.allclose(qn, expect, rtol=0, atol=1e-10 * np.abs(q0).max())
    m1 = oracle.moments(cfg, F)
    for k in ("rho", "ux", "uy", "uz", "T"):
        assert np.allclose(m1[k], m0[k], rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("Pr", [2.0 / 3.0, 0.3])
def test_heat_flux_semi_implicit_rate(dim, Pr):
    """Eq. ImpSchemeDD with the Shakhov equilibrium in a homogeneous gas: the
    heat flux follows q^{n+1} = q^n / (1 + Pr nu), nu = dt/tau, at dt/tau = 4
    (where the explicit scheme is unstable); rho, u and T stay fixed."""
    cfg, F, start, rho = homogeneous(dim, Pr, 1)
    tau = oracle.tau0(cfg) / rho
    cfg = dict(cfg, time_scheme=1, dt=4.0 * tau)
    q0, _ = oracle.heat_flux(cfg, start)
    m0 = oracle.moments(cfg, F)
    nu = 4.0
    n = 6
    run = oracle.run if dim == 2 else oracle.run3d
    assert run(cfg, F, n)["status"] == 0
    cell0 = F[: F.size // (2 ** dim)]
    qn, _ = oracle.heat_flux(cfg, cell0)
    expect = q0 / (1.0 + Pr * nu) ** n
    assert np.allclose(qn, expect, rtol=0, atol=1e-10 * np.abs(q0).max()), (qn, expect)
    m1 = oracle.moments(cfg, F)
    for k in ("rho", "ux", "uy", "uz", "T"):
        assert np.allclose(m1[k], m0[k], rtol=0, atol=1e-12)


def test_pr_one_is_bgk_semi_implicit():
    cfg = dict(W.cylinder_mach2(nx=32, nv=12), Kn=1e-3, time_scheme=1)
    F0 = oracle.initial_state(cfg)
    a, b = F0.copy(), F0.copy()
    assert oracle.run(cfg, a, 5)["status"] == 0
    assert oracle.run(dict(cfg, model=1, Pr=1.0), b, 5)["status"] == 0
    assert np.array_equal(a, b)


def test_stiff_semi_implicit_step_is_the_maxwellian():
    """nu -> infinity: q^{n+1} -> 0 and the step gives the Maxwellian of the
    transported state's moments (textbook 2D Maxwellian, fine grid)."""
    cfg, F, start, rho = homogeneous(2, 2.0 / 3.0, 1)
    cfg = dict(cfg, time_scheme=1, dt=1e9 * oracle.tau0(cfg) / rho)
    m = oracle.moments(cfg, F)
    assert oracle.run(cfg, F, 1)["status"] == 0
    vx, vy = velocity_axis(cfg, "x"), velocity_axis(cfg, "y")
    VX, VY = np.meshgrid(vx, vy)
    r, ux, uy, T = m["rho"][0], m["ux"][0], m["uy"][0], m["T"][0]
    M = (r / (2 * np.pi * T) * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2) / (2 * T))).ravel()
    nv = M.size
    assert np.abs(F[:nv] - M).max() <= 1e-8 * M.max()
    assert np.abs(F[nv:2 * nv] - T / 2 * M).max() <= 1e-8 * M.max()


def test_shakhov_needs_pr_and_direct_moments():
    cfg = W.cylinder_mach2(nx=16, nv=8)
    F = oracle.initial_state(cfg)
    assert oracle.run(dict(cfg, model=1, Pr=-0.5), F.copy(), 1)["status"] != 0
    assert oracle.run(dict(cfg, model=1, Pr=2.0 / 3.0, conservative=1), F.copy(), 1)["status"] != 0
    with pytest.raises(ValueError):
        oracle.equilibrium(one_cell(2, 8, 4.0, model=1, Pr=-1.0), 1.0, (0, 0), 1.0, (0, 0))


def test_pr_one_is_bgk_moving_body():
    """A rotating ellipse (area ratios S^n / S^{n+1,*} of merged control
    volumes, appearing cells): Pr = 1 is the BGK run bit for bit."""
    cfg = W.rotating_ellipse(nx=48, nv=10, scheme=1)
    F0 = oracle.initial_state(cfg)
    a, b = F0.copy(), F0.copy()
    ha = oracle.run(cfg, a, 6)
    hb = oracle.run(dict(cfg, model=1, Pr=1.0), b, 6)
    assert ha["status"] == 0 and hb["status"] == 0
    assert np.array_equal(a, b)
    assert np.array_equal(ha["torque"], hb["torque"])
