"""Pins of the oracle's discrete adjoint (drag gradient) against central
finite differences of the oracle's own forward run, FP64.  CPU only.

J = F_x of the state after N steps (Eqs. StressTensorDD, eq-force); the
adjoint gives dJ/dT_w per wall sector, dJ/d(inflow state) and dJ/dF^0.  A
wrong transpose anywhere (a dropped relaxation-through-moments term, a
limiter branch derivative, the wall-density coupling, the ghost cells or the
fusion transpose) shows up as a mismatch with the finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import workloads as W

H = 1e-6
NX, NV, NSEG, STEPS = 24, 12, 8, 12


def drag_after(cfg, steps, F0=None):
    F = oracle.initial_state(cfg) if F0 is None else F0.copy()
    h = oracle.run(cfg, F, steps + 1)
    assert h["status"] == 0
    return h["Fx"][steps]                   # force of the state at t^N


def problem(scheme, mach=2.0, tw=None):
    cfg = W.cylinder_adjoint(nx=NX, nv=NV, nseg=NSEG, mach=mach, steps=STEPS)
    cfg["scheme"] = scheme
    if tw is not None:
        cfg["Tw_seg"] = tw
    return cfg


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_wall_temperatures_and_mach_match_central_fd(scheme):
    """All 8 sector temperatures and the inflow Mach number (through the
    inflow ghost cells and the initial state, u = Ma sqrt(5/3))."""
    cfg = problem(scheme)
    a = oracle.adjoint2d(cfg, oracle.initial_state(cfg), STEPS)
    assert a["status"] == 0
    assert abs(a["J"] - drag_after(cfg, STEPS)) <= 1e-14 * abs(a["J"])
    tw = cfg["Tw_seg"].copy()
    fd = np.zeros(NSEG)
    for s in range(NSEG):
        tp, tm = tw.copy(), tw.copy()
        tp[s] += H
        tm[s] -= H
        fd[s] = (drag_after(problem(scheme, tw=tp), STEPS) - drag_after(problem(scheme, tw=tm), STEPS)) / (2 * H)
    assert np.abs(fd).max() > 1e-3
    assert np.abs(a["gTw"] - fd).max() <= 1e-6 * np.abs(fd).max(), (a["gTw"], fd)
    gi = oracle.init_maxwellian_vjp(cfg, a["lam0"])
    gmach = math.sqrt(5.0 / 3.0) * (gi[:, 1].sum() + a["gbc"][0][:, 1].sum())
    fdm = (drag_after(problem(scheme, mach=2.0 + H), STEPS) - drag_after(problem(scheme, mach=2.0 - H), STEPS)) / (2 * H)
    assert abs(gmach - fdm) <= 1e-6 * abs(fdm), (gmach, fdm)


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_state_directional_derivative(scheme):
    """<dJ/dF^0, dF> equals the central difference of J along a random
    perturbation dF of the initial state (every cell, both components, all
    velocities): checks the whole state adjoint.  The limited scheme starts
    from a smooth non-uniform state (in a uniform state every limiter
    difference is exactly 0, where minmod has a kink and no derivative)."""
    cfg = problem(scheme)
    if scheme == 1:
        x = (np.arange(NX) + 0.5) / NX
        X, Y = np.meshgrid(x, x)
        u = math.sqrt(5.0 / 3.0) * 2.0
        cfg["init"] = dict(rho=(1.0 + 0.2 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y)).ravel(),
                           ux=(u * (1.0 + 0.1 * np.cos(2 * np.pi * Y))).ravel(),
                           uy=(0.2 * np.sin(2 * np.pi * X)).ravel(), uz=0.0,
                           T=(1.0 + 0.1 * X * Y).ravel())
    F0 = oracle.initial_state(cfg)
    a = oracle.adjoint2d(cfg, F0, STEPS)
    rng = np.random.default_rng(4)
    dF = F0 * rng.uniform(-1, 1, F0.size)          # relative perturbation keeps F >= 0
    eps = 1e-7
    fd = (drag_after(cfg, STEPS, F0 + eps * dF) - drag_after(cfg, STEPS, F0 - eps * dF)) / (2 * eps)
    ad = float(a["lam0"] @ dF)
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_adjoint_zero_steps_is_the_force_gradient():
    """N = 0: dJ/dF^0 is the gradient of the force functional itself
    (stress of the outgoing state plus the diffuse reflection through phi)."""
    cfg = problem(0)
    F0 = oracle.initial_state(cfg)
    a = oracle.adjoint2d(cfg, F0, 0)
    rng = np.random.default_rng(5)
    dF = F0 * rng.uniform(-1, 1, F0.size)
    eps = 1e-6
    fd = (drag_after(cfg, 0, F0 + eps * dF) - drag_after(cfg, 0, F0 - eps * dF)) / (2 * eps)
    assert abs(float(a["lam0"] @ dF) - fd) <= 1e-7 * abs(fd)
    # only wall cells carry a sensitivity at N = 0
    g = oracle.geometry2d(cfg)
    walls = (g["type"] == 1) & (g["lw"] > 0)
    lam = a["lam0"].reshape(NX * NX, -1)
    assert np.abs(lam[~walls]).max() == 0.0 and np.abs(lam[walls]).max() > 0


def test_uniform_wall_temperature():
    """nseg = 0: one wall temperature; its gradient equals the sum of the
    sector gradients of the same problem split into sectors."""
    cfg = problem(1)
    tw0 = 1.05
    cfg_u = dict(cfg, nseg=0, Tw=tw0)
    cfg_s = dict(cfg, Tw_seg=np.full(NSEG, tw0))
    au = oracle.adjoint2d(cfg_u, oracle.initial_state(cfg_u), STEPS)
    as_ = oracle.adjoint2d(cfg_s, oracle.initial_state(cfg_s), STEPS)
    assert abs(au["J"] - as_["J"]) <= 1e-13 * abs(au["J"])
    assert abs(au["gTw"][0] - as_["gTw"].sum()) <= 1e-12 * abs(au["gTw"][0])


def _smooth(cfg):
    x = (np.arange(NX) + 0.5) / NX
    X, Y = np.meshgrid(x, x)
    u = math.sqrt(5.0 / 3.0) * 2.0
    cfg["init"] = dict(rho=(1.0 + 0.2 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y)).ravel(),
                       ux=(u * (1.0 + 0.1 * np.cos(2 * np.pi * Y))).ravel(),
                       uy=(0.2 * np.sin(2 * np.pi * X)).ravel(), uz=0.0, T=(1.0 + 0.1 * X * Y).ravel())
    return cfg


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_linear_functional_directional_derivative(scheme):
    """J = <seed, F^N> for a random seed on every non-solid cell, component
    and velocity (no drag): <lambda^0, dF> equals the central difference of J
    along a random relative perturbation dF of F^0, and one sector's dJ/dT_w
    its central difference.  Every cell carries a sensitivity from the start,
    the domain boundaries included."""
    cfg = _smooth(problem(scheme))
    steps = 6
    F0 = oracle.initial_state(cfg)
    rng = np.random.default_rng(9)
    live = np.repeat(F0.reshape(-1, 2 * NV * NV).max(axis=1) > 0, 2 * NV * NV)
    seed = rng.uniform(-1, 1, F0.size) * live
    a = oracle.adjoint2d_seed(cfg, F0, steps, seed)
    assert a["status"] == 0 and a["J"] == 0.0

    def G(c, F):
        F = F.copy()
        assert oracle.run(c, F, steps)["status"] == 0
        return float(seed @ F)

    dF = F0 * rng.uniform(-1, 1, F0.size)
    eps = 1e-7
    fd = (G(cfg, F0 + eps * dF) - G(cfg, F0 - eps * dF)) / (2 * eps)
    ad = float(a["lam0"] @ dF)
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)
    k = 3
    tw = cfg["Tw_seg"].copy()
    tp, tm = tw.copy(), tw.copy()
    tp[k] += H
    tm[k] -= H
    fdt = (G(dict(cfg, Tw_seg=tp), F0) - G(dict(cfg, Tw_seg=tm), F0)) / (2 * H)
    assert abs(a["gTw"][k] - fdt) <= 1e-6 * max(abs(fdt), np.abs(a["gTw"]).max()), (a["gTw"][k], fdt)


def test_adjoint_drag_plus_seed_is_linear():
    cfg = _smooth(problem(1))
    F0 = oracle.initial_state(cfg)
    seed = np.random.default_rng(2).uniform(-1, 1, F0.size)
    a = oracle.adjoint2d_seed(cfg, F0, 5, None, with_drag=True)
    b = oracle.adjoint2d_seed(cfg, F0, 5, seed)
    c = oracle.adjoint2d_seed(cfg, F0, 5, seed, with_drag=True)
    d = oracle.adjoint2d(cfg, F0, 5)
    assert np.array_equal(a["lam0"], d["lam0"]) and a["J"] == d["J"]
    assert np.abs(a["lam0"] + b["lam0"] - c["lam0"]).max() <= 1e-13 * np.abs(c["lam0"]).max()
