"""The closed containers on the GPU (2D, the gas inside a disk or a box):
geometry bit for bit against the oracle, the state after a run against the
oracle's (FP64 within 1e-12 of the largest value, FP32 moments within 1e-5),
and exact mass conservation with a hot diffuse wall.  GPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GEO_KEYS = ("type", "cgas", "lx", "ly", "lw", "nwx", "nwy", "rwx", "rwy", "sbar")


def rel_inf(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max()
    s = np.abs(np.asarray(b, np.float64)).max()
    return d / s if s > 0 else d


@pytest.mark.parametrize("shape,kw", [(4, dict(ra=0.45)), (4, dict(ra=0.4312, cx=0.503, cy=0.49)),
                                      (5, dict(ra=0.41, rb=0.33, cx=0.5013, cy=0.4987))])
@pytest.mark.parametrize("nx", [64, 129])
def test_container_geometry_bit_exact(shape, kw, nx):
    cfg = W.base2d(nx, nx, 4, 4.0, shape=shape, **kw)
    s = dvm.Solver(cfg, dvm.FP64)
    s.geometry2d_at(1.0, 0.0)
    gg = s.geometry2d()
    go = oracle.geometry2d(cfg, 1.0, 0.0)
    for k in GEO_KEYS:
        assert np.array_equal(gg[k], go[k]), k
    mo, rc = oracle.masters2d(cfg, go)
    assert rc == 0
    assert np.array_equal(gg["master"], mo)
    s.close()


@pytest.mark.parametrize("which,scheme", [("disk", 1), ("box", 1), ("box", 0)])
def test_container_state_fp64(which, scheme):
    """30 steps from the oracle's initial state (hot wall, density bump;
    drifting gas in the box): the whole state equals the oracle's, and so
    does the force history on the wall."""
    cfg = (W.disk_container if which == "disk" else W.box_container)(nx=40, nv=12, scheme=scheme)
    F0 = oracle.initial_state(cfg)
    s = dvm.Solver(cfg, dvm.FP64)
    s.set_state(F0)
    s.step(30)
    s.check()
    Fo = F0.copy()
    h = oracle.run(cfg, Fo, 30)
    assert h["status"] == 0
    assert rel_inf(s.get_state(), Fo) <= 1e-12
    # the net force on a closed wall is a cancellation of wall terms of order
    # one (pressure times length) down to about 1e-5: bound the difference
    # absolutely, a few hundred units in the last place of those terms
    hg = s.history(30)
    assert np.abs(hg["Fx"] - h["Fx"]).max() <= 1e-13 and np.abs(hg["Fy"] - h["Fy"]).max() <= 1e-13
    s.close()


@pytest.mark.parametrize("which", ["disk", "box"])
def test_container_moments_fp32(which):
    cfg = (W.disk_container if which == "disk" else W.box_container)(nx=48, nv=16)
    F0 = oracle.initial_state(cfg)
    s = dvm.Solver(cfg, dvm.FP32)
    s.set_state(F0)
    s.step(40)
    s.check()
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 40)["status"] == 0
    mo = oracle.moments(cfg, Fo)
    mg = s.moments()
    live = mo["rho"] > 0
    for k in ("rho", "ux", "uy", "T"):
        scale = np.abs(mo[k][live]).max()
        if k in ("ux", "uy"):
            scale = max(scale, 1.0)
        assert np.abs(mg[k][live] - mo[k][live]).max() <= 1e-5 * scale, k
    s.close()


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_container_mass_conservation_gpu(prec):
    """Eq. def-masse on the device: the disk container of radius 0.45 with a
    hot wall keeps the mass of its gas (FP64 to round-off)."""
    cfg = W.disk_container(nx=48, nv=32)
    cfg.update(vxmin=-10.0, vxmax=10.0, vymin=-10.0, vymax=10.0)
    s = dvm.Solver(cfg, prec)
    s.init_maxwellian()
    m0 = s.mass()
    s.step(150)
    s.check()
    m1 = s.mass()
    drift = abs(m1 - m0) / m0
    assert drift < (1e-13 if prec == dvm.FP64 else 1e-5), drift
    assert math.isfinite(m1)
    s.close()
