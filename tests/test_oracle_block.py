"""The block restriction used by the full-size sphere parity test, checked on
the oracle alone: stepping a block of cells that holds the whole body, from
the full grid's state, gives the full grid's result on every block cell more
than 2n cells from the block's faces after n steps (the MUSCL stencil of
Eq. eq-schema3D reaches two cells; the wall, fusion and force terms are
local to the body), and the same force history."""
import numpy as np

import oracle
from paper_1503_04544_gb300 import workloads as W


def block_cfg(cfg, lo, hi, dt):
    n = cfg["nx"]
    b = dict(cfg)
    b.update(nx=hi - lo, ny=hi - lo, nz=hi - lo, dt=dt, bc=[2] * 6, bc_state=[None] * 6)
    for ax in ("x", "y", "z"):
        b[ax + "min"] = lo / n
        b[ax + "max"] = hi / n
    return b


def test_sphere_block_restriction_is_exact():
    cfg = W.sphere_mach15(n=24, nv=8, scheme=1)
    n, nv = cfg["nx"], cfg["nvx"] * cfg["nvy"] * cfg["nvz"]
    lo, hi, steps = 4, 20, 2
    m = hi - lo
    # a perturbed start, so that no block face sees the free stream that a
    # zero-gradient face would reproduce
    F = oracle.initial_state(cfg) * W.perturbation(n ** 3 * nv, seed=3)
    assert oracle.run3d(cfg, F, 3)["status"] == 0
    Fb = F.reshape(n, n, n, nv)[lo:hi, lo:hi, lo:hi].copy().ravel()
    bcfg = block_cfg(cfg, lo, hi, oracle.time_step(cfg))
    g = oracle.geometry3d(cfg)
    gb = oracle.geometry3d(bcfg)
    assert np.array_equal(gb["type"], g["type"].reshape(n, n, n)[lo:hi, lo:hi, lo:hi].ravel())
    cut = np.argwhere((gb["type"] == oracle.CUT).reshape(m, m, m))
    assert len(cut) > 0 and cut.min() >= 2 * steps and cut.max() < m - 2 * steps
    hf = oracle.run3d(cfg, F, steps)
    hb = oracle.run3d(bcfg, Fb, steps)
    assert hf["status"] == 0 and hb["status"] == 0
    e = 2 * steps
    full = F.reshape(n, n, n, nv)[lo + e:hi - e, lo + e:hi - e, lo + e:hi - e]
    blk = Fb.reshape(m, m, m, nv)[e:m - e, e:m - e, e:m - e]
    assert np.abs(blk - full).max() <= 1e-14 * np.abs(full).max()
    assert np.abs(hb["Fx"] - hf["Fx"]).max() <= 1e-12 * np.abs(hf["Fx"]).max()
    # one cell closer to the faces the block is no longer exact: the bound
    # above is tight, so the test would see a wider stencil
    near = F.reshape(n, n, n, nv)[lo + e - 1:hi - e + 1, lo + e - 1:hi - e + 1, lo + e - 1:hi - e + 1]
    bnear = Fb.reshape(m, m, m, nv)[e - 1:m - e + 1, e - 1:m - e + 1, e - 1:m - e + 1]
    assert np.abs(bnear - near).max() > 1e-10 * np.abs(full).max()
