"""The block restriction used by the full-size sphere parity test, checked on
the oracle alone.  The block is the corner [0, m)^3 of the grid, with the cell
size of the full grid exactly (node coordinates 0 + a dx in both), so its
geometry and control volumes are the full grid's bit for bit; it holds the
whole body and keeps the grid's own conditions on its three low faces.
Stepping it from the full grid's state gives the full grid's result on every
cell more than 2n cells from its high faces after n steps (the MUSCL stencil
of Eq. eq-schema3D reaches two cells; the wall, fusion and force terms are
local to the body), and the same force history."""
import numpy as np

import oracle
from block3d import GEO3, block_view, corner_block, full_index
from paper_1503_04544_gb300 import workloads as W


def test_sphere_block_restriction_is_exact():
    cfg = W.sphere_mach15(n=24, nv=8, scheme=1)
    n, nv = cfg["nx"], cfg["nvx"] * cfg["nvy"] * cfg["nvz"]
    m, steps = 20, 2
    # a perturbed start, so that no high block face sees the free stream
    # that a zero-gradient face would reproduce
    F = oracle.initial_state(cfg) * W.perturbation(n ** 3 * nv, seed=3)
    assert oracle.run3d(cfg, F, 3)["status"] == 0
    Fb = F.reshape(n, n, n, nv)[:m, :m, :m].copy().ravel()
    bcfg = corner_block(cfg, m, oracle.time_step(cfg))
    g = oracle.geometry3d(cfg)
    gb = oracle.geometry3d(bcfg)
    for k in GEO3:
        assert np.array_equal(gb[k], block_view(g[k], n, m)), k
    assert np.array_equal(gb["ax"], block_view(g["ax"], n, m, (n, n, n + 1)))
    assert np.array_equal(gb["ay"], block_view(g["ay"], n, m, (n, n + 1, n)))
    assert np.array_equal(gb["az"], block_view(g["az"], n, m, (n + 1, n, n)))
    mf, _ = oracle.masters3d(cfg, g)
    mb, _ = oracle.masters3d(bcfg, gb)
    assert np.array_equal(full_index(mb, n, m), block_view(mf, n, m))
    cut = np.argwhere((gb["type"] == oracle.CUT).reshape(m, m, m))
    assert len(cut) > 0 and cut.max() < m - 2 * steps
    hf = oracle.run3d(cfg, F, steps)
    hb = oracle.run3d(bcfg, Fb, steps)
    assert hf["status"] == 0 and hb["status"] == 0
    e = m - 2 * steps
    full = F.reshape(n, n, n, nv)[:e, :e, :e]
    blk = Fb.reshape(m, m, m, nv)[:e, :e, :e]
    assert np.array_equal(blk, full)
    assert np.abs(hb["Fx"] - hf["Fx"]).max() <= 1e-12 * np.abs(hf["Fx"]).max()
    # one cell closer to the high faces the block is no longer exact: the
    # bound above is tight, so the test would see a wider stencil
    near = F.reshape(n, n, n, nv)[:e + 1, :e + 1, :e + 1]
    bnear = Fb.reshape(m, m, m, nv)[:e + 1, :e + 1, :e + 1]
    assert np.abs(bnear - near).max() > 1e-10 * np.abs(full).max()
