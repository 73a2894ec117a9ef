"""The velocity split's host path on CPU: two or three gloo ranks (Sec. 5.2).

Each rank holds a slab of v_y rows of a periodic two-cell box (a space-
homogeneous gas) and steps it through the same protocol as the library's
split contexts: its moment sums into the exchange buffer in the library's
layout ([4][ncell]: sum f, vx f, vy f, |v|^2/2 f + g over the rank's
velocities), the sum over the ranks by torch.distributed (gloo), then the
BGK relaxation of its own velocities with the moments of the summed buffer.
Under the semi-implicit scheme (Eq. ImpSchemeDD) the finish writes the
moment sums of the transported values (here, with no space dependence, the
state itself) and the ranks sum the buffer a second time before relaxing.
The stand-ins for the library's begin, finish and relax are a few numpy
lines; the partition (vsplit.rows, slab_cfg, slab_of_state,
assemble_state), the exchange and the step order (vsplit.step) are the
product code under test.  The assembled state must equal the oracle's
whole-grid run, and the exchanged moments the oracle's moments.
"""
from __future__ import annotations

import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_1503_04544_gb300 import workloads as W
    return W.base2d(2, 1, 12, 6.0, Kn=0.05, Lref=1.0, dt=2e-3,
                    init=dict(rho=np.array([1.0, 1.0]), ux=0.3, uy=-0.2, uz=0.0, T=1.2))


def _initial(scheme=0):
    """A two-Maxwellian mixture in both cells (not an equilibrium)."""
    cfg = _problem()
    cfg["time_scheme"] = scheme
    dv = (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]
    v = cfg["vxmin"] + np.arange(cfg["nvx"]) * dv
    VX, VY = np.meshgrid(v, v)
    VX, VY = VX.ravel(), VY.ravel()
    m = lambda r, ux, uy, T: r / (2 * np.pi * T) * np.exp(-((VX - ux) ** 2 + (VY - uy) ** 2) / (2 * T))
    f = m(0.6, 0.5, 0.1, 0.9) + m(0.5, -0.3, -0.2, 1.3)
    g = 0.45 * m(0.6, 0.5, 0.1, 0.9) + 0.65 * m(0.5, -0.3, -0.2, 1.3)
    cell = np.concatenate([f, g])
    return cfg, np.concatenate([cell, cell])


class _HomogeneousRank:
    """The protocol of a split context (vsplit.SplitSolver's begin, finish
    and relax) on a space-homogeneous box."""

    def __init__(self, cfg, F0, rank, nranks, xbuf):
        from paper_1503_04544_gb300 import vsplit
        self.lcfg = vsplit.slab_cfg(cfg, rank, nranks)
        self.F = vsplit.slab_of_state(cfg, F0, rank, nranks).copy()
        self.imex = int(cfg.get("time_scheme", 0)) == 1
        self.xbuf = xbuf
        self.first = None
        c = self.lcfg
        dvx = (c["vxmax"] - c["vxmin"]) / c["nvx"]
        dvy = (c["vymax"] - c["vymin"]) / c["nvy"]
        vx = c["vxmin"] + np.arange(c["nvx"]) * dvx
        vy = c["vymin"] + np.arange(c["nvy"]) * dvy
        VX, VY = np.meshgrid(vx, vy)
        self.VX, self.VY, self.dv = VX.ravel(), VY.ravel(), dvx * dvy
        self.nc = c["nx"] * c["ny"]
        self.tau0 = math.sqrt(math.pi) / 2 * c["Kn"] * c["Lref"] / math.sqrt(2)

    def _sums(self):
        Fv = self.F.reshape(self.nc, 2, self.VX.size)
        f, g = Fv[:, 0], Fv[:, 1]
        x = np.stack([f.sum(1), (f * self.VX).sum(1), (f * self.VY).sum(1),
                      (0.5 * (self.VX ** 2 + self.VY ** 2) * f + g).sum(1)])
        self.xbuf.numpy()[:] = x.ravel()

    def _maxwellian(self, x, k):
        rho = x[0, k] * self.dv
        ux, uy = x[1, k] / x[0, k], x[2, k] / x[0, k]
        T = (2 * x[3, k] / x[0, k] - ux * ux - uy * uy) / 3
        M = rho / (2 * np.pi * T) * np.exp(-((self.VX - ux) ** 2 + (self.VY - uy) ** 2) / (2 * T))
        return rho, T, M

    def begin(self):
        self._sums()
        return self.xbuf

    def finish(self):
        x = self.xbuf.numpy().reshape(4, self.nc)
        if self.first is None:
            self.first = x.copy()
        if self.imex:
            # no transport in a homogeneous box: the sums of the state again
            self._sums()
            return True
        Fv = self.F.reshape(self.nc, 2, self.VX.size)
        for k in range(self.nc):
            rho, T, M = self._maxwellian(x, k)
            r = self.lcfg["dt"] * rho / self.tau0
            Fv[k, 0] += r * (M - Fv[k, 0])
            Fv[k, 1] += r * (T / 2 * M - Fv[k, 1])
        return False

    def relax(self):
        x = self.xbuf.numpy().reshape(4, self.nc)
        Fv = self.F.reshape(self.nc, 2, self.VX.size)
        for k in range(self.nc):
            rho, T, M = self._maxwellian(x, k)
            nu = self.lcfg["dt"] * rho / self.tau0
            Fv[k, 0] = (Fv[k, 0] + nu * M) / (1 + nu)
            Fv[k, 1] = (Fv[k, 1] + nu * T / 2 * M) / (1 + nu)


def _rank_main(rank, world, port, out_dir, nsteps, scheme):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_1503_04544_gb300 import vsplit

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, F0 = _initial(scheme)
        r = _HomogeneousRank(cfg, F0, rank, world, torch.zeros(8, dtype=torch.float64))
        vsplit.step([r], vsplit.dist_allreduce, nsteps)
        np.save(os.path.join(out_dir, f"slab{rank}.npy"), r.F)
        np.save(os.path.join(out_dir, f"x0_{rank}.npy"), r.first)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("scheme", [0, 1])
def test_velocity_split_protocol_gloo(world, scheme, tmp_path):
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1503_04544_gb300 import vsplit

    nsteps = 30
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), nsteps, scheme), nprocs=world, join=True)
    cfg, F0 = _initial(scheme)
    # the exchanged sums of the first step are the whole grid's moments
    mo = oracle.moments(cfg, F0)
    dv = ((cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"]) ** 2
    for rank in range(world):
        x = np.load(tmp_path / f"x0_{rank}.npy").reshape(4, 2)
        assert np.allclose(x[0] * dv, mo["rho"], rtol=1e-14, atol=0)
        assert np.allclose(x[1] / x[0], mo["ux"], rtol=1e-13, atol=1e-15)
    # the assembled state equals the oracle's whole-grid run
    parts = [np.load(tmp_path / f"slab{r}.npy") for r in range(world)]
    got = vsplit.assemble_state(cfg, parts)
    F = F0.copy()
    assert oracle.run(cfg, F, nsteps)["status"] == 0
    assert np.abs(got - F).max() <= 1e-13 * np.abs(F).max()
    # the two schemes differ by O(dt^2) per step: the run tells them apart
    if scheme == 1:
        Fe = F0.copy()
        cfge, _ = _initial(0)
        assert oracle.run(cfge, Fe, nsteps)["status"] == 0
        assert np.abs(Fe - F).max() > 1e-9 * np.abs(F).max()


def test_partition_helpers():
    sys.path.insert(0, ROOT)
    from paper_1503_04544_gb300 import vsplit
    from paper_1503_04544_gb300 import workloads as W
    assert [vsplit.rows(32, r, 3) for r in range(3)] == [(0, 10), (10, 21), (21, 32)]
    with pytest.raises(ValueError):
        vsplit.rows(4, 0, 5)
    cfg = W.cylinder_mach2(nx=8, nv=8)
    loc = vsplit.slab_cfg(cfg, 1, 2)
    dvy = (cfg["vymax"] - cfg["vymin"]) / cfg["nvy"]
    assert loc["nvy"] == 4 and loc["vymin"] == cfg["vymin"] + 4 * dvy and loc["vymax"] == cfg["vymax"]
    F = np.arange(64 * 2 * 64, dtype=np.float64)
    parts = [vsplit.slab_of_state(cfg, F, r, 2) for r in range(2)]
    assert np.array_equal(vsplit.assemble_state(cfg, parts), F)
    # 3D: rows of v_z, one component
    c3 = W.sphere_mach15(n=4, nv=6)
    l3 = vsplit.slab_cfg(c3, 2, 3)
    assert l3["nvz"] == 2 and l3["nvx"] == 6 and l3["nvy"] == 6
    F3 = np.arange(64 * 216, dtype=np.float64)
    parts = [vsplit.slab_of_state(c3, F3, r, 3) for r in range(3)]
    assert parts[0].size == 64 * 72
    assert np.array_equal(vsplit.assemble_state(c3, parts), F3)
