"""Velocity split of the step over ranks (arXiv:1503.04544, Sec. 5.2,
"velocity parallelization"): every rank holds every cell for a slab of rows
of the last velocity axis (v_y in 2D, v_z in 3D), transports and relaxes its
own velocities, and the ranks sum one exchange buffer per step (the moment
sums of every cell and the wall sums of every wall cell, dvm_split_begin /
dvm_split_finish).  The semi-implicit scheme sums it a second time: the
moment sums of the transported values, from which every rank relaxes its own
velocities (dvm_split_relax).

The sum is the caller's collective: ``torch.distributed.all_reduce`` on the
buffer (NCCL between GPUs), or ``local_allreduce`` for several contexts of
one process.  This module only partitions the velocity grid and orders the
calls; every step of the method runs in libdvm.
"""
from __future__ import annotations

import numpy as np

from . import dvm


def rows(nvy: int, rank: int, nranks: int) -> tuple[int, int]:
    """The v_y rows [k0, k1) of ``rank``: a balanced contiguous partition."""
    if not 0 <= rank < nranks or nranks > nvy:
        raise ValueError("rank out of range or more ranks than v_y rows")
    return rank * nvy // nranks, (rank + 1) * nvy // nranks


def _axis(cfg: dict) -> str:
    return "z" if cfg.get("dim", 2) == 3 else "y"


def slab_cfg(cfg: dict, rank: int, nranks: int) -> dict:
    """The problem of one rank: the same cells, body and boundaries, the
    rows of ``rows`` of the last velocity axis and the whole grid for the
    split."""
    a = _axis(cfg)
    k0, k1 = rows(cfg["nv" + a], rank, nranks)
    step = (cfg["v" + a + "max"] - cfg["v" + a + "min"]) / cfg["nv" + a]
    out = dict(cfg)
    out["nv" + a] = k1 - k0
    out["v" + a + "min"] = cfg["v" + a + "min"] + k0 * step
    out["v" + a + "max"] = cfg["v" + a + "min"] + k1 * step
    out["vsplit_global"] = {k: cfg[k] for k in ("nvx", "nvy", "nvz", "vxmin", "vxmax", "vymin", "vymax",
                                                "vzmin", "vzmax") if k in cfg}
    out["vsplit_rows"] = (k0, k1)
    return out


def _shape(cfg: dict):
    """Cells, components, rows of the split axis, velocities per row."""
    if cfg.get("dim", 2) == 3:
        nc = cfg["nx"] * cfg["ny"] * cfg["nz"]
        return nc, 1, cfg["nvz"], cfg["nvx"] * cfg["nvy"]
    return cfg["nx"] * cfg["ny"], 2, cfg["nvy"], cfg["nvx"]


def slab_of_state(cfg: dict, F: np.ndarray, rank: int, nranks: int) -> np.ndarray:
    """The part of a whole state ([cell][comp][p], the split axis' row the
    slowest index of p) that ``rank`` holds."""
    nc, ncomp, nrow, per = _shape(cfg)
    k0, k1 = rows(nrow, rank, nranks)
    return np.ascontiguousarray(F.reshape(nc, ncomp, nrow * per)[:, :, k0 * per: k1 * per]).ravel()


def assemble_state(cfg: dict, parts: list[np.ndarray]) -> np.ndarray:
    """The whole state from the ranks' slabs, in rank order."""
    nc, ncomp, _, _ = _shape(cfg)
    return np.concatenate([p.reshape(nc, ncomp, -1) for p in parts], axis=2).ravel()


class SplitSolver:
    """One rank's libdvm context and its exchange buffer.  ``stream`` is the
    torch CUDA stream the context enqueues on; the sum over the ranks must be
    ordered on it (make it torch's current stream)."""

    def __init__(self, cfg: dict, rank: int, nranks: int, stream, precision: int = dvm.FP64):
        import torch
        if stream.cuda_stream == 0:
            raise ValueError("give the split contexts a non-default CUDA stream")
        self.cfg = slab_cfg(cfg, rank, nranks)
        self.rank, self.nranks = rank, nranks
        self.solver = dvm.Solver(self.cfg, precision, stream=stream.cuda_stream)
        self.xbuf = torch.zeros(self.solver.split_size(), dtype=torch.float64, device="cuda")

    def begin(self):
        self.solver.split_begin(self.xbuf)
        return self.xbuf

    def finish(self) -> bool:
        """Finish the step; True when it waits for the second exchange (the
        semi-implicit scheme), with this rank's sums in the buffer."""
        self.solver.split_finish(self.xbuf)
        return self.solver.time_scheme == dvm.IMEX

    def relax(self):
        self.solver.split_relax(self.xbuf)

    def close(self):
        self.solver.close()


def step(ranks: list[SplitSolver], allreduce, nsteps: int = 1):
    """``nsteps`` steps of the contexts in ``ranks`` (the ones this process
    holds), with ``allreduce(list of buffers)`` summing the buffers over all
    ranks in place."""
    for _ in range(nsteps):
        bufs = [r.begin() for r in ranks]
        allreduce(bufs)
        pending = [r.finish() for r in ranks]
        if any(pending):
            if not all(pending):
                raise RuntimeError("velocity split: the ranks use different time schemes")
            allreduce(bufs)
            for r in ranks:
                r.relax()


def local_allreduce(bufs):
    """The sum over contexts held by one process (one GPU): every buffer
    becomes the element-wise sum, added in rank order."""
    total = bufs[0].clone()
    for b in bufs[1:]:
        total.add_(b)
    for b in bufs:
        b.copy_(total)


def dist_allreduce(bufs):
    """The sum over the processes of the default torch.distributed group (one
    context per process)."""
    import torch.distributed as dist
    for b in bufs:
        dist.all_reduce(b)
