"""PyTorch autograd interface to the drag and its adjoint gradient.

``drag(tw_seg, mach, ...)`` returns the drag J = F_x of the cylinder flow
after ``nsteps`` steps (a 2D fixed cylinder with per-sector wall temperatures
``tw_seg`` and a Maxwellian inflow at Mach ``mach``, see
:func:`paper_1503_04544_gb300.workloads.cylinder_adjoint`) as a 0-d tensor
whose backward pass gives dJ/dT_w per sector and dJ/dMach.  The gradient
comes from the library's discrete adjoint (dvm_drag_adjoint: checkpointed
forward run, recomputation and transposed steps on the GPU); when a gradient
is requested it is computed together with J in one call.

The Mach number sets u = Ma sqrt(5/3) in the inflow Maxwellian and in the
initial state, so dJ/dMach = sqrt(5/3) (sum of dJ/du_x over the inflow cells
and over the initial-state cells).

``evolve(F0, cfg, nsteps)`` is the state after ``nsteps`` steps as a tensor
differentiable in the initial state F0; its backward pass is the adjoint of
the whole sweep with the incoming gradient as the seed (dvm_adjoint).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import dvm
from . import workloads as W

_SQ = math.sqrt(5.0 / 3.0)


def _problem(tw: np.ndarray, mach: float, nx: int, nv: int, nsteps: int) -> dict:
    cfg = W.cylinder_adjoint(nx=nx, nv=nv, nseg=len(tw), mach=mach, steps=nsteps)
    cfg["Tw_seg"] = np.asarray(tw, dtype=np.float64)
    return cfg


class DragFunction(torch.autograd.Function):
    """J(T_w, Ma) with the discrete-adjoint gradient."""

    @staticmethod
    def forward(ctx, tw_seg, mach, nx, nv, nsteps, checkpoint_every, precision):
        tw = tw_seg.detach().to("cpu", torch.float64).numpy()
        m = float(mach.detach().cpu())
        s = dvm.Solver(_problem(tw, m, nx, nv, nsteps), precision)
        try:
            s.init_maxwellian()
            if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
                out = s.drag_adjoint(nsteps, checkpoint_every)
                J = out["J"]
                gmach = _SQ * (out["gbc"][0][:, 1].sum() + out["gprim0"][:, 1].sum())
                ctx.save_for_backward(torch.as_tensor(out["gTw"], dtype=tw_seg.dtype, device=tw_seg.device),
                                      torch.as_tensor(gmach, dtype=mach.dtype, device=mach.device))
            else:
                s.step(nsteps + 1)
                J = float(s.history(1)["Fx"][0])
        finally:
            s.close()
        return torch.as_tensor(J, dtype=torch.float64, device=tw_seg.device)

    @staticmethod
    def backward(ctx, gJ):
        gtw, gmach = ctx.saved_tensors
        return gJ.to(gtw.dtype) * gtw, gJ.to(gmach.dtype) * gmach, None, None, None, None, None


def drag(tw_seg: torch.Tensor, mach: torch.Tensor, nx: int = 256, nv: int = 32, nsteps: int = 200,
         checkpoint_every: int = 20, precision: int = dvm.FP32) -> torch.Tensor:
    """Drag of the per-sector-temperature cylinder after ``nsteps`` steps."""
    return DragFunction.apply(tw_seg, mach, nx, nv, nsteps, checkpoint_every, precision)


class EvolveFunction(torch.autograd.Function):
    """F^N = Step^N(F^0) of a fixed-obstacle 2D problem, differentiable with
    respect to the initial state: the backward pass is the library's
    checkpointed adjoint with the seed dL/dF^N (dvm_adjoint, no drag term),
    all on the GPU."""

    @staticmethod
    def forward(ctx, F0, cfg, nsteps, checkpoint_every, precision):
        s = dvm.Solver(cfg, precision, stream=torch.cuda.current_stream().cuda_stream)
        try:
            s.set_state(F0.detach().contiguous())
            s.step(nsteps)
            FN = torch.empty_like(F0)
            s.get_state(FN)
        finally:
            s.close()
        ctx.save_for_backward(F0.detach())
        ctx.cfg, ctx.nsteps, ctx.K, ctx.precision = cfg, nsteps, checkpoint_every, precision
        return FN

    @staticmethod
    def backward(ctx, gFN):
        (F0,) = ctx.saved_tensors
        s = dvm.Solver(ctx.cfg, ctx.precision, stream=torch.cuda.current_stream().cuda_stream)
        try:
            s.set_state(F0.contiguous())
            out = s.adjoint(ctx.nsteps, ctx.K, with_drag=False, seed=gFN.contiguous().to(F0.dtype))
        finally:
            s.close()
        return out["lambda0"], None, None, None, None


def evolve(F0: torch.Tensor, cfg: dict, nsteps: int, checkpoint_every: int = 20) -> torch.Tensor:
    """``nsteps`` steps of ``cfg`` from the CUDA state ``F0`` (public layout;
    float32 or float64 sets the precision), differentiable in ``F0``."""
    precision = dvm.FP32 if F0.dtype == torch.float32 else dvm.FP64
    return EvolveFunction.apply(F0, cfg, nsteps, checkpoint_every, precision)
