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
