"""torch.autograd interface to the drag gradient (paper_1503_04544_gb300.autograd).
GPU only."""
import math

import numpy as np
import pytest
import torch

from paper_1503_04544_gb300 import autograd as AG
from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_backward_equals_library_adjoint():
    tw = torch.tensor(W.cylinder_adjoint(nx=24, nv=12, nseg=8)["Tw_seg"], dtype=torch.float64, requires_grad=True)
    mach = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    J = AG.drag(tw, mach, nx=24, nv=12, nsteps=10, checkpoint_every=4, precision=dvm.FP64)
    J.backward()
    cfg = W.cylinder_adjoint(nx=24, nv=12, nseg=8, steps=10)
    s = dvm.Solver(cfg, dvm.FP64)
    s.init_maxwellian()
    out = s.drag_adjoint(10, 4)
    s.close()
    assert abs(J.item() - out["J"]) <= 1e-13 * abs(out["J"])
    np.testing.assert_allclose(tw.grad.numpy(), out["gTw"], rtol=0, atol=1e-14 * np.abs(out["gTw"]).max())
    gm = math.sqrt(5 / 3) * (out["gbc"][0][:, 1].sum() + out["gprim0"][:, 1].sum())
    assert abs(mach.grad.item() - gm) <= 1e-13 * abs(gm)


def test_no_grad_forward_gives_the_same_drag():
    tw = torch.tensor(W.cylinder_adjoint(nx=24, nv=12, nseg=8)["Tw_seg"], dtype=torch.float64)
    mach = torch.tensor(2.0, dtype=torch.float64)
    with torch.no_grad():
        J0 = AG.drag(tw, mach, nx=24, nv=12, nsteps=10, checkpoint_every=4, precision=dvm.FP64)
    J1 = AG.drag(tw.clone().requires_grad_(True), mach, nx=24, nv=12, nsteps=10, checkpoint_every=4,
                 precision=dvm.FP64)
    assert abs(J0.item() - J1.item()) <= 1e-12 * abs(J1.item())


def test_gradcheck():
    """torch.autograd.gradcheck: central differences of the FP64 forward
    against the adjoint, for 4 sectors and the Mach number."""
    tw = torch.tensor([0.9, 1.1, 1.05, 0.95], dtype=torch.float64, requires_grad=True)
    mach = torch.tensor(1.7, dtype=torch.float64, requires_grad=True)
    f = lambda a, b: AG.drag(a, b, nx=24, nv=12, nsteps=6, checkpoint_every=4, precision=dvm.FP64)
    assert torch.autograd.gradcheck(f, (tw, mach), eps=1e-6, atol=1e-7, rtol=1e-5)
