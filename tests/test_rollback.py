"""Failure detection of dvm_step: a failing call leaves the state, the body
and the step count at the last good step (the input of the first step whose
output has a non-positive density or temperature).  The failure is the
explicit scheme's own instability at dt/tau ~ 50, made on the host side by
the choice of Kn: no GPU fault is involved.  GPU only."""
import numpy as np
import pytest

from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NONPHYSICAL = 4


def unstable(cfg):
    cfg = dict(cfg)
    cfg.update(Kn=1e-4)            # explicit relaxation with dt/tau far above 2
    return cfg


def steps_done(s):
    return len(s.history(100000)["Fx"])


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_failing_step_leaves_last_good_state(prec):
    cfg = unstable(W.cylinder_mach2(nx=48, nv=16))
    a = dvm.Solver(cfg, prec)
    a.init_maxwellian()
    with pytest.raises(dvm.DVMError) as err:
        a.step(300)
    assert err.value.code == NONPHYSICAL
    k = steps_done(a)
    assert 0 < k < 300
    Fa = a.get_state()
    assert np.isfinite(Fa).all()
    a.close()
    # k steps from the same start succeed and give the same state; the next
    # step fails and leaves it unchanged
    b = dvm.Solver(cfg, prec)
    b.init_maxwellian()
    b.step(k)
    assert np.array_equal(b.get_state(), Fa)
    with pytest.raises(dvm.DVMError):
        b.step(1)
    assert steps_done(b) == k
    assert np.array_equal(b.get_state(), Fa)
    b.close()


def test_failing_step_moving_body():
    """The rigid body and its geometry go back with the state."""
    cfg = unstable(W.rotating_ellipse(nx=64, nv=12, scheme=1))
    a = dvm.Solver(cfg, dvm.FP64)
    a.init_maxwellian()
    with pytest.raises(dvm.DVMError):
        a.step(300)
    k = steps_done(a)
    Fa, body = a.get_state(), a.body_state()
    a.close()
    b = dvm.Solver(cfg, dvm.FP64)
    b.init_maxwellian()
    b.step(k)
    assert np.array_equal(b.get_state(), Fa)
    assert b.body_state() == body
    b.close()


def test_without_rollback_the_state_runs_on():
    """dvm_rollback(ctx, 0): the failing call leaves the state after its last
    step (all 300 steps are taken)."""
    cfg = unstable(W.cylinder_mach2(nx=48, nv=16))
    s = dvm.Solver(cfg, dvm.FP64)
    s.rollback(False)
    s.init_maxwellian()
    with pytest.raises(dvm.DVMError):
        s.step(300)
    assert steps_done(s) == 300
    s.close()


def test_stable_run_is_unchanged_by_the_checks():
    """A run that never fails gives the same state with and without the
    per-chunk copies and checks (1030 steps: a full chunk and a partial one)."""
    cfg = W.cylinder_mach2(nx=32, nv=12)
    out = []
    for rb in (True, False):
        s = dvm.Solver(cfg, dvm.FP32)
        s.rollback(rb)
        s.init_maxwellian()
        s.step(1030)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0], out[1])
