"""Two-step CUDA graph replays of dvm_step: the same kernels in the same
order as launch-by-launch stepping, so the state, the force history and the
rigid-body state must agree bit for bit.  GPU only."""
import numpy as np
import pytest

from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(cfg, prec, steps, graphs, chunks=(1,)):
    s = dvm.Solver(cfg, prec)
    s.graphs(graphs)
    s.init_maxwellian()
    done = 0
    k = 0
    while done < steps:
        n = min(chunks[k % len(chunks)], steps - done)
        s.step(n)
        done += n
        k += 1
    out = dict(F=s.get_state(), hist=s.history(steps + 4), body=s.body_state(), launches=s.launches())
    s.close()
    return out


def same(a, b):
    assert np.array_equal(a["F"], b["F"])
    for k in a["hist"]:
        assert np.array_equal(a["hist"][k], b["hist"][k]), k
    assert a["body"] == b["body"]
    assert a["launches"] == b["launches"]


@pytest.mark.parametrize("prec", [dvm.FP32, dvm.FP64])
def test_graph_cylinder_bitwise(prec):
    """Fixed cylinder, MUSCL: one call of 23 steps (first step plain, 11
    replays) and calls of 9 and 14 steps against launch by launch."""
    cfg = W.cylinder_mach2(nx=64, nv=16)
    ref = run(cfg, prec, 23, graphs=False)
    same(run(cfg, prec, 23, graphs=True), ref)
    same(run(cfg, prec, 23, graphs=True, chunks=(9, 14)), ref)


def test_graph_moving_ellipse_bitwise():
    """Moving body: the geometry is rebuilt every step on two levels, the
    rigid-body ODE advances on the device; the replays keep both in step."""
    cfg = W.rotating_ellipse(nx=96, nv=12, scheme=1)
    ref = run(cfg, dvm.FP32, 20, graphs=False)
    out = run(cfg, dvm.FP32, 20, graphs=True)
    same(out, ref)
    assert out["body"][1] != 0.0


def test_graph_sphere_bitwise():
    cfg = W.sphere_mach15(n=20, nv=8)
    same(run(cfg, dvm.FP32, 12, graphs=True), run(cfg, dvm.FP32, 12, graphs=False))


def test_graph_timing_marks():
    """With per-launch timing on, the steps go launch by launch and every
    bulk launch is timed."""
    cfg = W.cylinder_mach2(nx=64, nv=16)
    s = dvm.Solver(cfg, dvm.FP32)
    s.init_maxwellian()
    s.step(1)
    s.timing(True)
    s.step_async(31)
    s.check()
    ms, n = s.kernel_time()
    s.timing(False)
    assert n == 31
    assert ms > 0
    s.close()


def test_graph_many_async_calls():
    """70 unchecked dvm_step_async calls of 10 steps each (one step launch by
    launch, four replays of the two-step graph, one more step) pass the point
    where the launched graphs are released with one wait; the state still
    agrees bit for bit with 700 steps launch by launch."""
    cfg = W.cylinder_mach2(nx=32, nv=16)
    s = dvm.Solver(cfg, dvm.FP32)
    s.init_maxwellian()
    for _ in range(70):
        s.step_async(10)
    s.check()
    F = s.get_state()
    s.close()
    ref = run(cfg, dvm.FP32, 700, graphs=False)
    assert np.array_equal(F, ref["F"])
