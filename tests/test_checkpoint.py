"""Checkpoint and restart (dvm_save / dvm_load): 2n steps in one run equal n
steps, a save, a load into a fresh context and n more steps, bit for bit
(state, body angle and angular velocity, last force).  GPU only."""
import numpy as np
import pytest

from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def final(s):
    return s.get_state(), s.body_state(), s.wall_force()[0]


def resume_case(cfg, prec, n, tmp_path):
    a = dvm.Solver(cfg, prec)
    a.init_maxwellian()
    a.step(2 * n)
    ref = final(a)
    a.close()
    b = dvm.Solver(cfg, prec)
    b.init_maxwellian()
    b.step(n)
    path = str(tmp_path / "ckpt.dvm")
    b.save(path)
    b.close()
    c = dvm.Solver(cfg, prec)
    c.load(path)
    c.step(n)
    got = final(c)
    c.close()
    assert np.array_equal(got[0], ref[0])
    assert got[1] == ref[1]
    assert np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("prec", [dvm.FP32, dvm.FP64])
def test_resume_cylinder(prec, tmp_path):
    resume_case(W.cylinder_mach2(nx=48, nv=16), prec, 12, tmp_path)


def test_resume_moving_ellipse(tmp_path):
    """The geometry of the saved angle is rebuilt from the saved (cos, sin)."""
    resume_case(W.rotating_ellipse(nx=64, nv=12, scheme=1), dvm.FP32, 10, tmp_path)


def test_resume_sphere(tmp_path):
    resume_case(W.sphere_mach15(n=16, nv=8), dvm.FP32, 5, tmp_path)


def test_resume_semi_implicit(tmp_path):
    cfg = W.cylinder_mach2(nx=48, nv=16)
    cfg.update(Kn=1e-3, time_scheme=1)
    resume_case(cfg, dvm.FP32, 10, tmp_path)


def test_load_rejects_other_problem_and_garbage(tmp_path):
    s = dvm.Solver(W.cylinder_mach2(nx=48, nv=16), dvm.FP32)
    s.init_maxwellian()
    path = str(tmp_path / "a.dvm")
    s.save(path)
    s.close()
    for other in (W.cylinder_mach2(nx=32, nv=16), W.cylinder_mach2(nx=48, nv=8)):
        t = dvm.Solver(other, dvm.FP32)
        with pytest.raises(dvm.DVMError):
            t.load(path)
        t.close()
    t = dvm.Solver(W.cylinder_mach2(nx=48, nv=16), dvm.FP64)
    with pytest.raises(dvm.DVMError):
        t.load(path)
    bad = tmp_path / "b.dvm"
    bad.write_bytes(b"not a checkpoint" * 8)
    with pytest.raises(dvm.DVMError):
        t.load(str(bad))
    with pytest.raises(dvm.DVMError):
        t.load(str(tmp_path / "missing.dvm"))
    t.close()


def test_load_rejects_same_sizes_other_problem(tmp_path):
    """The same grid, velocities, precision and time step, but another wall
    temperature, obstacle size, inflow state or collision model: the header's
    problem hash refuses the checkpoint."""
    base = W.cylinder_mach2(nx=48, nv=16)
    s = dvm.Solver(base, dvm.FP32)
    s.init_maxwellian()
    path = str(tmp_path / "a.dvm")
    s.save(path)
    s.close()
    same = dvm.Solver(base, dvm.FP32)
    same.load(path)                       # the same problem loads
    same.close()
    others = [W.cylinder_mach2(nx=48, nv=16, Tw=1.3), W.cylinder_mach2(nx=48, nv=16, mach=1.5)]
    bigger = W.cylinder_mach2(nx=48, nv=16)
    bigger["ra"] = 0.12
    shak = W.cylinder_mach2(nx=48, nv=16)
    shak.update(model=1, Pr=2.0 / 3.0)
    others += [bigger, shak]
    for other in others:
        t = dvm.Solver(other, dvm.FP32)
        with pytest.raises(dvm.DVMError):
            t.load(path)
        t.close()


def test_save_needs_a_state(tmp_path):
    s = dvm.Solver(W.cylinder_mach2(nx=32, nv=8), dvm.FP32)
    with pytest.raises(dvm.DVMError):
        s.save(str(tmp_path / "x.dvm"))
    s.close()
