"""The velocity split on the GPU (Sec. 5.2): rank contexts, each holding
every cell for a slab of v_y rows, stepped with dvm_split_begin, a sum of
the exchange buffers over the ranks and dvm_split_finish, against the
unsplit context and the oracle.  The ranks are contexts of one process on
one GPU, stepped one after the other by the host; their buffers are summed
by torch on the contexts' stream (the same element-wise sum an all-reduce
over GPUs gives).  GPU only.

The split reorders only the velocity sums (per rank, then over the ranks),
so FP64 states agree to round-off (1e-13 of the largest value here) and FP32
moments within 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1503_04544_gb300 import dvm, vsplit
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def split_run(cfg, nranks, prec, steps, F0=None):
    import torch
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ranks = [vsplit.SplitSolver(cfg, r, nranks, st, prec) for r in range(nranks)]
        for r in ranks:
            if F0 is None:
                r.solver.init_maxwellian()
            else:
                r.solver.set_state(vsplit.slab_of_state(cfg, F0, r.rank, nranks))
        vsplit.step(ranks, vsplit.local_allreduce, steps)
        for r in ranks:
            r.solver.check()
        F = vsplit.assemble_state(cfg, [r.solver.get_state() for r in ranks])
        hist = ranks[0].solver.history(steps)
        others = [r.solver.history(steps) for r in ranks[1:]]
        body = [r.solver.body_state() for r in ranks]
        mass = sum(r.solver.mass() for r in ranks)
        for r in ranks:
            r.close()
    # every rank computed the same force history and body state
    for h in others:
        assert np.array_equal(h["Fx"], hist["Fx"]) and np.array_equal(h["torque"], hist["torque"])
    assert all(b == body[0] for b in body)
    return F, hist, body[0], mass


def whole_run(cfg, prec, steps, F0=None):
    s = dvm.Solver(cfg, prec)
    if F0 is None:
        s.init_maxwellian()
    else:
        s.set_state(F0)
    s.step(steps)
    out = s.get_state(), s.history(steps), s.body_state(), s.mass()
    s.close()
    return out


def rel(a, b):
    return np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max() / np.abs(b).max()


@pytest.mark.parametrize("nranks", [2, 3])
@pytest.mark.parametrize("scheme", [0, 1])
def test_split_cylinder_fp64_matches_whole_and_oracle(nranks, scheme):
    """Fixed cylinder, Mach 2, 40^2 cells x 12^2 velocities, 10 steps (the
    first fuses the merged control volumes): the assembled split state equals
    the unsplit one and the oracle's, and so do the drag histories."""
    cfg = W.cylinder_mach2(nx=40, nv=12, scheme=scheme)
    F0 = oracle.initial_state(cfg)
    Fs, hs, _, ms = split_run(cfg, nranks, dvm.FP64, 10, F0)
    Fw, hw, _, mw = whole_run(cfg, dvm.FP64, 10, F0)
    assert rel(Fs, Fw) <= 1e-13, rel(Fs, Fw)
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-12
    assert abs(ms - mw) <= 1e-13 * abs(mw)
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 10)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


def test_split_cylinder_fp32():
    cfg = W.cylinder_mach2(nx=48, nv=16, scheme=1)
    Fs, hs, _, _ = split_run(cfg, 2, dvm.FP32, 20)
    Fw, hw, _, _ = whole_run(cfg, dvm.FP32, 20)
    ms = oracle.moments(cfg, Fs.astype(np.float64))
    mw = oracle.moments(cfg, Fw.astype(np.float64))
    live = mw["rho"] > 0
    for k in ("rho", "ux", "uy", "T"):
        scale = max(np.abs(mw[k][live]).max(), 1.0 if k != "rho" and k != "T" else 0.0)
        assert np.abs(ms[k][live] - mw[k][live]).max() <= 1e-5 * scale, k
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-5


def test_split_rotating_ellipse_fp64():
    """Rotating ellipse: geometry rebuilt every step on every rank, the
    torque and the rigid-body update from the summed wall sums."""
    cfg = W.rotating_ellipse(nx=48, nv=12, scheme=1)
    F0 = oracle.initial_state(cfg)
    Fs, hs, bs, _ = split_run(cfg, 2, dvm.FP64, 12, F0)
    Fw, hw, bw, _ = whole_run(cfg, dvm.FP64, 12, F0)
    assert rel(Fs, Fw) <= 1e-13
    assert abs(bs[0] - bw[0]) <= 1e-13 and abs(bs[1] - bw[1]) <= 1e-11 * max(abs(bw[1]), 1.0)
    assert rel(hs["torque"], hw["torque"]) <= 1e-11


def test_split_conservative_equilibrium():
    """The conservative equilibrium (Sec. 3.1) solves Newton over the whole
    velocity grid from the summed moments."""
    cfg = W.cylinder_mach2(nx=40, nv=10, scheme=1)
    cfg["conservative"] = 1
    F0 = oracle.initial_state(cfg)
    Fs, _, _, _ = split_run(cfg, 2, dvm.FP64, 8, F0)
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 8)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


@pytest.mark.parametrize("nranks", [2, 3])
@pytest.mark.parametrize("conservative", [0, 1])
def test_split_imex_cylinder_fp64(nranks, conservative):
    """The semi-implicit scheme (Eq. ImpSchemeDD) with the velocity split:
    the relaxation takes the moments of the transported values summed over
    the ranks (a second exchange per step), with the direct moments or the
    conservative parameters (Sec. 3.1).  Fixed cylinder, 40^2 cells x 12^2
    velocities, MUSCL, 10 steps: the assembled state equals the unsplit
    context's and the oracle's."""
    cfg = W.cylinder_mach2(nx=40, nv=12, scheme=1)
    cfg.update(time_scheme=1, conservative=conservative)
    F0 = oracle.initial_state(cfg)
    Fs, hs, _, ms = split_run(cfg, nranks, dvm.FP64, 10, F0)
    Fw, hw, _, mw = whole_run(cfg, dvm.FP64, 10, F0)
    assert rel(Fs, Fw) <= 1e-13, rel(Fs, Fw)
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-12
    assert abs(ms - mw) <= 1e-13 * abs(mw)
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 10)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


def test_split_imex_rotating_ellipse_fp64():
    """Semi-implicit, rotating ellipse: the cell types of t^{n+1} in the
    relaxation of every rank."""
    cfg = W.rotating_ellipse(nx=48, nv=12, scheme=0)
    cfg["time_scheme"] = 1
    F0 = oracle.initial_state(cfg)
    Fs, hs, bs, _ = split_run(cfg, 2, dvm.FP64, 12, F0)
    Fw, hw, bw, _ = whole_run(cfg, dvm.FP64, 12, F0)
    assert rel(Fs, Fw) <= 1e-13
    assert abs(bs[1] - bw[1]) <= 1e-11 * max(abs(bw[1]), 1.0)
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 12)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


def test_split_imex_cylinder_fp32():
    cfg = W.cylinder_mach2(nx=48, nv=16, scheme=1)
    cfg["time_scheme"] = 1
    Fs, hs, _, _ = split_run(cfg, 2, dvm.FP32, 20)
    Fw, hw, _, _ = whole_run(cfg, dvm.FP32, 20)
    ms = oracle.moments(cfg, Fs.astype(np.float64))
    mw = oracle.moments(cfg, Fw.astype(np.float64))
    live = mw["rho"] > 0
    for k in ("rho", "ux", "uy", "T"):
        scale = max(np.abs(mw[k][live]).max(), 1.0 if k != "rho" and k != "T" else 0.0)
        assert np.abs(ms[k][live] - mw[k][live]).max() <= 1e-5 * scale, k
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-5


def test_split_errors():
    """The order of the split calls; both ranks step with summed buffers so
    that the steps taken are valid ones."""
    import torch
    cfg = W.cylinder_mach2(nx=32, nv=8)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ranks = [vsplit.SplitSolver(cfg, k, 2, st) for k in range(2)]
        r = ranks[0]
        s = r.solver
        for q in ranks:
            q.solver.init_maxwellian()
        for call in (lambda: s.step(1), lambda: s.moments(), lambda: s.set_collision_model(1, 0.7),
                     lambda: s.split_finish(r.xbuf), lambda: s.split_relax(r.xbuf)):
            with pytest.raises(dvm.DVMError):
                call()
        bufs = [q.begin() for q in ranks]
        F = s.get_state()
        # between the calls of a step nothing may change the state or the scheme
        for call in (lambda: s.split_begin(r.xbuf), lambda: s.split_relax(r.xbuf), lambda: s.set_time_scheme(1),
                     lambda: s.set_state(F), lambda: s.init_maxwellian(), lambda: s.set_equilibrium(1)):
            with pytest.raises(dvm.DVMError) as e:
                call()
            assert e.value.code == dvm.ERR_STATE
        vsplit.local_allreduce(bufs)
        assert not any(q.finish() for q in ranks)
        # the explicit step is complete: no relaxation pending
        with pytest.raises(dvm.DVMError) as e:
            s.split_relax(r.xbuf)
        assert e.value.code == dvm.ERR_STATE
        # the semi-implicit step waits for the second exchange
        for q in ranks:
            q.solver.set_time_scheme(1)
        bufs = [q.begin() for q in ranks]
        vsplit.local_allreduce(bufs)
        assert all(q.finish() for q in ranks)
        for call in (lambda: s.split_begin(r.xbuf), lambda: s.split_finish(r.xbuf), lambda: s.set_time_scheme(0)):
            with pytest.raises(dvm.DVMError) as e:
                call()
            assert e.value.code == dvm.ERR_STATE
        vsplit.local_allreduce(bufs)
        for q in ranks:
            q.relax()
            q.solver.check()
            q.close()
    # a velocity grid that is not a slab of the whole grid
    bad = vsplit.slab_cfg(cfg, 1, 2)
    bad["vymin"] += 0.1
    bad["vymax"] += 0.1
    with pytest.raises(dvm.DVMError) as e:
        dvm.Solver(bad, dvm.FP64)
    assert e.value.code == dvm.ERR_ARG


@pytest.mark.parametrize("nranks", [2, 3])
def test_split_sphere_fp64_matches_whole_and_oracle(nranks):
    """3D sphere, 16^3 cells x 9^3 velocities split along v_z, MUSCL,
    Mach 1.5, 4 steps: the assembled state equals the unsplit one and the
    oracle's; the ranks' drag histories are identical."""
    cfg = W.sphere_mach15(n=16, nv=9, scheme=1)
    cfg["ra"] = 0.23
    F0 = oracle.initial_state(cfg)
    Fs, hs, _, ms = split_run(cfg, nranks, dvm.FP64, 4, F0)
    Fw, hw, _, mw = whole_run(cfg, dvm.FP64, 4, F0)
    assert rel(Fs, Fw) <= 1e-13, rel(Fs, Fw)
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-12
    assert abs(ms - mw) <= 1e-13 * abs(mw)
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 4)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


def test_split_sphere_fp32_conservative():
    """3D, FP32, with the conservative equilibrium (the Newton over the
    whole grid from the summed moments): moments within 1e-5 of the unsplit
    context's."""
    cfg = W.sphere_mach15(n=16, nv=8, scheme=1)
    cfg.update(ra=0.23, conservative=1)
    Fs, _, _, _ = split_run(cfg, 2, dvm.FP32, 5)
    Fw, _, _, _ = whole_run(cfg, dvm.FP32, 5)
    ms = oracle.moments(cfg, Fs.astype(np.float64))
    mw = oracle.moments(cfg, Fw.astype(np.float64))
    live = mw["rho"] > 0
    for k in ("rho", "ux", "uy", "uz", "T"):
        scale = np.abs(mw[k][live]).max()
        if k.startswith("u"):
            scale = max(scale, 1.0)
        assert np.abs(ms[k][live] - mw[k][live]).max() <= 1e-5 * scale, k


@pytest.mark.parametrize("conservative", [0, 1])
def test_split_imex_sphere_fp64(conservative):
    """3D semi-implicit split along v_z, direct and conservative equilibrium:
    the assembled state equals the unsplit one and the oracle's."""
    cfg = W.sphere_mach15(n=16, nv=9, scheme=1)
    cfg.update(ra=0.23, time_scheme=1, conservative=conservative)
    F0 = oracle.initial_state(cfg)
    Fs, hs, _, _ = split_run(cfg, 3, dvm.FP64, 4, F0)
    Fw, hw, _, _ = whole_run(cfg, dvm.FP64, 4, F0)
    assert rel(Fs, Fw) <= 1e-13, rel(Fs, Fw)
    assert rel(hs["Fx"], hw["Fx"]) <= 1e-12
    Fo = F0.copy()
    assert oracle.run(cfg, Fo, 4)["status"] == 0
    assert rel(Fs, Fo) <= 1e-12


def test_split_imex_sphere_fp32():
    cfg = W.sphere_mach15(n=16, nv=8, scheme=1)
    cfg.update(ra=0.23, time_scheme=1)
    Fs, _, _, _ = split_run(cfg, 2, dvm.FP32, 5)
    Fw, _, _, _ = whole_run(cfg, dvm.FP32, 5)
    ms = oracle.moments(cfg, Fs.astype(np.float64))
    mw = oracle.moments(cfg, Fw.astype(np.float64))
    live = mw["rho"] > 0
    for k in ("rho", "ux", "uy", "uz", "T"):
        scale = np.abs(mw[k][live]).max()
        if k.startswith("u"):
            scale = max(scale, 1.0)
        assert np.abs(ms[k][live] - mw[k][live]).max() <= 1e-5 * scale, k
