"""The allocation-free mass entry point (dvm_mass_noalloc) against dvm_mass.

dvm_mass_noalloc exists for callers that cannot call cudaMalloc (a hook
under a framework allocator that owns all device memory, a loop with a fixed
memory budget); it keeps its per-cell scratch in a static device array shared
by all calls.  Two calls in a row on different
states must each reproduce the context's own mass, so nothing of the first
call's scratch may leak into the second.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1503_04544_gb300 import dvm
from paper_1503_04544_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _dv(cfg):
    return (cfg["vxmax"] - cfg["vxmin"]) / cfg["nvx"] * ((cfg["vymax"] - cfg["vymin"]) / cfg["nvy"])


@pytest.mark.parametrize("prec", [dvm.FP64, dvm.FP32])
def test_mass_noalloc_matches_context_mass(prec):
    import torch
    lib = dvm.load()
    cfg = W.cylinder_mach2(nx=64, nv=16)
    s = dvm.Solver(cfg, prec)
    s.init_maxwellian()
    tdt = torch.float32 if prec == dvm.FP32 else torch.float64
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(3 + call)                     # a different state for each call
        ref = s.mass()
        f = torch.empty(s.state_size, dtype=tdt, device="cuda")
        s.get_state(f)
        sbar = torch.tensor(s.geometry2d()["sbar"], dtype=torch.float64, device="cuda")
        rc = lib.dvm_mass_noalloc(ctypes.c_void_p(f.data_ptr()), prec, s.ncell, s.ncomp, s.nv,
                                  ctypes.c_void_p(sbar.data_ptr()), _dv(cfg),
                                  ctypes.c_void_p(out.data_ptr() + 8 * call), None)
        assert rc == dvm.OK, lib.dvm_last_error().decode()
        torch.cuda.synchronize()
        got = out[call].item()
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
    s.close()


def test_mass_noalloc_matches_context_mass_3d():
    """The same on a 3D state: one component F, sbar = the virtual-cell
    volumes, dv = dvx dvy dvz; two calls in a row on different states."""
    import torch
    lib = dvm.load()
    cfg = W.sphere_mach15(n=24, nv=8, scheme=1)
    s = dvm.Solver(cfg, dvm.FP32)
    s.init_maxwellian()
    dv = _dv(cfg) * (cfg["vzmax"] - cfg["vzmin"]) / cfg["nvz"]
    vol = torch.tensor(s.geometry3d()["vol"], dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        s.step(2 + call)
        ref = s.mass()
        f = torch.empty(s.state_size, dtype=torch.float32, device="cuda")
        s.get_state(f)
        rc = lib.dvm_mass_noalloc(ctypes.c_void_p(f.data_ptr()), dvm.FP32, s.ncell, s.ncomp, s.nv,
                                  ctypes.c_void_p(vol.data_ptr()), dv,
                                  ctypes.c_void_p(out.data_ptr() + 8 * call), None)
        assert rc == dvm.OK, lib.dvm_last_error().decode()
        torch.cuda.synchronize()
        got = out[call].item()
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
    s.close()


def test_mass_noalloc_rejects_oversized_state():
    import torch
    lib = dvm.load()
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.dvm_mass_noalloc(ctypes.c_void_p(buf.data_ptr()), dvm.FP64, (1 << 20) + 1, 1, 1,
                              ctypes.c_void_p(buf.data_ptr()), 1.0, ctypes.c_void_p(buf.data_ptr()), None)
    assert rc == dvm.ERR_ARG
    assert "capacity" in lib.dvm_last_error().decode()
