#!/usr/bin/env python3
"""Throughput of the cut-cell discrete-velocity step on GB300.

Default workload: 2D fixed cylinder, 256x256 cells on [0,1]^2, cylinder
r = 0.1, 32x32 velocities on [-8,8)^2, Mach-2 inflow, Kn 0.05, MUSCL-minmod,
FP32 state.  ``--workload sphere``: 3D fixed sphere, 96^3 cells on [0,1]^3,
r = 0.15, 20^3 velocities on [-5,5)^3, Mach-1.5 inflow, Kn 0.1, MUSCL-minmod.
One bench step is one time step of the whole method (wall density and
stress, force/torque, fluxes, relaxation, cut-cell control volumes,
moments).  Metric: (cell, velocity) pair updates per second over the
non-solid cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                  [--workload cylinder|sphere|ellipse|bump] [--impl gb300|reference]
                  [--time-scheme explicit|imex] [--model bgk|shakhov]
                  [--equilibrium direct|conservative]
                  [--no-sublines] [--no-accuracy] [--no-adjoint] [--no-cpu-baseline]

The default run (cylinder, FP32) also reports, nested in its line: the
errors of the FP32 and FP64 GPU paths against the oracle after the oracle
sample's steps and of FP32 against FP64 after the configuration's 2000
steps (``accuracy``); the FP64 line of the same workload (``fp64``, against
the measured FP64 FMA throughput); the 3D sphere line, 96^3 cells x 20^3
velocities in FP32 (``sphere``); and the cost of the drag gradient
(``adjoint``).

For N > 1 each rank runs an independent replica (the path is not sharded
here); value = pairs updated by all ranks / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-velocity pair updates/s"
UNIT = "pair-updates/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0        # the part's nominal HBM3e bandwidth
# FP64 ceiling of the 2D FP64 line: 152 SMs x 2 FP64 FMA lanes per clock x
# 2 flop x 2.07 GHz (the part's nominal 1.25 TFLOP/s FP64 rate)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
# algorithmic FP64 flops of one 2D MUSCL pair update (f and g): limited
# fluxes 2 x 16, update 2 x 7, Maxwellian 9, moments 8 (add/sub/mul 1,
# fma 2, exp 1, min/max 0)
FP64_FLOPS_PER_PAIR = 63


def workload(name: str):
    from paper_1503_04544_gb300 import workloads as W
    if name == "cylinder":
        return W.cylinder_mach2(nx=256, nv=32, scheme=1)
    if name == "ellipse":
        return W.rotating_ellipse(nx=512, nv=40)
    if name == "bump":
        return W.periodic_bump()
    if name == "sphere":
        return W.sphere_mach15(n=96, nv=20, scheme=1)
    raise SystemExit(f"unknown workload {name}")


DEFAULT_STEPS = {"cylinder": 2000, "ellipse": 5000, "bump": 2000, "sphere": 60}


def _dims(cfg):
    if cfg.get("dim", 2) == 3:
        return [cfg["nx"], cfg["ny"], cfg["nz"]], [cfg["nvx"], cfg["nvy"], cfg["nvz"]]
    return [cfg["nx"], cfg["ny"]], [cfg["nvx"], cfg["nvy"]]


def config_dict(cfg, prec, nsolid_free, extra=None):
    cells, vels = _dims(cfg)
    d = {
        "workload": cfg["name"],
        "cells": cells,
        "velocities": vels,
        "scheme": "muscl-minmod" if cfg.get("scheme", 0) == 1 else "upwind",
        "time_scheme": "semi-implicit" if cfg.get("time_scheme", 0) == 1 else "explicit",
        "collision": "shakhov, Pr 2/3" if cfg.get("model", 0) == 1 else "bgk",
        "equilibrium": "conservative (Newton)" if cfg.get("conservative", 0) else "direct moments",
        "precision": prec,
        "pairs_per_step": nsolid_free,
        "l2": "inputs larger than L2 (state per copy > 129 MB)",
    }
    if extra:
        d.update(extra)
    return d


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(kernel_src: str) -> str:
    """sha256/16 over a kernel's source file and the two headers it includes
    (the device helpers and the shared constants such as tile and ring sizes)."""
    import hashlib
    d = os.path.dirname(kernel_src)
    h = hashlib.sha256()
    for f in (kernel_src, os.path.join(d, "dvm_device.cuh"), os.path.join(d, "dvm_internal.h")):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(summary: str, kernel_src: str):
    """DRAM bytes per launch of the bulk kernel from the committed ncu summary,
    or None if the kernel source changed since the capture."""
    summ = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(summ):
        return None
    h = kernel_source_hash(kernel_src)
    rec = {}
    for line in open(summ):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            rec[k.strip()] = v.strip()
    if rec.get("kernel source sha256/16") != h:
        return None
    try:
        return float(rec["dram bytes per launch (scaled)"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in region"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_sample_cfg(cfg):
    """The oracle's bounded sample: the 2D workloads as they are; the 3D
    sphere on a 24^3 grid with the same velocity grid, physics and scheme
    (one full step at 96^3 takes minutes on the host cores)."""
    if cfg.get("dim", 2) == 3:
        from paper_1503_04544_gb300 import workloads as W
        return W.sphere_mach15(n=24, nv=cfg["nvx"], scheme=cfg.get("scheme", 1))
    return cfg


def cpu_baseline(cfg, budget_s: float = 12.0, max_steps: int = 1000, keep: bool = False):
    """Time the FP64 oracle as it stands on the host cores: whole steps from the
    initial state until about budget_s seconds of work (a bounded sample).
    keep: also return the oracle's state and last drag (keys _F, _fx) for the
    accuracy check of the GPU path."""
    import numpy as np
    import oracle
    cfg = cpu_sample_cfg(cfg)
    F = oracle.initial_state(cfg)
    if cfg.get("dim", 2) == 3:
        g = oracle.geometry3d(cfg)
        pairs = int(np.sum(g["type"] != 2)) * cfg["nvx"] * cfg["nvy"] * cfg["nvz"]
    else:
        g = oracle.geometry2d(cfg)
        pairs = int(np.sum(g["type"] != 2)) * cfg["nvx"] * cfg["nvy"]
    done = 0
    fx = 0.0
    t0 = time.perf_counter()
    while done < max_steps:
        h = oracle.run(cfg, F, 1)
        fx = float(h["Fx"][0])
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"value": pairs * done / el, "unit": UNIT, "cores": cores, "kind": "oracle", "steps": done,
           "sample": f"{done} FP64 oracle step(s) of {cfg['name']} from the initial state, {el:.1f} s"}
    if keep:
        out["_F"] = F
        out["_fx"] = fx
    return out


def adjoint_cost(precision_fp32: bool = True):
    """Cost of the drag gradient at the adjoint workload (256^2 cylinder, 32^2
    velocities, 64 wall sectors, 200 steps, checkpoints every 20): device time
    of the plain forward run, of the checkpointed forward and of the reverse
    sweep (recomputation and transposed steps)."""
    import torch
    from paper_1503_04544_gb300 import dvm
    from paper_1503_04544_gb300 import workloads as W
    cfg = W.cylinder_adjoint(nx=256, nv=32, nseg=64, steps=200)
    prec = dvm.FP32 if precision_fp32 else dvm.FP64
    # a dedicated stream: the library enqueues on it and the events below are
    # recorded on it
    stream = torch.cuda.Stream()
    s = dvm.Solver(cfg, prec, stream=stream.cuda_stream)
    s.init_maxwellian()
    s.step(3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s.init_maxwellian()
    torch.cuda.synchronize()
    e0.record(stream)
    s.step_async(200)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = e0.elapsed_time(e1)
    s.init_maxwellian()
    out = s.drag_adjoint(200, 20)
    # the same with the forward run's tape kept in HBM (dvm_set_adjoint_tape):
    # the checkpoint segments need no recomputation; a first call allocates
    # the tape buffers, the second is timed
    budget = 160 << 30
    s.set_adjoint_tape(budget)
    s.init_maxwellian()
    s.drag_adjoint(200, 20)
    s.init_maxwellian()
    kt = s.drag_adjoint(200, 20)
    s.set_adjoint_tape(0)
    s.close()
    return {"workload": cfg["name"], "steps": 200, "checkpoint_every": 20,
            "precision": "fp32" if precision_fp32 else "fp64",
            "ms_forward": ms_fwd, "ms_checkpointed_forward": out["ms_forward"],
            "ms_reverse": out["ms_reverse"],
            "reverse_over_forward": out["ms_reverse"] / ms_fwd,
            "gradient_over_forward": (out["ms_forward"] + out["ms_reverse"]) / ms_fwd,
            "kept_tape": {"budget_bytes": budget, "ms_forward": kt["ms_forward"], "ms_reverse": kt["ms_reverse"],
                          "gradient_over_forward": (kt["ms_forward"] + kt["ms_reverse"]) / ms_fwd,
                          "drag_rel_diff": abs(kt["J"] - out["J"]) / max(abs(out["J"]), 1e-300)},
            "note": "reverse = recomputation from checkpoints + transposed steps; "
                    "gradient = checkpointed forward + reverse; kept_tape: the forward run keeps "
                    "every segment's states and limiter branches on the device (no recomputation)"}


def max_over_ranks(values, device="cpu"):
    """Element-wise maximum of ``values`` over the ranks of the default process
    group; the values themselves when no group of more than one rank exists."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_throughput(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job rate of ``world`` independent replicas (weak scaling): the units
    every rank processed over the slowest rank's time."""
    if seconds <= 0.0:
        raise ValueError("non-positive time")
    return world * units_per_rank / seconds


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workload(args.workload)
    if args.time_scheme == "imex":
        cfg["time_scheme"] = 1
    if args.model == "shakhov":
        cfg.update(model=1, Pr=2.0 / 3.0)
    if args.equilibrium == "conservative":
        cfg["conservative"] = 1
    cb = cpu_baseline(cfg, budget_s=60.0, max_steps=max(1, min(args.steps, 8)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config_dict(cfg, "fp64", None, {"sample": cb["sample"]}),
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rel_errors(mg: dict, mo: dict, live, dim: int) -> dict:
    """Per moment field ||m - m_ref||_inf / ||m_ref||_inf over the non-solid
    cells; velocities are normalised by max(||u_ref||_inf, 1) (the velocity
    unit is sqrt(R T0))."""
    import numpy as np
    out = {}
    keys = ("rho", "ux", "uy", "uz", "T") if dim == 3 else ("rho", "ux", "uy", "T")
    for k in keys:
        ref = mo[k][live]
        scale = np.abs(ref).max()
        if k in ("ux", "uy", "uz"):
            scale = max(scale, 1.0)
        out[k] = float(np.abs(mg[k][live] - ref).max() / scale)
    out["max"] = max(out.values())
    return out


def gpu_run(cfg, prec, steps, stream, F0=None):
    """Moments and the force history of ``steps`` steps of ``cfg`` on the GPU
    from its initial Maxwellian (or the state F0)."""
    import numpy as np
    from paper_1503_04544_gb300 import dvm
    s = dvm.Solver(cfg, prec, stream=stream.cuda_stream)
    if F0 is None:
        s.init_maxwellian()
    else:
        s.set_state(F0)
    done = 0
    while done < steps:
        k = min(1000, steps - done)
        s.step_async(k)
        s.check()
        done += k
    m = s.moments()
    fx = s.history(min(steps, 32768))["Fx"]
    s.close()
    return m, (float(fx[-1]) if len(fx) else 0.0), np.asarray(fx)


def fp32_vs_fp64(cfg, steps, stream) -> dict:
    """FP32 moments and drag after ``steps`` steps against the FP64 GPU path
    (which matches the oracle within 1e-12 per step) from the same initial
    state."""
    import numpy as np
    from paper_1503_04544_gb300 import dvm
    t0 = time.perf_counter()
    m32, fx32, _ = gpu_run(cfg, dvm.FP32, steps, stream)
    m64, fx64, _ = gpu_run(cfg, dvm.FP64, steps, stream)
    live = m64["rho"] > 0
    dim = cfg.get("dim", 2)
    out = {"steps": steps, "moments": rel_errors(m32, m64, live, dim),
           "drag": abs(fx32 - fx64) / max(abs(fx64), 1e-300), "drag_fp64": fx64,
           "tolerance": 1e-5, "seconds": time.perf_counter() - t0}
    out["pass"] = bool(out["moments"]["max"] <= 1e-5)
    return out


def vs_oracle(cfg, F_oracle, fx_oracle, done, stream) -> dict:
    """GPU FP32 and FP64 runs of the oracle sample's ``done`` steps from the
    same initial state, against the oracle's state (moments) and drag."""
    import oracle
    from paper_1503_04544_gb300 import dvm
    mo = oracle.moments(cfg, F_oracle)
    live = mo["rho"] > 0
    dim = cfg.get("dim", 2)
    out = {"steps": done, "workload": cfg["name"]}
    for name, prec, tol in (("fp32", dvm.FP32, 1e-5), ("fp64", dvm.FP64, 1e-12)):
        mg, fx, _ = gpu_run(cfg, prec, done, stream)
        e = rel_errors(mg, mo, live, dim)
        out[name] = {"moments": e, "drag": abs(fx - fx_oracle) / max(abs(fx_oracle), 1e-300),
                     "tolerance": tol, "pass": bool(e["max"] <= tol)}
    return out


def measure(cfg, prec, args, world, local, stream, peak, peak_kind, fp64_peak=None):
    """One bench line of ``cfg`` at precision ``prec``: device-timed steps with
    per-launch timing of the dominant kernel, clocks, and the end-to-end run
    through the public API with pinned host buffers."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1503_04544_gb300 import dvm

    prec_name = "fp32" if prec == dvm.FP32 else "fp64"
    s = dvm.Solver(cfg, prec, stream=stream.cuda_stream)
    s.init_maxwellian()
    s.step(max(args.warmup, 3))
    counts = s.cell_counts()
    pairs_per_step = counts["nonsolid"] * s.nv
    bulk_pairs = counts["bulk"] * s.nv
    bytes_per_pair = 2 * s.ncomp * s.elem      # one read and one write of each component

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    s.timing(True)
    l0 = s.launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_async(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = s.launches() - l0
    s.check()
    ms = e0.elapsed_time(e1)
    bulk_ms, nb = s.kernel_time()
    s.timing(False)
    shak_ms, ns = 0.0, 0
    if cfg.get("model", 0) == 1:
        # the Shakhov model's own kernel (3D: k_shakhov3 every step; 2D:
        # k_heatflux, every step in FP64, in FP32 only on a step that has no
        # raw moments of its state), timed over a second run of the same steps
        s.timing(2)
        s.step_async(min(args.steps, 500))
        shak_ms, ns = s.kernel_time()
        s.timing(False)
    barrier()

    # end to end through the public API with pinned host buffers
    host = torch.empty(s.state_size, dtype=torch.float32 if prec == dvm.FP32 else torch.float64,
                       pin_memory=True)
    s.get_state(host)
    s.set_state(host)
    s.step(1)
    s.moments()
    barrier()
    t0 = time.perf_counter()
    s.set_state(host)
    s.step(args.steps)
    m = s.moments()
    barrier()
    e2e_s = time.perf_counter() - t0
    ms_max, e2e_s = max_over_ranks([ms, e2e_s], "cuda")
    h2d = s.state_size * s.elem
    d2h = 5 * 8 * s.ncell
    e2e = {"value": replica_throughput(pairs_per_step * args.steps, e2e_s, world), "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "per run: state H2D from pinned host memory, K steps, moments D2H"}
    assert np.isfinite(m["rho"]).all()
    del host
    s.close()

    avg_bulk_s = bulk_ms / max(nb, 1) / 1e3
    achieved = bulk_pairs * bytes_per_pair / avg_bulk_s / 1e9
    dim3 = cfg.get("dim", 2) == 3
    wl = workload_key(cfg)
    # the explicit Shakhov step runs its own variant of the bulk kernel (2D;
    # 3D in FP32)
    shak_tag = "shakhov_" if (cfg.get("model", 0) == 1 and cfg.get("time_scheme", 0) == 0
                              and (not dim3 or prec == dvm.FP32)) else ""
    traffic = recorded_traffic(
        f"k_bulk{'3' if dim3 else ''}_{shak_tag}{wl}_{prec_name}.md",
        os.path.join(ROOT, "paper_1503_04544_gb300", "csrc", "dvm_step3d.cu" if dim3 else "dvm_step2d.cu"))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "traffic": traffic,
                "kernel": ("k_bulk3" if dim3 else "k_bulk") + " (fused stream + relax + moments)",
                "peak_source": f"{peak_kind} HBM copy bandwidth",
                "bytes_per_pair": bytes_per_pair,
                "bulk_ms_per_launch": avg_bulk_s * 1e3,
                "bulk_share_of_step": (bulk_ms / max(nb, 1)) / (ms / args.steps)}
    if ns:
        # Shakhov: k_heatflux / k_heatflux3 read F^n of every gas cell once
        # (the step kernels form the Shakhov equilibrium themselves); FP64
        # 3D: k_shakhov3 reads F^n (heat flux) and reads and writes F^{n+1}
        avg_s = shak_ms / ns / 1e3
        post = dim3 and prec == dvm.FP64
        sb = (3 if post else 1) * s.ncomp * s.elem
        ach = pairs_per_step * sb / avg_s / 1e9
        kname = "k_shakhov3" if post else ("k_heatflux3" if dim3 else "k_heatflux")
        shak = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "frac_of_nominal": ach / NOMINAL_HBM_GBS,
                "traffic": recorded_traffic(f"{kname}_{wl}_{prec_name}.md",
                                            os.path.join(ROOT, "paper_1503_04544_gb300", "csrc",
                                                         "dvm_shakhov3d.cu" if dim3 else "dvm_shakhov2d.cu")),
                "kernel": kname + (" (heat flux of F^n + Shakhov term on F^{n+1} + moments)" if post
                                   else " (heat flux of F^n for the Shakhov equilibrium)"),
                "peak_source": f"{peak_kind} HBM copy bandwidth", "bytes_per_pair": sb,
                "ms_per_launch": avg_s * 1e3, "share_of_step": avg_s * 1e3 / (ms / args.steps)}
        if avg_s > avg_bulk_s:
            shak["k_bulk"] = roofline
            roofline = shak
        else:
            roofline[kname] = shak
    if prec == dvm.FP64 and not dim3 and cfg.get("scheme", 1) == 1 and roofline["kernel"].startswith("k_bulk"):
        # the FP64 step is bound by the FP64 pipe on this part: report that
        # ceiling (the measured FP64 FMA throughput), with the HBM view beside it
        gflops = FP64_FLOPS_PER_PAIR * bulk_pairs / avg_bulk_s / 1e9
        hbm = {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "frac_of_nominal", "peak_source",
                                        "bytes_per_pair")}
        del roofline["frac_of_nominal"]
        pk = fp64_peak if fp64_peak else FP64_PEAK_GFLOPS
        roofline.update({"bound": "alu", "achieved": gflops, "peak": pk, "unit": "GFLOP/s",
                         "frac": gflops / pk, "flops_per_pair": FP64_FLOPS_PER_PAIR,
                         "peak_source": ("measured: FP64 FMA throughput kernel (dvm_fp64_peak)" if fp64_peak
                                         else "nominal: 152 SMs x 2 FP64 FMA lanes/clock x 2 flop x 2.07 GHz"),
                         "peak_nominal": FP64_PEAK_GFLOPS, "hbm": hbm})
    return {
        "metric": METRIC,
        "value": replica_throughput(pairs_per_step * args.steps, ms_max / 1e3, world),
        "unit": UNIT,
        "steps": args.steps,
        "ms_per_step": ms_max / args.steps,
        "dtype": "f32" if prec == dvm.FP32 else "f64",
        "config": config_dict(cfg, prec_name, pairs_per_step,
                              {"parallelism": f"replicas{world}" if world > 1 else "single",
                               "bulk_pairs_per_step": bulk_pairs,
                               "cut_cell_cvs": counts["cvs"], "wall_cells": counts["walls"]}),
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": launches,
    }


def workload_key(cfg) -> str:
    name = cfg.get("name", "")
    for k in ("cylinder", "ellipse", "bump", "sphere"):
        if k in name:
            return k
    return name


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--workload", default="cylinder")
    ap.add_argument("--time-scheme", choices=["explicit", "imex"], default="explicit",
                    help="explicit (Eq. ExSchemeDD) or first-order semi-implicit (Eq. ImpSchemeDD) steps")
    ap.add_argument("--model", choices=["bgk", "shakhov"], default="bgk",
                    help="collision model: BGK (Eq. BGKDD) or Shakhov with Pr = 2/3 (Eq. ShakhovDD; Sec. 2.1 in 3D)")
    ap.add_argument("--equilibrium", choices=["direct", "conservative"], default="direct",
                    help="BGK equilibrium from the direct moments (Eq. MacroscopicDDv) or the conservative "
                         "Newton parameters (Sec. 3.1)")
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the drag-gradient cost measurement")
    ap.add_argument("--no-sublines", action="store_true",
                    help="default workload only: skip the FP64 and sphere sub-lines")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the error measurements")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 2000)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    from paper_1503_04544_gb300 import dvm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    cfg = workload(args.workload)
    if args.time_scheme == "imex":
        cfg["time_scheme"] = 1
    if args.model == "shakhov":
        cfg.update(model=1, Pr=2.0 / 3.0)
    if args.equilibrium == "conservative":
        cfg["conservative"] = 1
    prec = dvm.FP32 if args.precision == "fp32" else dvm.FP64
    # a dedicated stream: the library enqueues on it and the events are
    # recorded on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    peak, peak_kind = read_peaks()
    fp64_pk = dvm.fp64_peak(stream.cuda_stream)
    line = measure(cfg, prec, args, world, local, stream, peak, peak_kind, fp64_pk)
    line.update({"n_gpus": world, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                 "vs_baseline": None, "data": "synthetic"})
    default = (args.workload == "cylinder" and args.time_scheme == "explicit" and args.model == "bgk"
               and args.precision == "fp32" and args.equilibrium == "direct")
    if rank == 0 and world == 1:
        acc = {}
        cb = None
        if not args.no_cpu_baseline:
            cb = cpu_baseline(cfg, keep=True)
            if not args.no_accuracy:
                acc["vs_oracle"] = vs_oracle(cpu_sample_cfg(cfg), cb.pop("_F"), cb.pop("_fx"), cb["steps"],
                                             stream)
            cb.pop("_F", None); cb.pop("_fx", None)
            line["cpu_baseline"] = cb
        if not args.no_accuracy:
            run_len = int(cfg.get("steps", args.steps))
            if cfg.get("dim", 2) == 3:
                run_len = min(run_len, 20)    # FP64 sphere steps take ~0.3 s
            acc["fp32_vs_fp64"] = fp32_vs_fp64(cfg, run_len, stream)
        if acc:
            line["accuracy"] = acc
        if default and not args.no_adjoint:
            line["adjoint"] = adjoint_cost(True)
        if default and not args.no_sublines:
            # the FP64 half of the metric on the same workload (at most 200
            # timed steps: an FP64 step takes ~8 ms)
            a64 = argparse.Namespace(**vars(args))
            a64.steps = min(args.steps, 200)
            sub = measure(cfg, dvm.FP64, a64, world, local, stream, peak, peak_kind, fp64_pk)
            if cb is not None:
                sub["cpu_baseline"] = dict(cb, note="the same oracle sample as the main line")
            if "vs_oracle" in acc:
                sub["accuracy"] = {"vs_oracle": {"steps": acc["vs_oracle"]["steps"],
                                                 "fp64": acc["vs_oracle"]["fp64"]}}
            line["fp64"] = sub
            # the 3D sphere (96^3 cells x 20^3 velocities), FP32
            scfg = workload("sphere")
            sargs = argparse.Namespace(**vars(args))
            sargs.workload = "sphere"
            sargs.steps = min(args.steps, DEFAULT_STEPS["sphere"])
            sub3 = measure(scfg, dvm.FP32, sargs, world, local, stream, peak, peak_kind, fp64_pk)
            sacc = {}
            if not args.no_cpu_baseline:
                scb = cpu_baseline(scfg, keep=not args.no_accuracy)
                if not args.no_accuracy:
                    sacc["vs_oracle"] = vs_oracle(cpu_sample_cfg(scfg), scb.pop("_F"), scb.pop("_fx"),
                                                  scb["steps"], stream)
                scb.pop("_F", None); scb.pop("_fx", None)
                sub3["cpu_baseline"] = scb
            if not args.no_accuracy:
                sacc["fp32_vs_fp64"] = fp32_vs_fp64(scfg, min(args.steps, 10), stream)
            if sacc:
                sub3["accuracy"] = sacc
            line["sphere"] = sub3
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
