"""Run one of the benchmark problems through libdvm and report what it computed.

    python -m paper_1503_04544_gb300.run --workload sphere --cells 40 --nv 16 --steps 5
    python -m paper_1503_04544_gb300.run --workload adjoint --steps 20 --checkpoint-every 10

Builds the problem (optionally at other grid and velocity sizes), installs
the Maxwellian initial state, advances ``--steps`` steps and prints one JSON
line with the force and torque of the last step, the total mass and the
measured milliseconds per step.  ``--workload adjoint`` (the cylinder with 64
wall sectors) instead computes the drag after ``--steps`` steps and its
gradient by the discrete adjoint.  Every computation runs in the CUDA library.
"""
from __future__ import annotations

import argparse
import json
import time

from . import dvm
from . import workloads as W


def problem(name: str, cells: int | None, nv: int | None, scheme: int) -> dict:
    if name == "cylinder":
        return W.cylinder_mach2(nx=cells or 256, nv=nv or 32, scheme=scheme)
    if name == "ellipse":
        return W.rotating_ellipse(nx=cells or 512, nv=nv or 40, scheme=scheme)
    if name == "bump":
        return W.periodic_bump(nx=cells or 32, nv=nv or 16)
    if name == "sphere":
        return W.sphere_mach15(n=cells or 96, nv=nv or 20, scheme=scheme)
    if name == "adjoint":
        cfg = W.cylinder_adjoint(nx=cells or 256, nv=nv or 32, nseg=64)
        cfg["scheme"] = scheme
        return cfg
    raise SystemExit(f"unknown workload {name}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="cylinder", choices=["cylinder", "ellipse", "bump", "sphere", "adjoint"])
    ap.add_argument("--cells", type=int, default=None, help="cells per axis (default: the problem's)")
    ap.add_argument("--nv", type=int, default=None, help="velocities per axis (default: the problem's)")
    ap.add_argument("--scheme", type=int, default=1, choices=[0, 1], help="0 upwind, 1 MUSCL-minmod")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--checkpoint-every", type=int, default=20)
    ap.add_argument("--time-scheme", choices=["explicit", "imex"], default="explicit")
    ap.add_argument("--model", choices=["bgk", "shakhov"], default="bgk",
                    help="collision model (Shakhov: Pr = 2/3)")
    ap.add_argument("--equilibrium", choices=["direct", "conservative"], default="direct",
                    help="BGK equilibrium from the direct moments or the conservative Newton parameters (Sec. 3.1)")
    args = ap.parse_args(argv)
    cfg = problem(args.workload, args.cells, args.nv, args.scheme)
    if args.time_scheme == "imex":
        cfg["time_scheme"] = 1
    if args.model == "shakhov":
        cfg.update(model=1, Pr=2.0 / 3.0)
    if args.equilibrium == "conservative":
        cfg["conservative"] = 1
    s = dvm.Solver(cfg, dvm.FP32 if args.precision == "fp32" else dvm.FP64)
    s.init_maxwellian()
    if args.workload == "adjoint":
        out = s.drag_adjoint(args.steps, args.checkpoint_every)
        print(json.dumps({"workload": cfg["name"], "steps": args.steps, "J": out["J"],
                          "dJ_dTw_max": float(abs(out["gTw"]).max()), "ms_forward": out["ms_forward"],
                          "ms_reverse": out["ms_reverse"]}))
        s.close()
        return
    s.step(1)
    t0 = time.perf_counter()
    s.step(args.steps)
    el = time.perf_counter() - t0
    F, tq = s.wall_force()
    print(json.dumps({"workload": cfg["name"], "steps": args.steps + 1, "ms_per_step": 1e3 * el / max(args.steps, 1),
                      "force": list(F), "torque": tq, "mass": s.mass(), "cells": s.cell_counts()}))
    s.close()


if __name__ == "__main__":
    main()
