"""ctypes binding of libdvm (include/dvm.h): argument marshalling only.

Every computation runs in the CUDA library.  ``load()`` raises if the
library is missing or cannot be loaded; there is no fallback.

``Solver(cfg, precision)`` builds a context from a problem dict (keys in
:mod:`paper_1503_04544_gb300.workloads`) and exposes the C entry points with
the same names.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdvm.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CFL, ERR_GEOMETRY, ERR_NONPHYSICAL, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_UNSUPPORTED = range(9)
FP32, FP64 = 32, 64
UPWIND, MUSCL = 0, 1
PERIODIC, MAXWELLIAN, ZEROGRAD = 0, 1, 2
EXPLICIT, IMEX = 0, 1
BGK, SHAKHOV = 0, 1


class DVMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdvm error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double),
                ("ymax", C.c_double), ("zmin", C.c_double), ("zmax", C.c_double)]


class VGrid(C.Structure):
    _fields_ = [("nvx", C.c_int), ("nvy", C.c_int), ("nvz", C.c_int),
                ("vxmin", C.c_double), ("vxmax", C.c_double), ("vymin", C.c_double),
                ("vymax", C.c_double), ("vzmin", C.c_double), ("vzmax", C.c_double)]


class Physics(C.Structure):
    _fields_ = [("Kn", C.c_double), ("Lref", C.c_double), ("cfl", C.c_double), ("dt", C.c_double)]


class Body(C.Structure):
    _fields_ = [("shape", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
                ("ra", C.c_double), ("rb", C.c_double), ("theta", C.c_double),
                ("omega", C.c_double), ("vbx", C.c_double), ("vby", C.c_double),
                ("mass", C.c_double), ("inertia", C.c_double), ("movable", C.c_int),
                ("Tw", C.c_double), ("nseg", C.c_int), ("Tw_seg", C.POINTER(C.c_double)),
                ("seg_dir", C.POINTER(C.c_double))]


_PD = C.POINTER(C.c_double)
_PI8 = C.POINTER(C.c_int8)
_PI32 = C.POINTER(C.c_int32)
_P = C.c_void_p

# name -> argtypes; every entry point returns int except the two below
SIGNATURES = {
    "dvm_create": [C.POINTER(Grid), C.POINTER(VGrid), C.POINTER(Physics), C.c_int, C.c_int, _P,
                   C.POINTER(_P)],
    "dvm_destroy": [_P],
    "dvm_set_bc": [_P, C.c_int, C.c_int, _PD],
    "dvm_set_body": [_P, C.POINTER(Body)],
    "dvm_init_maxwellian": [_P, _PD, _PD, _PD, _PD, _PD],
    "dvm_set_state": [_P, _P, C.c_size_t, C.c_int],
    "dvm_get_state": [_P, _P, C.c_size_t, C.c_int],
    "dvm_step": [_P, C.c_int],
    "dvm_step_async": [_P, C.c_int],
    "dvm_graphs": [_P, C.c_int],
    "dvm_rollback": [_P, C.c_int],
    "dvm_save": [_P, C.c_char_p],
    "dvm_load": [_P, C.c_char_p],
    "dvm_set_time_scheme": [_P, C.c_int],
    "dvm_set_collision_model": [_P, C.c_int, C.c_double],
    "dvm_set_adjoint_tape": [_P, C.c_size_t],
    "dvm_set_equilibrium": [_P, C.c_int],
    "dvm_check": [_P],
    "dvm_moments": [_P, _P, _P, _P, _P, _P, C.c_int],
    "dvm_set_velocity_split": [_P, C.POINTER(VGrid)],
    "dvm_split_size": [_P, C.POINTER(C.c_size_t)],
    "dvm_split_begin": [_P, _P],
    "dvm_split_finish": [_P, _P],
    "dvm_split_relax": [_P, _P],
    "dvm_wall_force": [_P, _PD, _PD],
    "dvm_history": [_P, _PD, _PD, _PD, _PD, _PD, _PD, C.c_int, C.POINTER(C.c_int)],
    "dvm_body_state": [_P, _PD, _PD],
    "dvm_mass": [_P, _PD],
    "dvm_info": [_P, _PD, _PD, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int),
                 C.POINTER(C.c_int)],
    "dvm_geometry2d": [_P, _PI8, _PI8, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PI32],
    "dvm_geometry2d_at": [_P, C.c_double, C.c_double],
    "dvm_geometry3d": [_P, _PI8, _PI8, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PI32],
    "dvm_drag_adjoint": [_P, C.c_int, C.c_int, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD],
    "dvm_adjoint": [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int, _P, C.c_int, _PD, _PD, _PD, _PD, _PD, _PD, _PD],
    "dvm_step_vjp": [_P, _P, _P, C.c_int, _PD],
    "dvm_timing": [_P, C.c_int],
    "dvm_kernel_time": [_P, _PD, C.POINTER(C.c_longlong)],
    "dvm_launches": [_P, C.POINTER(C.c_longlong)],
    "dvm_cell_counts": [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                        C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)],
    "dvm_mass_noalloc": [_P, C.c_int, C.c_longlong, C.c_int, C.c_int, _P, C.c_double, _P, _P],
    "dvm_fp64_peak": [_P, _PD],
    "dvm_last_error": [],
}


def load():
    """Load libdvm.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            lib = C.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = C.c_int
            lib.dvm_destroy.restype = None
            lib.dvm_last_error.restype = C.c_char_p
            _lib = lib
    return _lib


def fp64_peak(stream: int | None = None) -> float:
    """FP64 FMA throughput of the current device in GFLOP/s (dvm_fp64_peak)."""
    out = C.c_double(0.0)
    _check(load().dvm_fp64_peak(_P(stream) if stream else None, C.byref(out)))
    return out.value


def _ptr(a, t=_PD):
    return a.ctypes.data_as(t) if a is not None else None


def _check(rc: int):
    if rc != OK:
        raise DVMError(rc, load().dvm_last_error().decode())


class Solver:
    """One libdvm context for a problem dict."""

    def __init__(self, cfg: dict, precision: int = FP64, stream: int | None = None):
        lib = load()
        self.cfg = cfg
        self.precision = precision
        g = Grid(int(cfg.get("dim", 2)), cfg["nx"], cfg["ny"], int(cfg.get("nz", 1)),
                 cfg.get("xmin", 0.0), cfg.get("xmax", 1.0), cfg.get("ymin", 0.0),
                 cfg.get("ymax", 1.0), cfg.get("zmin", 0.0), cfg.get("zmax", 1.0))
        v = VGrid(cfg["nvx"], cfg["nvy"], int(cfg.get("nvz", 1)), cfg["vxmin"], cfg["vxmax"],
                  cfg["vymin"], cfg["vymax"], cfg.get("vzmin", 0.0), cfg.get("vzmax", 1.0))
        ph = Physics(cfg["Kn"], cfg["Lref"], cfg.get("cfl", 0.5), cfg.get("dt", 0.0))
        h = _P()
        _check(lib.dvm_create(C.byref(g), C.byref(v), C.byref(ph), int(precision),
                              int(cfg.get("scheme", 0)), _P(stream) if stream else None, C.byref(h)))
        self.h = h
        if cfg.get("vsplit_global") is not None:
            gv = cfg["vsplit_global"]
            _check(lib.dvm_set_velocity_split(h, C.byref(VGrid(gv["nvx"], gv["nvy"], int(gv.get("nvz", 1)),
                                                                gv["vxmin"], gv["vxmax"], gv["vymin"], gv["vymax"],
                                                                gv.get("vzmin", 0.0), gv.get("vzmax", 1.0)))))
        dim = int(cfg.get("dim", 2))
        states = list(cfg.get("bc_state", [None] * 6)) + [None] * 6
        for side, kind in enumerate(list(cfg.get("bc", [0] * 6))[: 2 * dim]):
            st = None
            if kind == MAXWELLIAN:
                st = np.ascontiguousarray(states[side], dtype=np.float64)
            _check(lib.dvm_set_bc(h, side, int(kind), _ptr(st)))
        self._keep = []
        self.time_scheme = EXPLICIT
        if cfg.get("shape", 0):
            self.set_body(cfg)
        if int(cfg.get("time_scheme", 0)):
            self.set_time_scheme(int(cfg["time_scheme"]))
        if int(cfg.get("model", 0)):
            self.set_collision_model(int(cfg["model"]), float(cfg.get("Pr", 1.0)))
        if int(cfg.get("conservative", 0)):
            self.set_equilibrium(int(cfg["conservative"]))
        dt = C.c_double()
        tau0 = C.c_double()
        nc = C.c_longlong()
        nv = C.c_int()
        ncomp = C.c_int()
        el = C.c_int()
        _check(lib.dvm_info(h, C.byref(dt), C.byref(tau0), C.byref(nc), C.byref(nv), C.byref(ncomp),
                            C.byref(el)))
        self.dt, self.tau0 = dt.value, tau0.value
        self.ncell, self.nv, self.ncomp, self.elem = nc.value, nv.value, ncomp.value, el.value
        self.dtype = np.float32 if self.elem == 4 else np.float64

    # -------------------------------------------------------------- set-up
    def set_body(self, cfg: dict):
        nseg = int(cfg.get("nseg", 0))
        tw = sd = None
        if nseg > 0:
            tw = np.ascontiguousarray(cfg["Tw_seg"], dtype=np.float64)
            sd = np.ascontiguousarray(cfg["seg_dir"], dtype=np.float64)
        b = Body(int(cfg.get("shape", 0)), cfg.get("cx", 0.5), cfg.get("cy", 0.5), cfg.get("cz", 0.5),
                 cfg.get("ra", 0.0), cfg.get("rb", 0.0), cfg.get("theta", 0.0), cfg.get("omega", 0.0),
                 cfg.get("vbx", 0.0), cfg.get("vby", 0.0), cfg.get("mass", 1.0),
                 cfg.get("inertia", 1.0), int(cfg.get("movable", 0)), cfg.get("Tw", 1.0), nseg,
                 _ptr(tw), _ptr(sd))
        _check(load().dvm_set_body(self.h, C.byref(b)))

    def init_maxwellian(self, init: dict | None = None):
        init = self.cfg["init"] if init is None else init
        n = self.ncell
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(init.get(k, d), np.float64), (n,)))
                for k, d in (("rho", 1.0), ("ux", 0.0), ("uy", 0.0), ("uz", 0.0), ("T", 1.0))]
        _check(load().dvm_init_maxwellian(self.h, *[_ptr(a) for a in arrs]))

    @property
    def state_size(self) -> int:
        return self.ncell * self.ncomp * self.nv

    def set_state(self, F):
        """Install a state from a numpy array or a torch tensor (host or CUDA)."""
        if isinstance(F, np.ndarray):
            a = np.ascontiguousarray(F, dtype=self.dtype)
            _check(load().dvm_set_state(self.h, a.ctypes.data, a.nbytes, 0))
        else:
            _check(load().dvm_set_state(self.h, F.data_ptr(), F.numel() * F.element_size(),
                                        1 if F.is_cuda else 0))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.state_size, self.dtype)
        if isinstance(out, np.ndarray):
            _check(load().dvm_get_state(self.h, out.ctypes.data, out.nbytes, 0))
        else:
            _check(load().dvm_get_state(self.h, out.data_ptr(), out.numel() * out.element_size(),
                                        1 if out.is_cuda else 0))
        return out

    # -------------------------------------------------------------- stepping
    def step(self, n: int = 1):
        _check(load().dvm_step(self.h, int(n)))

    def step_async(self, n: int = 1):
        _check(load().dvm_step_async(self.h, int(n)))

    def save(self, path: str):
        """Checkpoint the context's state, moment sums and body to ``path`` (dvm_save)."""
        _check(load().dvm_save(self.h, os.fsencode(path)))

    def load(self, path: str):
        """Restart from a checkpoint of the same problem (dvm_load)."""
        _check(load().dvm_load(self.h, os.fsencode(path)))

    def set_time_scheme(self, scheme: int):
        """0: explicit (Eq. ExSchemeDD), 1: first-order semi-implicit (Eq. ImpSchemeDD)."""
        _check(load().dvm_set_time_scheme(self.h, int(scheme)))
        self.time_scheme = int(scheme)

    def set_adjoint_tape(self, max_bytes: int):
        """Device bytes the adjoint may use to keep the forward run's tape of
        whole checkpoint segments, so that the reverse sweep does not
        recompute them (0, the default: recompute every segment)."""
        _check(load().dvm_set_adjoint_tape(self.h, int(max_bytes)))

    def set_collision_model(self, model: int, Pr: float = 1.0):
        """0: BGK (Eq. BGKDD), 1: Shakhov with Prandtl number Pr (Eq. ShakhovDD)."""
        _check(load().dvm_set_collision_model(self.h, int(model), float(Pr)))

    def set_equilibrium(self, mode: int):
        """0: the equilibrium takes the direct moments (Eq. MacroscopicDDv);
        1: the conservative parameters found by Newton's method (Sec. 3.1)."""
        _check(load().dvm_set_equilibrium(self.h, int(mode)))

    def rollback(self, enable: bool = True):
        """dvm_step leaves the state at the last good step on a failure (on by default)."""
        _check(load().dvm_rollback(self.h, int(bool(enable))))

    def graphs(self, enable: bool = True):
        """Two-step CUDA graph replays in step / step_async (on by default)."""
        _check(load().dvm_graphs(self.h, int(bool(enable))))

    def check(self):
        _check(load().dvm_check(self.h))

    # -------------------------------------------------------------- outputs
    def moments(self, out: dict | None = None) -> dict:
        """rho, ux, uy, uz, T per cell: numpy arrays, or the CUDA float64
        tensors of ``out`` (written on the device, no host copy)."""
        if out is not None:
            keys = ("rho", "ux", "uy", "uz", "T")
            _check(load().dvm_moments(self.h, *[_P(out[k].data_ptr()) if out.get(k) is not None else None
                                                for k in keys], 1))
            return out
        out = {k: np.zeros(self.ncell) for k in ("rho", "ux", "uy", "uz", "T")}
        _check(load().dvm_moments(self.h, *[_P(out[k].ctypes.data) for k in ("rho", "ux", "uy", "uz", "T")], 0))
        return out

    # -------------------------------------------------------------- velocity split
    def split_size(self) -> int:
        n = C.c_size_t()
        _check(load().dvm_split_size(self.h, C.byref(n)))
        return n.value

    def split_begin(self, xbuf):
        """This rank's moment and wall sums into the CUDA tensor ``xbuf``."""
        _check(load().dvm_split_begin(self.h, _P(xbuf.data_ptr())))

    def split_finish(self, xbuf):
        """Finish the step from ``xbuf`` summed over the ranks.  Under the
        semi-implicit scheme: transport, and this rank's moment sums of the
        transported values into ``xbuf`` for the second exchange."""
        _check(load().dvm_split_finish(self.h, _P(xbuf.data_ptr())))

    def split_relax(self, xbuf):
        """Semi-implicit scheme: relax from ``xbuf`` summed over the ranks
        again, and end the step."""
        _check(load().dvm_split_relax(self.h, _P(xbuf.data_ptr())))

    def wall_force(self):
        F = np.zeros(3)
        tq = np.zeros(1)
        _check(load().dvm_wall_force(self.h, _ptr(F), _ptr(tq)))
        return F, float(tq[0])

    def history(self, n: int) -> dict:
        out = {k: np.zeros(max(n, 1)) for k in ("Fx", "Fy", "Fz", "torque", "theta", "omega")}
        cnt = C.c_int()
        _check(load().dvm_history(self.h, *[_ptr(out[k]) for k in ("Fx", "Fy", "Fz", "torque", "theta", "omega")],
                                  int(n), C.byref(cnt)))
        return {k: v[: cnt.value] for k, v in out.items()}

    def body_state(self):
        th = np.zeros(1)
        om = np.zeros(1)
        _check(load().dvm_body_state(self.h, _ptr(th), _ptr(om)))
        return float(th[0]), float(om[0])

    def mass(self) -> float:
        m = np.zeros(1)
        _check(load().dvm_mass(self.h, _ptr(m)))
        return float(m[0])

    def geometry2d(self) -> dict:
        nx, ny = self.cfg["nx"], self.cfg["ny"]
        nc = nx * ny
        out = dict(type=np.zeros(nc, np.int8), cgas=np.zeros(nc, np.int8),
                   lx=np.zeros((nx + 1) * ny), ly=np.zeros(nx * (ny + 1)), lw=np.zeros(nc),
                   nwx=np.zeros(nc), nwy=np.zeros(nc), rwx=np.zeros(nc), rwy=np.zeros(nc),
                   sbar=np.zeros(nc), master=np.zeros(nc, np.int32))
        _check(load().dvm_geometry2d(
            self.h, _ptr(out["type"], _PI8), _ptr(out["cgas"], _PI8),
            *[_ptr(out[k]) for k in ("lx", "ly", "lw", "nwx", "nwy", "rwx", "rwy", "sbar")],
            _ptr(out["master"], _PI32)))
        return out

    def geometry3d(self) -> dict:
        nx, ny, nz = self.cfg["nx"], self.cfg["ny"], self.cfg["nz"]
        nc = nx * ny * nz
        out = dict(type=np.zeros(nc, np.int8), cgas=np.zeros(nc, np.int8),
                   ax=np.zeros((nx + 1) * ny * nz), ay=np.zeros(nx * (ny + 1) * nz),
                   az=np.zeros(nx * ny * (nz + 1)), master=np.zeros(nc, np.int32))
        for k in ("sw", "nwx", "nwy", "nwz", "rwx", "rwy", "rwz", "vol"):
            out[k] = np.zeros(nc)
        _check(load().dvm_geometry3d(
            self.h, _ptr(out["type"], _PI8), _ptr(out["cgas"], _PI8),
            *[_ptr(out[k]) for k in ("ax", "ay", "az", "sw", "nwx", "nwy", "nwz", "rwx", "rwy", "rwz", "vol")],
            _ptr(out["master"], _PI32)))
        return out

    def geometry2d_at(self, cos_t: float, sin_t: float):
        _check(load().dvm_geometry2d_at(self.h, float(cos_t), float(sin_t)))

    def drag_adjoint(self, nsteps: int, checkpoint_every: int = 20, want_init: bool = True) -> dict:
        """Drag J = F_x after ``nsteps`` steps and its gradient (dvm_drag_adjoint):
        dJ/dT_w per sector, per Maxwellian side cell and per initial-state
        cell, with the device times of the forward and reverse sweeps."""
        ns = max(int(self.cfg.get("nseg", 0)), 1)
        gtw = np.zeros(ns)
        nside = [self.cfg["ny"], self.cfg["ny"], self.cfg["nx"], self.cfg["nx"]]
        gbc = [np.zeros(5 * n) for n in nside]
        gp = np.zeros(5 * self.ncell) if want_init else None
        J = np.zeros(1)
        tf = np.zeros(1)
        tr = np.zeros(1)
        _check(load().dvm_drag_adjoint(self.h, int(nsteps), int(checkpoint_every), _ptr(J), _ptr(gtw),
                                       *[_ptr(g) for g in gbc], _ptr(gp), _ptr(tf), _ptr(tr)))
        return dict(J=float(J[0]), gTw=gtw, gbc=[g.reshape(-1, 5) for g in gbc],
                    gprim0=None if gp is None else gp.reshape(-1, 5), ms_forward=float(tf[0]),
                    ms_reverse=float(tr[0]))

    def adjoint(self, nsteps: int, checkpoint_every: int = 20, with_drag: bool = False, seed=None,
                want_lambda0: bool = True, want_init: bool = False) -> dict:
        """Gradient of J = [with_drag] F_x(F^N) + <seed, F^N> (dvm_adjoint).
        ``seed``: numpy array or CUDA tensor in the public layout; lambda0 is
        returned the same way (a CUDA tensor if the seed is one)."""
        ns = max(int(self.cfg.get("nseg", 0)), 1)
        gtw = np.zeros(ns)
        nside = [self.cfg["ny"], self.cfg["ny"], self.cfg["nx"], self.cfg["nx"]]
        gbc = [np.zeros(5 * n) for n in nside]
        gp = np.zeros(5 * self.ncell) if want_init else None
        J = np.zeros(1)
        dev = seed is not None and not isinstance(seed, np.ndarray)
        if seed is None:
            sp, sd = None, 0
        elif dev:
            sp, sd = _P(seed.data_ptr()), 1
        else:
            seed = np.ascontiguousarray(seed, dtype=self.dtype)
            sp, sd = _P(seed.ctypes.data), 0
        lam = None
        lp = None
        if want_lambda0:
            if dev:
                import torch
                lam = torch.empty(self.state_size, dtype=seed.dtype, device=seed.device)
                lp = _P(lam.data_ptr())
            else:
                lam = np.empty(self.state_size, self.dtype)
                lp = _P(lam.ctypes.data)
        _check(load().dvm_adjoint(self.h, int(nsteps), int(checkpoint_every), int(bool(with_drag)), sp, sd, lp,
                                  1 if dev else 0, _ptr(J), _ptr(gtw), *[_ptr(g) for g in gbc], _ptr(gp)))
        return dict(J=float(J[0]), gTw=gtw, lambda0=lam, gbc=[g.reshape(-1, 5) for g in gbc],
                    gprim0=None if gp is None else gp.reshape(-1, 5))

    def step_vjp(self, lam_np1) -> tuple:
        """One transposed step around the current state (dvm_step_vjp): returns
        (lambda_n, dJ/dT_w); the context advances one step."""
        ns = max(int(self.cfg.get("nseg", 0)), 1)
        gtw = np.zeros(ns)
        if isinstance(lam_np1, np.ndarray):
            lam_np1 = np.ascontiguousarray(lam_np1, dtype=self.dtype)
            out = np.empty(self.state_size, self.dtype)
            _check(load().dvm_step_vjp(self.h, _P(lam_np1.ctypes.data), _P(out.ctypes.data), 0, _ptr(gtw)))
        else:
            import torch
            out = torch.empty_like(lam_np1)
            _check(load().dvm_step_vjp(self.h, _P(lam_np1.data_ptr()), _P(out.data_ptr()), 1, _ptr(gtw)))
        return out, gtw

    # -------------------------------------------------------------- instrumentation
    def timing(self, enable):
        """Event timing of one kernel per step: True/1 the bulk kernel, 2 the
        Shakhov term, False/0 off."""
        _check(load().dvm_timing(self.h, int(enable)))

    def kernel_time(self):
        ms = C.c_double()
        n = C.c_longlong()
        _check(load().dvm_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launches(self) -> int:
        n = C.c_longlong()
        _check(load().dvm_launches(self.h, C.byref(n)))
        return n.value

    def cell_counts(self) -> dict:
        v = [C.c_longlong() for _ in range(4)]
        _check(load().dvm_cell_counts(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("nonsolid", "bulk", "cvs", "walls"), (x.value for x in v)))

    def close(self):
        if getattr(self, "h", None):
            load().dvm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
