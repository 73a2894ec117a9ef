"""Plain FP64 CPU oracle for the cut-cell discrete-velocity method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library: the C sources next to this file are compiled on demand
into ``liboracle.so`` and called through ctypes.

A problem is described by a plain ``dict`` (see ``paper_1503_04544_gb300.workloads``
for the keys); this module converts it into the oracle's own C struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "dvm_oracle.c")]
_HDR = [os.path.join(_HERE, "dvm_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAS, CUT, SOLID = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` (gcc, -ffp-contract=off)."""
    newest = max(os.path.getmtime(p) for p in _SRC + _HDR)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("xmin", C.c_double), ("xmax", C.c_double), ("ymin", C.c_double),
        ("ymax", C.c_double), ("zmin", C.c_double), ("zmax", C.c_double),
        ("nvx", C.c_int), ("nvy", C.c_int), ("nvz", C.c_int),
        ("vxmin", C.c_double), ("vxmax", C.c_double), ("vymin", C.c_double),
        ("vymax", C.c_double), ("vzmin", C.c_double), ("vzmax", C.c_double),
        ("Kn", C.c_double), ("Lref", C.c_double), ("cfl", C.c_double), ("dt", C.c_double),
        ("scheme", C.c_int), ("bc", C.c_int * 6), ("bc_state", C.POINTER(C.c_double) * 6),
        ("shape", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("cz", C.c_double),
        ("ra", C.c_double), ("rb", C.c_double), ("theta", C.c_double), ("omega", C.c_double),
        ("vbx", C.c_double), ("vby", C.c_double), ("mass", C.c_double), ("inertia", C.c_double),
        ("movable", C.c_int), ("Tw", C.c_double), ("nseg", C.c_int),
        ("Tw_seg", C.POINTER(C.c_double)), ("seg_dir", C.POINTER(C.c_double)),
        ("axis", C.c_int), ("time_scheme", C.c_int), ("model", C.c_int), ("Pr", C.c_double),
        ("conservative", C.c_int),
    ]


_PD = C.POINTER(C.c_double)
_PI8 = C.POINTER(C.c_int8)
_PI32 = C.POINTER(C.c_int32)


class _Geo2d(C.Structure):
    _fields_ = [("phi", _PD), ("type", _PI8), ("cgas", _PI8), ("lx", _PD), ("ly", _PD),
                ("lw", _PD), ("nwx", _PD), ("nwy", _PD), ("rwx", _PD), ("rwy", _PD),
                ("sbar", _PD)]


class _Geo3d(C.Structure):
    _fields_ = [("phi", _PD), ("type", _PI8), ("cgas", _PI8), ("ax", _PD), ("ay", _PD),
                ("az", _PD), ("sw", _PD), ("nwx", _PD), ("nwy", _PD), ("nwz", _PD),
                ("rwx", _PD), ("rwy", _PD), ("rwz", _PD), ("vol", _PD)]


_GEO3D_KEYS = ("phi", "type", "cgas", "ax", "ay", "az", "sw", "nwx", "nwy", "nwz", "rwx",
               "rwy", "rwz", "vol")


class _Hist(C.Structure):
    _fields_ = [("Fx", _PD), ("Fy", _PD), ("Fz", _PD), ("torque", _PD), ("theta", _PD),
                ("omega", _PD), ("mass", _PD)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Cfg)
            lib.orc_tau0.argtypes = [P]; lib.orc_tau0.restype = C.c_double
            lib.orc_dt.argtypes = [P]; lib.orc_dt.restype = C.c_double
            lib.orc_geometry2d.argtypes = [P, C.c_double, C.c_double, C.POINTER(_Geo2d)]
            lib.orc_masters2d.argtypes = [P, C.POINTER(_Geo2d), C.POINTER(_Geo2d), _PI32]
            lib.orc_init_maxwellian.argtypes = [P, _PD, _PD, _PD, _PD, _PD, _PD]
            lib.orc_moments.argtypes = [P, _PD, _PD, _PD, _PD, _PD, _PD]
            lib.orc_run2d.argtypes = [P, _PD, C.c_int, C.POINTER(_Hist), _PD, _PD]
            lib.orc_mass2d.argtypes = [P, _PD]; lib.orc_mass2d.restype = C.c_double
            lib.orc_adjoint2d.argtypes = [P, _PD, C.c_int, _PD, _PD, _PD, _PD, _PD, _PD, _PD]
            lib.orc_init_maxwellian_vjp.argtypes = [P, _PD, _PD, _PD, _PD, _PD, _PD]
            lib.orc_adjoint2d_ex.argtypes = [P, _PD, C.c_int, C.c_int, _PD, _PD, _PD, _PD, _PD, _PD, _PD, _PD]
            lib.orc_geometry3d.argtypes = [P, C.POINTER(_Geo3d)]
            lib.orc_masters3d.argtypes = [P, C.POINTER(_Geo3d), _PI32]
            lib.orc_run3d.argtypes = [P, _PD, C.c_int, C.POINTER(_Hist)]
            lib.orc_mass3d.argtypes = [P, _PD]; lib.orc_mass3d.restype = C.c_double
            lib.orc_heat_flux.argtypes = [P, _PD, _PD]
            lib.orc_equilibrium.argtypes = [P, C.c_double, _PD, C.c_double, _PD, _PD]
            lib.orc_equilibrium_params.argtypes = [P, _PD, _PD, C.POINTER(C.c_int)]
            _lib = lib
    return _lib


def _ptr(a, t=_PD):
    return a.ctypes.data_as(t) if a is not None else None


class _CfgHolder:
    """Keeps the numpy buffers a C config points into alive."""

    def __init__(self, cfg: dict):
        s = _Cfg()
        self.keep = []
        s.dim = int(cfg.get("dim", 2))
        for k in ("nx", "ny", "nz", "nvx", "nvy", "nvz", "scheme", "shape", "movable", "nseg"):
            setattr(s, k, int(cfg.get(k, 1 if k in ("nz", "nvz") else 0)))
        for k in ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax", "vxmin", "vxmax", "vymin",
                  "vymax", "vzmin", "vzmax", "Kn", "Lref", "cfl", "dt", "cx", "cy", "cz",
                  "ra", "rb", "theta", "omega", "vbx", "vby", "mass", "inertia", "Tw"):
            setattr(s, k, float(cfg.get(k, 0.0)))
        bc = list(cfg.get("bc", [0] * 6)) + [0] * 6
        for q in range(6):
            s.bc[q] = int(bc[q])
        states = list(cfg.get("bc_state", [None] * 6)) + [None] * 6
        for q in range(6):
            if states[q] is not None:
                a = np.ascontiguousarray(states[q], dtype=np.float64)
                self.keep.append(a)
                s.bc_state[q] = _ptr(a)
        if s.nseg > 0:
            tw = np.ascontiguousarray(cfg["Tw_seg"], dtype=np.float64)
            sd = np.ascontiguousarray(cfg["seg_dir"], dtype=np.float64)
            self.keep += [tw, sd]
            s.Tw_seg = _ptr(tw)
            s.seg_dir = _ptr(sd)
        s.axis = int(cfg.get("axis", 2))
        s.time_scheme = int(cfg.get("time_scheme", 0))   # 0 explicit, 1 semi-implicit (Eq. ImpSchemeDD)
        s.model = int(cfg.get("model", 0))               # 0 BGK (Eq. BGKDD), 1 Shakhov (Eq. ShakhovDD)
        s.Pr = float(cfg.get("Pr", 1.0))
        s.conservative = int(cfg.get("conservative", 0))  # 1: Newton on the discrete moments (Sec. 3.1)
        self.s = s
        self.cfg = cfg

    @property
    def ref(self):
        return C.byref(self.s)


def ncells(cfg: dict) -> int:
    return cfg["nx"] * cfg["ny"] * (cfg.get("nz", 1) if cfg.get("dim", 2) == 3 else 1)


def nvel(cfg: dict) -> int:
    return cfg["nvx"] * cfg["nvy"] * (cfg.get("nvz", 1) if cfg.get("dim", 2) == 3 else 1)


def ncomp(cfg: dict) -> int:
    return 1 if cfg.get("dim", 2) == 3 else 2


def tau0(cfg: dict) -> float:
    return _load().orc_tau0(_CfgHolder(cfg).ref)


def time_step(cfg: dict) -> float:
    return _load().orc_dt(_CfgHolder(cfg).ref)


def geometry2d(cfg: dict, cos_t: float | None = None, sin_t: float | None = None) -> dict:
    """Appendix A geometry at the body angle of ``cfg`` (or given cos/sin)."""
    lib = _load()
    nx, ny = cfg["nx"], cfg["ny"]
    th = float(cfg.get("theta", 0.0))
    ct = np.cos(th) if cos_t is None else cos_t
    st = np.sin(th) if sin_t is None else sin_t
    out = dict(
        phi=np.zeros((ny + 1) * (nx + 1)), type=np.zeros(nx * ny, np.int8),
        cgas=np.zeros(nx * ny, np.int8), lx=np.zeros((nx + 1) * ny), ly=np.zeros(nx * (ny + 1)),
        lw=np.zeros(nx * ny), nwx=np.zeros(nx * ny), nwy=np.zeros(nx * ny),
        rwx=np.zeros(nx * ny), rwy=np.zeros(nx * ny), sbar=np.zeros(nx * ny))
    g = _Geo2d(*[_ptr(out[k], _PI8 if k in ("type", "cgas") else _PD)
                 for k in ("phi", "type", "cgas", "lx", "ly", "lw", "nwx", "nwy", "rwx",
                           "rwy", "sbar")])
    h = _CfgHolder(cfg)
    rc = lib.orc_geometry2d(h.ref, float(ct), float(st), C.byref(g))
    out["status"] = rc
    out["_struct"] = g
    return out


def masters2d(cfg: dict, gn: dict, gp: dict | None = None) -> tuple[np.ndarray, int]:
    lib = _load()
    master = np.zeros(cfg["nx"] * cfg["ny"], np.int32)
    gp = gn if gp is None else gp
    rc = lib.orc_masters2d(_CfgHolder(cfg).ref, C.byref(gn["_struct"]), C.byref(gp["_struct"]),
                           _ptr(master, _PI32))
    return master, rc


def initial_state(cfg: dict) -> np.ndarray:
    """Maxwellian initial state of ``cfg['init']``; solid cells hold zero."""
    lib = _load()
    nc = ncells(cfg)
    ini = cfg["init"]
    rho = np.array(np.broadcast_to(np.asarray(ini["rho"], np.float64), (nc,)))
    comps = [np.ascontiguousarray(np.broadcast_to(np.asarray(ini.get(k, 0.0), np.float64), (nc,)))
             for k in ("ux", "uy", "uz", "T")]
    if cfg.get("shape", 0) != 0:
        if cfg.get("dim", 2) == 2:
            g = geometry2d(cfg)
            rho[g["type"] == SOLID] = 0.0
        else:
            g = geometry3d(cfg)
            rho[g["type"] == SOLID] = 0.0
    F = np.zeros(nc * ncomp(cfg) * nvel(cfg))
    lib.orc_init_maxwellian(_CfgHolder(cfg).ref, _ptr(rho), *[_ptr(a) for a in comps], _ptr(F))
    return F


def moments(cfg: dict, F: np.ndarray) -> dict:
    lib = _load()
    nc = ncells(cfg)
    out = {k: np.zeros(nc) for k in ("rho", "ux", "uy", "uz", "T")}
    lib.orc_moments(_CfgHolder(cfg).ref, _ptr(np.ascontiguousarray(F)),
                    *[_ptr(out[k]) for k in ("rho", "ux", "uy", "uz", "T")])
    return out


def heat_flux(cfg: dict, fk: np.ndarray) -> tuple[np.ndarray, int]:
    """Heat flux q (3 components) of one cell's state ``fk`` about its own
    velocity (Eq. MacroscopicDDv in 2D, Sec. 2.1 in 3D)."""
    q = np.zeros(3)
    rc = _load().orc_heat_flux(_CfgHolder(cfg).ref, _ptr(np.ascontiguousarray(fk, np.float64)), _ptr(q))
    return q, rc


def equilibrium(cfg: dict, rho: float, u, T: float, q) -> np.ndarray:
    """One cell's equilibrium of ``cfg['model']`` (BGK, Eq. BGKDD; Shakhov,
    Eq. ShakhovDD) on the velocity grid, in the state layout."""
    out = np.zeros(ncomp(cfg) * nvel(cfg))
    u3 = np.zeros(3); u3[: len(u)] = u
    q3 = np.zeros(3); q3[: len(q)] = q
    rc = _load().orc_equilibrium(_CfgHolder(cfg).ref, float(rho), _ptr(u3), float(T), _ptr(q3), _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_equilibrium: status {rc}")
    return out


def equilibrium_params(cfg: dict, fk: np.ndarray) -> tuple[np.ndarray, int, int]:
    """(rho, ux, uy, uz, T) of one cell's equilibrium: the direct moments, or
    with cfg['conservative'] the Newton root of Sec. 3.1; the Newton
    iterations taken and the status."""
    out = np.zeros(5)
    it = C.c_int(0)
    rc = _load().orc_equilibrium_params(_CfgHolder(cfg).ref, _ptr(np.ascontiguousarray(fk, np.float64)),
                                        _ptr(out), C.byref(it))
    return out, it.value, rc


def run(cfg: dict, F: np.ndarray, nsteps: int) -> dict:
    """Advance ``F`` (modified in place) by ``nsteps`` explicit steps."""
    lib = _load()
    if cfg.get("dim", 2) != 2:
        return run3d(cfg, F, nsteps)
    hist = {k: np.zeros(max(nsteps, 1)) for k in ("Fx", "Fy", "Fz", "torque", "theta", "omega", "mass")}
    h = _Hist(*[_ptr(hist[k]) for k in ("Fx", "Fy", "Fz", "torque", "theta", "omega", "mass")])
    th = np.zeros(1)
    om = np.zeros(1)
    assert F.dtype == np.float64 and F.flags.c_contiguous
    rc = lib.orc_run2d(_CfgHolder(cfg).ref, _ptr(F), int(nsteps), C.byref(h), _ptr(th), _ptr(om))
    hist = {k: v[:nsteps] for k, v in hist.items()}
    hist.update(status=rc, theta=float(th[0]), omega=float(om[0]),
                theta_hist=hist["theta"], omega_hist=hist["omega"])
    return hist


def mass2d(cfg: dict, F: np.ndarray) -> float:
    return _load().orc_mass2d(_CfgHolder(cfg).ref, _ptr(np.ascontiguousarray(F)))


def geometry3d(cfg: dict) -> dict:
    """3D cut-cell geometry (faces from the 2D construction of Appendix A)."""
    lib = _load()
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    nc = nx * ny * nz
    out = dict(
        phi=np.zeros((nx + 1) * (ny + 1) * (nz + 1)), type=np.zeros(nc, np.int8),
        cgas=np.zeros(nc, np.int8), ax=np.zeros((nx + 1) * ny * nz),
        ay=np.zeros(nx * (ny + 1) * nz), az=np.zeros(nx * ny * (nz + 1)))
    for k in ("sw", "nwx", "nwy", "nwz", "rwx", "rwy", "rwz", "vol"):
        out[k] = np.zeros(nc)
    g = _Geo3d(*[_ptr(out[k], _PI8 if k in ("type", "cgas") else _PD) for k in _GEO3D_KEYS])
    out["status"] = lib.orc_geometry3d(_CfgHolder(cfg).ref, C.byref(g))
    out["_struct"] = g
    return out


def masters3d(cfg: dict, g: dict) -> tuple[np.ndarray, int]:
    master = np.zeros(ncells(cfg), np.int32)
    rc = _load().orc_masters3d(_CfgHolder(cfg).ref, C.byref(g["_struct"]), _ptr(master, _PI32))
    return master, rc


def run3d(cfg: dict, F: np.ndarray, nsteps: int) -> dict:
    """Advance a 3D state ``F`` (modified in place) by ``nsteps`` steps (fixed body)."""
    lib = _load()
    hist = {k: np.zeros(max(nsteps, 1)) for k in ("Fx", "Fy", "Fz", "torque", "mass")}
    h = _Hist(_ptr(hist["Fx"]), _ptr(hist["Fy"]), _ptr(hist["Fz"]), _ptr(hist["torque"]),
              None, None, _ptr(hist["mass"]))
    assert F.dtype == np.float64 and F.flags.c_contiguous
    rc = lib.orc_run3d(_CfgHolder(cfg).ref, _ptr(F), int(nsteps), C.byref(h))
    hist = {k: v[:nsteps] for k, v in hist.items()}
    hist.update(status=rc)
    return hist


def mass3d(cfg: dict, F: np.ndarray) -> float:
    return _load().orc_mass3d(_CfgHolder(cfg).ref, _ptr(np.ascontiguousarray(F)))


def adjoint2d(cfg: dict, F0: np.ndarray, nsteps: int) -> dict:
    """Drag J = F_x after ``nsteps`` steps and its discrete adjoint: dJ/dF0,
    dJ/dT_w per sector (or the uniform T_w) and dJ/d(rho, ux, uy, uz, T) of
    every Maxwellian side cell."""
    lib = _load()
    F0 = np.ascontiguousarray(F0, dtype=np.float64)
    lam0 = np.zeros_like(F0)
    ntw = max(int(cfg.get("nseg", 0)), 1)
    gTw = np.zeros(ntw)
    nside = [cfg["ny"], cfg["ny"], cfg["nx"], cfg["nx"]]
    gbc = [np.zeros(5 * n) for n in nside]
    J = np.zeros(1)
    rc = lib.orc_adjoint2d(_CfgHolder(cfg).ref, _ptr(F0), int(nsteps), _ptr(J), _ptr(lam0), _ptr(gTw),
                           *[_ptr(g) for g in gbc])
    return dict(status=rc, J=float(J[0]), lam0=lam0, gTw=gTw, gbc=[g.reshape(-1, 5) for g in gbc])


def adjoint2d_seed(cfg: dict, F0: np.ndarray, nsteps: int, seed: np.ndarray | None,
                   with_drag: bool = False) -> dict:
    """The discrete adjoint for J = [with_drag] F_x(F^N) + <seed, F^N>."""
    lib = _load()
    F0 = np.ascontiguousarray(F0, dtype=np.float64)
    lam0 = np.zeros_like(F0)
    gTw = np.zeros(max(int(cfg.get("nseg", 0)), 1))
    nside = [cfg["ny"], cfg["ny"], cfg["nx"], cfg["nx"]]
    gbc = [np.zeros(5 * n) for n in nside]
    J = np.zeros(1)
    sd = None if seed is None else np.ascontiguousarray(seed, dtype=np.float64)
    rc = lib.orc_adjoint2d_ex(_CfgHolder(cfg).ref, _ptr(F0), int(nsteps), int(bool(with_drag)), _ptr(sd),
                              _ptr(J), _ptr(lam0), _ptr(gTw), *[_ptr(g) for g in gbc])
    return dict(status=rc, J=float(J[0]), lam0=lam0, gTw=gTw, gbc=[g.reshape(-1, 5) for g in gbc])


def init_maxwellian_vjp(cfg: dict, lam: np.ndarray) -> np.ndarray:
    """d<lam, F0>/d(rho, ux, uy, uz, T) per cell for the Maxwellian initial
    state of ``cfg['init']`` (solid cells have rho = 0 and give zeros)."""
    lib = _load()
    nc = ncells(cfg)
    ini = cfg["init"]
    rho = np.array(np.broadcast_to(np.asarray(ini["rho"], np.float64), (nc,)))
    if cfg.get("shape", 0) != 0:
        rho[geometry2d(cfg)["type"] == SOLID] = 0.0
    comps = [np.ascontiguousarray(np.broadcast_to(np.asarray(ini.get(k, 0.0), np.float64), (nc,)))
             for k in ("ux", "uy", "T")]
    g = np.zeros((nc, 5))
    lib.orc_init_maxwellian_vjp(_CfgHolder(cfg).ref, _ptr(rho), *[_ptr(a) for a in comps],
                                _ptr(np.ascontiguousarray(lam, dtype=np.float64)), _ptr(g))
    return g
