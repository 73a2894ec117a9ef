"""Corner blocks of a 3D problem for the full-size sphere parity test: the
cells [0, m)^3 of the grid as a problem of their own, with the full grid's
cell size bit for bit, so that geometry, control volumes and the state update
of the cells away from the block's high faces are the full grid's exactly."""
import numpy as np

GEO3 = ("type", "cgas", "sw", "nwx", "nwy", "nwz", "rwx", "rwy", "rwz", "vol")


def corner_block(cfg, m, dt):
    """cfg restricted to the cells [0, m) on every axis: same cell size, body,
    velocities, Knudsen number and time step; the grid's conditions on the
    low faces, zero-gradient on the high faces."""
    n = cfg["nx"]
    b = dict(cfg)
    side = None
    if cfg["bc"][0] == 1:
        # per face cell (k, j) of the x- side: the block's [0, m)^2 corner
        st = np.asarray(cfg["bc_state"][0]).reshape(cfg["nz"], cfg["ny"], 5)
        side = np.ascontiguousarray(st[:m, :m].reshape(m * m, 5))
    b.update(nx=m, ny=m, nz=m, dt=dt, bc=[cfg["bc"][0], 2, cfg["bc"][2], 2, cfg["bc"][4], 2],
             bc_state=[side, None, None, None, None, None])
    for ax in ("x", "y", "z"):
        assert cfg[ax + "min"] == 0.0 and cfg[ax + "max"] == 1.0
        b[ax + "max"] = m * (1.0 / n)
        assert b[ax + "max"] / m == 1.0 / n        # the same cell size, bit for bit
    return b


def block_view(a, n, m, shape=None):
    """The block [0, m)^3 of a full-grid per-cell (or per-face) array."""
    sh = shape or (n, n, n)
    sub = tuple(slice(0, m + (s - n)) for s in sh)
    return a.reshape(sh)[sub].ravel()


def full_index(mb, n, m):
    """Block cell indices as full-grid cell indices (negative stays)."""
    k, r = np.divmod(np.where(mb >= 0, mb, 0), m * m)
    j, i = np.divmod(r, m)
    return np.where(mb >= 0, (k * n + j) * n + i, mb)
