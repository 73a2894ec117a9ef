"""Seeded synthetic workloads: problem statements and random inputs.

This module holds no arithmetic of the method.  It only states problems
(grid, velocity window, physical parameters, boundary kinds, obstacle and
initial macroscopic fields) as plain dicts and draws seeded random numbers.
Both the CUDA library binding and the CPU oracle accept these dicts.

Keys of a problem dict
----------------------
dim                 2 or 3
nx, ny, nz          cells per axis on [xmin,xmax] x [ymin,ymax] (x [zmin,zmax])
nvx, nvy, nvz       velocity points per axis; the grid is v = vmin + p*(vmax-vmin)/n,
                    p = 0..n-1 (Sec. 3.1, taken literally: vmax is excluded)
Kn, Lref            Knudsen number and its reference length
cfl, dt             CFL number; dt > 0 overrides the CFL rule
scheme              0 first-order upwind, 1 MUSCL-minmod
bc                  6 ints for the x-, x+, y-, y+, z-, z+ sides:
                    0 periodic, 1 Maxwellian ghost, 2 zero-gradient
bc_state            per side: None or an array (n_side_cells, 5) of
                    (rho, ux, uy, uz, T) for Maxwellian sides
shape               0 none, 1 circle, 2 ellipse, 3 sphere, 4 disk container,
                    5 box container (2D; the gas inside, half-widths ra, rb)
                    (in 3D, 1 is an infinite circular cylinder along ``axis``)
axis                3D cylinder axis: 0 x, 1 y, 2 z
cx, cy, cz, ra, rb  obstacle centre, radius (ra) or semi-axes (ra, rb)
theta, omega        body angle and angular velocity
mass, inertia       rigid-body mass and moment of inertia
movable             1: the body rotates freely about its centre
Tw                  wall temperature; nseg > 0 with Tw_seg, seg_dir gives
                    piecewise-constant temperatures per angular sector
init                dict of per-cell (or scalar) rho, ux, uy, uz, T
steps               number of steps of the full run
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 5.0 / 3.0   # monatomic gas


def mach_speed(mach: float, T: float = 1.0) -> float:
    """Free-stream speed of a Mach number in units of sqrt(R T0)."""
    return mach * math.sqrt(GAMMA * T)


def _cell_centres(nx, ny, xmin=0.0, xmax=1.0, ymin=0.0, ymax=1.0):
    dx = (xmax - xmin) / nx
    dy = (ymax - ymin) / ny
    x = xmin + (np.arange(nx) + 0.5) * dx
    y = ymin + (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)        # [j, i]
    return X.ravel(), Y.ravel()


def _side_state(n, rho=1.0, ux=0.0, uy=0.0, uz=0.0, T=1.0):
    s = np.zeros((n, 5))
    s[:, 0] = rho
    s[:, 1] = ux
    s[:, 2] = uy
    s[:, 3] = uz
    s[:, 4] = T
    return s


def base2d(nx, ny, nv, vwin, **kw) -> dict:
    cfg = dict(dim=2, nx=nx, ny=ny, nz=1, xmin=0.0, xmax=1.0, ymin=0.0, ymax=1.0,
               zmin=0.0, zmax=1.0, nvx=nv, nvy=nv, nvz=1,
               vxmin=-vwin, vxmax=vwin, vymin=-vwin, vymax=vwin, vzmin=0.0, vzmax=1.0,
               Kn=0.1, Lref=1.0, cfl=0.5, dt=0.0, scheme=0, bc=[0] * 6,
               bc_state=[None] * 6, shape=0, cx=0.5, cy=0.5, cz=0.5, ra=0.0, rb=0.0,
               theta=0.0, omega=0.0, vbx=0.0, vby=0.0, mass=1.0, inertia=1.0, movable=0,
               Tw=1.0, nseg=0, init=dict(rho=1.0, ux=0.0, uy=0.0, uz=0.0, T=1.0), steps=1)
    cfg.update(kw)
    return cfg


def base3d(n, nv, vwin, **kw) -> dict:
    """A 3D problem on the unit cube with n cells and nv velocities per axis."""
    cfg = base2d(n, n, nv, vwin, dim=3, nz=n, nvz=nv, vzmin=-vwin, vzmax=vwin, axis=2)
    cfg.update(kw)
    return cfg


# ------------------------------------------------------------------ the five
# benchmark problems (sizes and parameters as stated for the method's
# hot path; synthetic stand-ins for the paper's figure-only experiments)

def periodic_bump(nx=32, nv=16) -> dict:
    """2D FP64, no obstacle: periodic unit square, Gaussian density bump."""
    X, Y = _cell_centres(nx, nx)
    rho = 1.0 + 0.1 * np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2) / 0.01)
    return base2d(nx, nx, nv, 6.0, Kn=0.1, Lref=1.0, cfl=0.5, scheme=0,
                  init=dict(rho=rho, ux=0.0, uy=0.0, uz=0.0, T=1.0), steps=20,
                  name=f"periodic_bump_{nx}x{nx}_v{nv}x{nv}")


def cylinder_mach2(nx=256, nv=32, scheme=1, mach=2.0, Tw=1.0) -> dict:
    """2D fixed cylinder r=0.1, Mach-2 inflow on the left, outflow elsewhere."""
    u = mach_speed(mach)
    bc_state = [_side_state(nx, ux=u), None, None, None, None, None]
    return base2d(nx, nx, nv, 8.0, Kn=0.05, Lref=0.2, cfl=0.5, scheme=scheme,
                  bc=[1, 2, 2, 2, 0, 0], bc_state=bc_state, shape=1, cx=0.5, cy=0.5,
                  ra=0.1, Tw=Tw, init=dict(rho=1.0, ux=u, uy=0.0, uz=0.0, T=1.0),
                  steps=2000, name=f"cylinder_mach{mach:g}_{nx}x{nx}_v{nv}x{nv}")


def rotating_ellipse(nx=512, nv=40, scheme=0) -> dict:
    """2D ellipse (0.12 x 0.04) rotating freely in a shear flow."""
    dy = 1.0 / nx
    yc = (np.arange(nx) + 0.5) * dy
    shear = 0.5 * (2.0 * yc - 1.0)
    left = _side_state(nx)
    left[:, 1] = shear
    right = left.copy()
    X, Y = _cell_centres(nx, nx)
    return base2d(nx, nx, nv, 6.0, Kn=0.02, Lref=0.24, cfl=0.5, scheme=scheme,
                  bc=[1, 1, 2, 2, 0, 0], bc_state=[left, right, None, None, None, None],
                  shape=2, cx=0.5, cy=0.5, ra=0.12, rb=0.04, theta=0.0, omega=0.0,
                  mass=1.0, inertia=1e-3, movable=1, Tw=1.0,
                  init=dict(rho=1.0, ux=0.5 * (2.0 * Y - 1.0), uy=0.0, uz=0.0, T=1.0),
                  steps=5000, name=f"rotating_ellipse_{nx}x{nx}_v{nv}x{nv}")


def disk_container(nx=64, nv=20, scheme=1, ra=0.45, Tw=1.3) -> dict:
    """2D closed disk container of radius ra, diffuse wall at Tw, holding a
    gas at rest (T = 1) with a density bump off the centre."""
    X, Y = _cell_centres(nx, nx)
    rho = 1.0 + 0.3 * np.exp(-((X - 0.42) ** 2 + (Y - 0.55) ** 2) / 0.01)
    return base2d(nx, nx, nv, 8.0, Kn=0.1, Lref=1.0, cfl=0.5, scheme=scheme,
                  shape=4, cx=0.5, cy=0.5, ra=ra, Tw=Tw,
                  init=dict(rho=rho, ux=0.0, uy=0.0, uz=0.0, T=1.0), steps=200,
                  name=f"disk_container_{nx}x{nx}_v{nv}x{nv}")


def box_container(nx=64, nv=20, scheme=1, ra=0.41, rb=0.33, Tw=1.3) -> dict:
    """2D closed box container with half-widths ra, rb about the centre of
    the domain, diffuse wall at Tw, a drifting gas with a density bump."""
    X, Y = _cell_centres(nx, nx)
    rho = 1.0 + 0.3 * np.exp(-((X - 0.42) ** 2 + (Y - 0.55) ** 2) / 0.01)
    return base2d(nx, nx, nv, 8.0, Kn=0.1, Lref=1.0, cfl=0.5, scheme=scheme,
                  shape=5, cx=0.5013, cy=0.4987, ra=ra, rb=rb, Tw=Tw,
                  init=dict(rho=rho, ux=0.3, uy=-0.2, uz=0.0, T=1.0), steps=200,
                  name=f"box_container_{nx}x{nx}_v{nv}x{nv}")


def sphere_mach15(n=96, nv=20, scheme=1) -> dict:
    """3D fixed sphere r=0.15, Mach-1.5 inflow on x-, outflow elsewhere."""
    u = mach_speed(1.5)
    cfg = base2d(n, n, nv, 5.0, dim=3, nz=n, nvz=nv, vzmin=-5.0, vzmax=5.0,
                 Kn=0.1, Lref=0.3, cfl=0.5, scheme=scheme, bc=[1, 2, 2, 2, 2, 2],
                 bc_state=[_side_state(n * n, ux=u), None, None, None, None, None],
                 shape=3, cx=0.5, cy=0.5, cz=0.5, ra=0.15, Tw=1.0,
                 init=dict(rho=1.0, ux=u, uy=0.0, uz=0.0, T=1.0), steps=500,
                 name=f"sphere_mach1.5_{n}^3_v{nv}^3")
    return cfg


def segment_directions(nseg: int) -> np.ndarray:
    """Unit directions bounding the angular sectors of per-segment walls."""
    a = 2.0 * np.pi * np.arange(nseg) / nseg
    return np.stack([np.cos(a), np.sin(a)], axis=1).ravel()


def cylinder_adjoint(nx=256, nv=32, nseg=64, seed=0, mach=2.0, steps=200) -> dict:
    """Cylinder flow with 64 per-sector wall temperatures in [0.8, 1.2]."""
    cfg = cylinder_mach2(nx, nv, mach=mach)
    rng = np.random.default_rng(seed)
    cfg.update(nseg=nseg, Tw_seg=rng.uniform(0.8, 1.2, nseg), seg_dir=segment_directions(nseg),
               steps=steps, checkpoint_every=20, mach=mach,
               name=f"cylinder_adjoint_{nx}x{nx}_v{nv}x{nv}_seg{nseg}")
    return cfg


# ------------------------------------------------------------ seeded inputs

def perturbation(n: int, seed: int, amp: float = 0.1) -> np.ndarray:
    """Seeded multiplicative perturbation factors 1 + amp*U(-1, 1)."""
    rng = np.random.default_rng(seed)
    return 1.0 + amp * rng.uniform(-1.0, 1.0, n)


def uniform_random(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n)
