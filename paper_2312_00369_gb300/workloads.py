"""Seeded synthetic inputs: solid masks, droplet lists, contact-angle fields.

This module holds no arithmetic of the lattice Boltzmann method. It only
describes geometry and initial droplets, and both the CUDA path and the CPU
oracle are driven from the same descriptions. Everything is numpy on the host.

Geometry conventions
--------------------
* ``solid[y, x] = 1`` marks a solid node; x is periodic; rows 0, 1, ny-2 and
  ny-1 are always solid (the library requires it).
* A node is solid when its centre lies strictly inside the solid region.
* ``wall`` describes the effective wall used by the contact-angle fit: the
  plane halfway between the ghost layer and the boundary layer, i.e. the
  geometric surface of the solid region moved one lattice spacing into the
  solid (for a flat wall whose top solid row is ``y_b`` that is ``y_b - 1/2``).
  ``type`` 0 is a straight wall through (px, py) with unit normal (nx, ny)
  pointing into the fluid; ``type`` 1 is a circular solid of centre (px, py)
  and radius r.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    """One solve: geometry, droplets, material parameters, step count."""
    name: str
    solid: np.ndarray                      # uint8 [ny, nx]
    droplets: list                         # [(x0, y0, R), ...]
    wall: dict                             # effective wall for the angle fit
    theta_deg: float = 90.0
    theta_field: np.ndarray | None = None  # float32 [ny, nx] degrees, or None
    sigma: float = 0.01
    W: float = 4.0
    M: float = 0.1
    tau_f: float = 0.8
    rho_l: float = 1.0
    rho_g: float = 0.1
    steps: int = 1000
    meta: dict = field(default_factory=dict)

    @property
    def nx(self) -> int:
        return int(self.solid.shape[1])

    @property
    def ny(self) -> int:
        return int(self.solid.shape[0])

    def physical(self) -> dict:
        return dict(sigma=self.sigma, W=self.W, M=self.M, tau_f=self.tau_f,
                    rho_l=self.rho_l, rho_g=self.rho_g)


def _frame(nx: int, ny: int) -> np.ndarray:
    s = np.zeros((ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    return s


def flat_channel(nx: int, ny: int, bottom: int = 2, top: int = 2):
    """Solid rows [0, bottom) and [ny-top, ny); returns (solid, wall)."""
    assert bottom >= 2 and top >= 2
    s = np.zeros((ny, nx), np.uint8)
    s[:bottom] = 1
    s[ny - top:] = 1
    yb = bottom - 1
    wall = dict(type=0, px=0.0, py=yb - 0.5, nx=0.0, ny=1.0)
    return s, wall


def inclined(nx: int, ny: int, gamma_deg: float):
    """Solid below the line y = tan(gamma) x (plus the frame rows)."""
    t = math.tan(math.radians(gamma_deg))
    y, x = np.mgrid[0:ny, 0:nx]
    s = _frame(nx, ny)
    s |= (y < t * x).astype(np.uint8)
    c, sn = math.cos(math.radians(gamma_deg)), math.sin(math.radians(gamma_deg))
    # unit normal into the fluid (upper-left side of the line)
    n = (-sn, c)
    wall = dict(type=0, px=-n[0], py=-n[1], nx=n[0], ny=n[1])
    return s, wall


def cylinder(nx: int, ny: int, xs: float, ys: float, Rs: float):
    """Solid disc of radius Rs centred at (xs, ys) (plus the frame rows)."""
    y, x = np.mgrid[0:ny, 0:nx]
    s = _frame(nx, ny)
    s |= (((x - xs) ** 2 + (y - ys) ** 2) < Rs * Rs).astype(np.uint8)
    wall = dict(type=1, px=float(xs), py=float(ys), r=float(Rs) - 1.0)
    return s, wall


# --------------------------------------------------------------------------
# The benchmark workloads
# --------------------------------------------------------------------------

def droplet_on_flat_wall(nx=100, ny=50, R=20.0, theta=60.0, steps=5000, **phys) -> Case:
    """Semicircular droplet of radius R on the bottom wall of a channel
    (100 x 50, R = 20, theta = 60 deg, FP64, 5000 steps by default).
    The droplet centre sits on the effective wall, as in the paper's
    flat-wall case (Sec. 3.1)."""
    s, wall = flat_channel(nx, ny)
    d = [(nx / 2.0, wall["py"], R)]
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case("flat", s, d, wall, theta_deg=theta, steps=steps, **kw)


def droplet_on_incline(nx=400, ny=200, gamma=30.0, R=40.0, theta=90.0, steps=20000,
                       **phys) -> Case:
    """Droplet on a staircase wall y = tan(gamma) x, centred on the line at
    x = nx/2 (Sec. 3.2 layout)."""
    s, wall = inclined(nx, ny, gamma)
    x0 = nx / 2.0
    d = [(x0, math.tan(math.radians(gamma)) * x0, R)]
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case("incline", s, d, wall, theta_deg=theta, steps=steps, **kw)


def droplet_on_cylinder(nx=512, ny=512, Rs=100.0, R=50.0, theta=90.0, steps=20000,
                        **phys) -> Case:
    """Droplet of radius R resting on top of a solid cylinder of radius Rs at
    the domain centre (Sec. 3.3 layout)."""
    xs, ys = nx / 2.0, ny / 2.0
    s, wall = cylinder(nx, ny, xs, ys, Rs)
    d = [(xs, ys + Rs, R)]
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case("cylinder", s, d, wall, theta_deg=theta, steps=steps, **kw)


def many_droplets_flat(nx=4096, ny=2048, n_drops=64, seed=2312, r_lo=30.0, r_hi=60.0,
                       th_lo=30.0, th_hi=150.0, W=4.0, steps=10000) -> Case:
    """Flat bottom wall with ``n_drops`` droplets of radius U[r_lo, r_hi] centred
    on the wall at x ~ U[0, nx) (overlapping droplets merge: the initial field
    is the pointwise maximum). Each droplet draws theta ~ U[th_lo, th_hi]; the
    per-node angle field takes the theta of the droplet whose centre is
    nearest in x (periodic). rho_l / rho_g = 10."""
    rng = np.random.default_rng(seed)
    s, wall = flat_channel(nx, ny)
    drops, thetas = [], []
    for _ in range(n_drops):
        R = float(rng.uniform(r_lo, r_hi))
        x0 = float(rng.uniform(0.0, nx))
        th = float(rng.uniform(th_lo, th_hi))
        drops.append((x0, wall["py"], R))
        thetas.append(th)
    xs = np.array([d[0] for d in drops])
    th_arr = np.array(thetas)
    xcol = np.arange(nx, dtype=np.float64)
    dist = np.abs(xcol[:, None] - xs[None, :])
    dist = np.minimum(dist, nx - dist)
    th_col = th_arr[np.argmin(dist, axis=1)]
    field_ = np.broadcast_to(th_col[None, :], (ny, nx)).astype(np.float32).copy()
    return Case("many_flat", s, drops, wall, theta_deg=90.0, theta_field=field_,
                sigma=0.01, W=W, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1, steps=steps,
                meta=dict(seed=seed, thetas=thetas))


BATCH_SIZES = [(64, 32), (128, 64), (256, 128), (512, 256)]


def batch_instance(rng, nx, ny, wall_type: int, theta: float, steps: int) -> Case:
    """One uneven batched instance: flat, 30 deg incline, or cylinder of radius
    ny/4 at (nx/2, 0.4 ny); droplet radius ny/5 on the wall."""
    R = ny / 5.0
    if wall_type == 0:
        s, wall = flat_channel(nx, ny)
        d = [(nx / 2.0, wall["py"], R)]
    elif wall_type == 1:
        s, wall = inclined(nx, ny, 30.0)
        x0 = nx / 2.0
        d = [(x0, math.tan(math.radians(30.0)) * x0, R)]
    else:
        xs, ys, Rs = nx / 2.0, 0.4 * ny, ny / 4.0
        s, wall = cylinder(nx, ny, xs, ys, Rs)
        d = [(xs, ys + Rs, R)]
    return Case(["flat", "incline", "cylinder"][wall_type], s, d, wall, theta_deg=theta,
                sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1, steps=steps)


def batched_instances(count=256, seed=369, steps=5000):
    """``count`` independent solves with sizes from BATCH_SIZES, a wall type
    chosen uniformly, theta ~ U[30, 150] deg."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx, ny = BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]
        wt = int(rng.integers(3))
        th = float(rng.uniform(30.0, 150.0))
        out.append(batch_instance(rng, nx, ny, wt, th, steps))
    return out


def request_stream(rate=2000.0, duration=60.0, seed=2024, n_max=None):
    """Poisson arrivals at ``rate`` per second for ``duration`` seconds. Each
    request: nx = 16 * round(exp(U[ln 128, ln 1024]) / 16), ny = nx / 2,
    steps ~ U{1000..20000}, wall type and theta as for the batched instances.
    Returns a list of dicts (arrival time in seconds and the case parameters);
    the cases themselves are built on demand with ``batch_instance``."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration or (n_max is not None and len(out) >= n_max):
            break
        nx = int(16 * round(math.exp(rng.uniform(math.log(128), math.log(1024))) / 16))
        ny = nx // 2
        out.append(dict(t=t, nx=nx, ny=ny, wall_type=int(rng.integers(3)),
                        theta=float(rng.uniform(30.0, 150.0)),
                        steps=int(rng.integers(1000, 20001))))
    return out


# --------------------------------------------------------------------------
# Three dimensions: masks are uint8 [nz, ny, nx]; x and y periodic; planes
# 0, 1, nz-2, nz-1 solid. The effective flat wall is z = z_b - 1/2 for a top
# solid plane z_b, as in 2D.
# --------------------------------------------------------------------------

@dataclass
class Case3D:
    name: str
    solid: np.ndarray                      # uint8 [nz, ny, nx]
    droplets: list                         # [(x0, y0, z0, R), ...]
    zw: float                              # effective bottom wall plane z = zw
    theta_deg: float = 90.0
    sigma: float = 0.01
    W: float = 4.0
    M: float = 0.1
    tau_f: float = 0.8
    rho_l: float = 1.0
    rho_g: float = 0.1
    steps: int = 1000
    meta: dict = field(default_factory=dict)
    # effective wall for the sphere fit: type 0 plane through p with unit
    # normal n into the fluid, type 1 solid sphere of centre p, radius r
    wall: dict = field(default_factory=dict)

    @property
    def shape(self):
        return tuple(int(v) for v in self.solid.shape)

    def physical(self) -> dict:
        return dict(sigma=self.sigma, W=self.W, M=self.M, tau_f=self.tau_f,
                    rho_l=self.rho_l, rho_g=self.rho_g)


def box3d(nx: int, ny: int, nz: int, bottom: int = 2, top: int = 2):
    """Solid planes [0, bottom) and [nz-top, nz); returns (solid, zw)."""
    assert bottom >= 2 and top >= 2
    s = np.zeros((nz, ny, nx), np.uint8)
    s[:bottom] = 1
    s[nz - top:] = 1
    return s, bottom - 1 - 0.5


def droplet_on_flat_wall_3d(nx=64, ny=64, nz=40, R=16.0, theta=60.0, steps=5000, **phys) -> Case3D:
    """Hemispherical droplet of radius R centred on the effective bottom wall."""
    s, zw = box3d(nx, ny, nz)
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case3D("flat3d", s, [(nx / 2.0, ny / 2.0, zw, R)], zw, theta_deg=theta, steps=steps,
                  wall=dict(type=0, p=(0.0, 0.0, zw), n=(0.0, 0.0, 1.0)), **kw)


def inclined3d(nx: int, ny: int, nz: int, gamma_deg: float, z0: float = 2.0):
    """Solid below the plane z = tan(gamma) x + z0 (a staircase in x, uniform
    in y) plus the frame planes. Returns (solid, wall): the effective wall is
    the plane moved one lattice spacing into the solid along its normal."""
    t = math.tan(math.radians(gamma_deg))
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    s, _ = box3d(nx, ny, nz)
    s |= (z < t * x + z0).astype(np.uint8)
    c, sn = math.cos(math.radians(gamma_deg)), math.sin(math.radians(gamma_deg))
    n = (-sn, 0.0, c)
    wall = dict(type=0, p=(-n[0], 0.0, z0 - n[2]), n=n)
    return s, wall


def droplet_on_incline_3d(nx=40, ny=20, nz=40, gamma=30.0, R=7.0, theta=90.0, steps=1000, **phys) -> Case3D:
    """Droplet centred on the staircase plane z = tan(gamma) x + 2 at x = nx/2."""
    s, wall = inclined3d(nx, ny, nz, gamma)
    x0 = nx / 2.0
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case3D("incline3d", s, [(x0, ny / 2.0, math.tan(math.radians(gamma)) * x0 + 2.0, R)], 1.5,
                  theta_deg=theta, steps=steps, wall=wall, meta=dict(gamma=gamma), **kw)


def droplet_on_sphere_3d(n=32, Rs=6.0, R=7.0, theta=90.0, steps=1000, **phys) -> Case3D:
    """Droplet of radius R on top of a solid sphere of radius Rs at the domain
    centre (a curved wall with every link configuration of D3Q19)."""
    s, zw = box3d(n, n, n)
    c = n / 2.0
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    s |= (((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) < Rs * Rs).astype(np.uint8)
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    kw.update(phys)
    return Case3D("sphere3d", s, [(c, c, c + Rs, R)], zw, theta_deg=theta, steps=steps,
                  meta=dict(Rs=Rs), wall=dict(type=1, p=(c, c, c), r=Rs - 1.0), **kw)


def many_droplets_3d(nx=512, ny=512, nz=128, n_drops=64, seed=2312, r_lo=12.0, r_hi=24.0,
                     theta=60.0, steps=1000) -> Case3D:
    """Flat bottom wall with ``n_drops`` hemispherical droplets of radius
    U[r_lo, r_hi] centred on the wall at (x, y) ~ U[0, nx) x U[0, ny)."""
    rng = np.random.default_rng(seed)
    s, zw = box3d(nx, ny, nz)
    d = [(float(rng.uniform(0, nx)), float(rng.uniform(0, ny)), zw, float(rng.uniform(r_lo, r_hi)))
         for _ in range(n_drops)]
    return Case3D("many_flat3d", s, d, zw, theta_deg=theta, steps=steps, meta=dict(seed=seed),
                  wall=dict(type=0, p=(0.0, 0.0, zw), n=(0.0, 0.0, 1.0)))
