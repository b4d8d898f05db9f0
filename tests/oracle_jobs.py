"""Oracle reference runs used by the GPU parity tests.

Each job builds a case from the seeded input generators, runs the FP64 oracle
and returns plain numpy arrays. The jobs run in a ``spawn`` process pool so
that the slow CPU oracle overlaps with the GPU tests (the pool is started
with ``spawn``, never forked from a process that already touched CUDA).
"""
import math

import numpy as np

import oracle
from paper_2312_00369_gb300 import workloads as wl


def case_by_name(name):
    if name == "flat60":
        return wl.droplet_on_flat_wall(theta=60.0)
    if name == "flat60_short":
        return wl.droplet_on_flat_wall(theta=60.0, steps=600)
    if name == "incline30":
        return wl.droplet_on_incline(theta=60.0, steps=800)
    if name == "incline45_ragged":
        return wl.droplet_on_incline(nx=130, ny=91, gamma=45.0, R=18.0, theta=120.0, steps=400)
    if name == "cylinder":
        return wl.droplet_on_cylinder(theta=120.0, steps=200)
    if name == "crop":
        return wl.many_droplets_flat(nx=512, ny=256, n_drops=8, seed=2312, steps=400)
    if name == "flat_visc_force":
        c = wl.droplet_on_flat_wall(theta=75.0, steps=800)
        c.meta = dict(nu_l=0.3, nu_g=0.05, gx=2e-6, gy=-1e-6)
        return c
    if name == "incline_nodgdt":
        c = wl.droplet_on_incline(nx=130, ny=91, gamma=45.0, R=18.0, theta=110.0, steps=500)
        c.meta = dict(dgdt=1)
        return c
    if name == "incline_w8":
        return wl.droplet_on_incline(nx=130, ny=91, gamma=14.036243467926479, R=24.0, theta=120.0,
                                     W=8.0, steps=300)
    if name in ("flat_chi1", "flat_chi3"):
        c = wl.droplet_on_flat_wall(theta=55.0 if name == "flat_chi1" else 125.0, steps=700)
        c.meta = dict(chi_case=int(name[-1]))
        return c
    if name == "odd_wide":            # odd width (the last node pair ends in the padding), fluid tiles inside
        return wl.many_droplets_flat(nx=201, ny=96, n_drops=3, seed=5, r_lo=14.0, r_hi=20.0, steps=300)
    if name == "tiny":
        s = np.ones((6, 3), np.uint8)
        s[2:4] = 0
        return wl.Case("tiny", s, [(1.0, 2.0, 1.5)], dict(type=0, px=0, py=0.5, nx=0, ny=1),
                       theta_deg=70.0, steps=50)
    if name == "block":
        from tests.oracle_fixtures import read_geometry
        mask, _, _ = read_geometry("geometry_block.txt")
        big = np.tile(mask, (1, 3))           # 36 x 10, x-periodic copies
        return wl.Case("block", big, [(17.0, 6.0, 4.0)], dict(type=0, px=0, py=0.5, nx=0, ny=1),
                       theta_deg=45.0, steps=120)
    raise KeyError(name)


def apply_options(o, case):
    m = case.meta or {}
    if m.get("nu_l") and m.get("nu_g"):
        o.set_viscosity(m["nu_l"], m["nu_g"])
    if m.get("gx") or m.get("gy"):
        o.set_body_force(m.get("gx", 0.0), m.get("gy", 0.0))
    if m.get("dgdt"):
        o.set_dgdt(m["dgdt"])
    if m.get("chi_case"):
        o.set_chi_case(m["chi_case"])


def solver_options(case):
    """The same options as keyword arguments of the GPU Solver."""
    m = case.meta or {}
    out = {}
    for k in ("nu_l", "nu_g", "gx", "gy"):
        if k in m:
            out[k] = m[k]
    if "dgdt" in m:
        out["dgdt_mode"] = m["dgdt"]
    if "chi_case" in m:
        out["chi_case"] = m["chi_case"]
    return out


def run_case(name, steps=None, with_angle=False):
    case = case_by_name(name)
    steps = case.steps if steps is None else steps
    o = oracle.Oracle(case.solid, theta_deg=case.theta_deg, theta_field=case.theta_field,
                      **case.physical())
    apply_options(o, case)
    for d in case.droplets:
        o.init_droplet(*d)
    o.step(steps)
    phi, u, p = o.get()
    out = dict(phi=phi, u=u, p=p, mass=o.mass(), steps=steps)
    if with_angle:
        w = dict(case.wall, exclude=1.5 * case.W)
        th, circ, n = oracle.contact_angle(phi, o.geometry()["cls"], w)
        out.update(theta=th, circle=circ, npts=n)
    return out


def geometry_of(name_or_mask):
    solid = case_by_name(name_or_mask).solid if isinstance(name_or_mask, str) else name_or_mask
    o = oracle.Oracle(solid)
    return o.geometry()


def window_run(case_name_kwargs, x_centre, half, steps):
    """Run the oracle on a full-height window [x_centre - half, x_centre + half]
    of a large case, built from the same generator, for `steps` steps. Nodes
    farther than 2 * steps + 1 from the window edges do not feel the wrong
    periodic wrap of the window, so the centre column equals the full run."""
    case = wl.many_droplets_flat(**case_name_kwargs)
    nx_full = case.nx
    xs = (np.arange(x_centre - half, x_centre + half + 1)) % nx_full
    solid = case.solid[:, xs]
    tf = case.theta_field[:, xs] if case.theta_field is not None else None
    o = oracle.Oracle(solid, theta_deg=case.theta_deg, theta_field=tf, **case.physical())
    ny = case.ny
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, len(xs)))
    x = np.broadcast_to(xs[None, :].astype(float), y.shape)
    phi0 = None
    for (x0, y0, R) in case.droplets:
        # Eq. initialphi with the period of the full lattice, max over droplets
        phi0 = oracle.droplet_phi(x, y, x0, y0, R, case.W, nx_full, out=phi0)
    o.init_phi(phi0)
    o.step(steps)
    phi, u, p = o.get()
    return dict(phi=phi[:, half], u=u[:, half], p=p[:, half])


# ---- three dimensions ------------------------------------------------------

def case3d_by_name(name):
    if name == "flat3d":          # ragged in x (40 = 32 + 8) and in y (20 = 8 + 8 + 4)
        s, zw = wl.box3d(40, 20, 20)
        return wl.Case3D("flat3d", s, [(20.0, 10.0, zw, 7.0)], zw, theta_deg=60.0, steps=300,
                         wall=dict(type=0, p=(0.0, 0.0, zw), n=(0.0, 0.0, 1.0), exclude=1.0))
    if name == "flat3d_two":      # two overlapping droplets (pointwise maximum), theta > 90
        s, zw = wl.box3d(40, 20, 20)
        return wl.Case3D("flat3d_two", s, [(14.0, 10.0, zw, 6.0), (25.0, 9.0, zw, 5.0)], zw,
                         theta_deg=120.0, steps=200)
    if name == "sphere3d":
        return wl.droplet_on_sphere_3d(n=32, Rs=6.0, R=7.0, theta=75.0, steps=200)
    if name == "incline3d":       # 30 deg staircase plane, theta > 90
        return wl.droplet_on_incline_3d(nx=40, ny=20, nz=40, gamma=30.0, R=7.0, theta=110.0, steps=250)
    if name == "flat3d_nodgdt":   # the (1/2) dG/dt term omitted
        s, zw = wl.box3d(40, 20, 20)
        return wl.Case3D("flat3d_nodgdt", s, [(20.0, 10.0, zw, 7.0)], zw, theta_deg=50.0, steps=300,
                         meta=dict(dgdt=1), wall=dict(type=0, p=(0.0, 0.0, zw), n=(0.0, 0.0, 1.0)))
    if name == "tiny3d":          # smaller than one tile and its halo in x and y
        s, zw = wl.box3d(3, 4, 9)
        return wl.Case3D("tiny3d", s, [(1.0, 2.0, zw, 3.0)], zw, theta_deg=50.0, steps=60)
    raise KeyError(name)


def run3d_case(name, steps=None):
    c = case3d_by_name(name)
    o = oracle.Oracle3D(c.solid, theta_deg=c.theta_deg, **c.physical())
    o.set_dgdt(c.meta.get("dgdt", 0))
    for d in c.droplets:
        o.init_droplet(*d)
    m0 = o.mass()
    o.step(c.steps if steps is None else steps)
    phi, u, p = o.get()
    g = o.geometry()
    out = dict(phi=phi, u=u, p=p, mass0=m0, mass=o.mass(), cls=g["cls"], av=g["av"])
    if c.wall:
        th, sph, n = oracle.contact_angle3(phi, g["cls"], dict(dict(exclude=1.5 * c.W), **c.wall))
        out.update(theta=th, sphere=sph, npts=n)
    return out


MAX3D = dict(nx=512, ny=512, nz=315)     # 26 * nz * ny * pitch = 2146959360 < 2^31


def max3d_case():
    """The largest accepted 3D box with a droplet hanging from the top wall at
    the far corner (the highest indices) and one on the bottom wall."""
    s, zw = wl.box3d(MAX3D["nx"], MAX3D["ny"], MAX3D["nz"])
    top = MAX3D["nz"] - 1.5
    return wl.Case3D("max3d", s, [(500.0, 500.0, top, 14.0), (60.0, 60.0, zw, 14.0)], zw, theta_deg=70.0,
                     steps=8)


def window3d_run(full_kwargs, xc, yc, half, steps):
    """Run the 3D oracle on a full-height window [xc - half, xc + half] x
    [yc - half, yc + half] of a large many-droplet box, built from the same
    generator, for `steps` steps. The initial field is Eq. initialphi with
    the periods of the full box (pointwise maximum over droplets). Nodes
    farther than 2 * steps + 1 from the window edges do not feel the wrong
    periodic wrap of the window, so the centre column equals the full run."""
    case = max3d_case() if full_kwargs == "max3d" else wl.many_droplets_3d(**full_kwargs)
    nz, ny_full, nx_full = case.shape
    xs = np.arange(xc - half, xc + half + 1) % nx_full
    ys = np.arange(yc - half, yc + half + 1) % ny_full
    solid = np.ascontiguousarray(case.solid[:, ys][:, :, xs])
    z, yy, xx = np.meshgrid(np.arange(nz, dtype=float), ys.astype(float), xs.astype(float), indexing="ij")
    phi0 = np.zeros(solid.shape)
    for (x0, y0, z0, R) in case.droplets:
        dx = np.abs(xx - x0) % nx_full
        dx = np.where(dx > 0.5 * nx_full, nx_full - dx, dx)
        dy = np.abs(yy - y0) % ny_full
        dy = np.where(dy > 0.5 * ny_full, ny_full - dy, dy)
        r = np.sqrt(dx * dx + dy * dy + (z - z0) ** 2)
        phi0 = np.maximum(phi0, 0.5 + 0.5 * np.tanh(2.0 * (R - r) / case.W))
    o = oracle.Oracle3D(solid, theta_deg=case.theta_deg, **case.physical())
    o.init_phi(phi0)
    o.step(steps)
    phi, u, p = o.get()
    return dict(phi=phi[:, half, half], u=u[:, half, half], p=p[:, half, half])


# ---- the largest 2D lattice the library accepts ------------------------------

MAX2D = dict(nx=16384, ny=7280)           # 18 * ny * pitch = 2146959360 < 2^31


def max2d_case():
    """Flat channel of the largest accepted size with a droplet hanging from
    the top wall at the far corner (the highest indices) and one on the
    bottom wall."""
    nx, ny = MAX2D["nx"], MAX2D["ny"]
    s, wall = wl.flat_channel(nx, ny)
    drops = [(16300.0, ny - 1.5, 20.0), (700.0, 1.5, 20.0)]
    return wl.Case("max2d", s, drops, wall, theta_deg=70.0, steps=6)


def max2d_window_run(x_centre, half, steps):
    """Oracle on the full-height window [x_centre - half, x_centre + half] of
    max2d_case() (the window wraps at its own edges; the centre column is
    farther than 2 * steps + 1 from them)."""
    case = max2d_case()
    nx, ny = case.nx, case.ny
    xs = np.arange(x_centre - half, x_centre + half + 1) % nx
    solid = np.ascontiguousarray(case.solid[:, xs])
    o = oracle.Oracle(solid, theta_deg=case.theta_deg, **case.physical())
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, len(xs)))
    x = np.broadcast_to(xs[None, :].astype(float), y.shape)
    phi0 = None
    for (x0, y0, R) in case.droplets:
        phi0 = oracle.droplet_phi(x, y, x0, y0, R, case.W, nx, out=phi0)
    o.init_phi(phi0)
    o.step(steps)
    phi, u, p = o.get()
    return dict(phi=phi[:, half], u=u[:, half], p=p[:, half])


def run_instance(nx, ny, wall_type, theta, steps, dgdt=0):
    """Oracle run of one batched / served instance (workloads.batch_instance):
    the fitted contact angle (the same wall and exclusion band as the
    library's fit), phi and the mass after ``steps``."""
    c = wl.batch_instance(None, nx, ny, wall_type, theta, steps)
    o = oracle.Oracle(c.solid, theta_deg=c.theta_deg, **c.physical())
    if dgdt:
        o.set_dgdt(dgdt)
    for d in c.droplets:
        o.init_droplet(*d)
    o.step(steps)
    phi, u, _ = o.get()
    th, circ, n = oracle.contact_angle(phi, o.geometry()["cls"], dict(c.wall, exclude=1.5 * c.W))
    return dict(theta=th, npts=n, phi=phi, mass=o.mass(), umax=float(np.abs(u).max()))

