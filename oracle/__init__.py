"""ctypes wrapper of the FP64 CPU oracle (``pflbm_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
and reference legs of ``bench.py`` import this package. It shares no code with
the CUDA library and imports nothing from it.
"""
import ctypes
import os

import numpy as np

from . import build_oracle

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u16p = ctypes.POINTER(ctypes.c_uint16)
_ip = ctypes.POINTER(ctypes.c_int)

FLUID, BOUNDARY, GHOST, INTERIOR = 0, 1, 2, 3


class Wall(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("px", ctypes.c_double), ("py", ctypes.c_double),
                ("nx_", ctypes.c_double), ("ny_", ctypes.c_double), ("r", ctypes.c_double),
                ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
                ("exclude", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.or_lattice.argtypes = [_ip, _ip, _dp, _ip]
        L.or_feq.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.or_geq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.or_force.argtypes = [ctypes.c_double] * 7 + [_dp]
        L.or_source.argtypes = [ctypes.c_double, _dp]
        L.or_velocity_pressure.argtypes = [_dp] + [ctypes.c_double] * 5 + [_dp] * 3
        L.or_stencil.argtypes = [_dp, _dp, _dp, _dp]
        L.or_create.restype = ctypes.c_void_p
        L.or_create.argtypes = ([ctypes.c_int] * 3 + [_u8p, ctypes.c_double, _dp]
                                + [ctypes.c_double] * 7)
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_set_viscosity.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.or_set_body_force.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.or_set_dgdt.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_set_chi_case.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_params.argtypes = [ctypes.c_void_p, _dp]
        L.or_geometry.argtypes = [ctypes.c_void_p, _u8p, _u8p, _dp, _dp, _u16p, _u16p]
        L.or_init_droplet.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 3
        L.or_init_phi.argtypes = [ctypes.c_void_p, _dp]
        L.or_droplet_phi.restype = ctypes.c_double
        L.or_droplet_phi.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int]
        L.or_droplet_phi_points.argtypes = ([_dp, _dp, ctypes.c_long] + [ctypes.c_double] * 4
                                            + [ctypes.c_int, ctypes.c_int, _dp])
        L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.or_get.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.or_mass.restype = ctypes.c_double
        L.or_mass.argtypes = [ctypes.c_void_p]
        L.or_budget.argtypes = [ctypes.c_void_p, _dp]
        L.or_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.or_set_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.or_steps.restype = ctypes.c_long
        L.or_steps.argtypes = [ctypes.c_void_p]
        L.or_contact_angle.restype = ctypes.c_int
        L.or_contact_angle.argtypes = [_dp, _u8p, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(Wall), _dp, _dp]
        L.or_circle_fit.restype = ctypes.c_int
        L.or_circle_fit.argtypes = [_dp, _dp, ctypes.c_int, _dp]
        _lib = L
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def lattice():
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9)
    opp = np.zeros(9, np.int32)
    lib().or_lattice(_p(cx, _ip), _p(cy, _ip), _p(w), _p(opp, _ip))
    return cx, cy, w, opp


def feq(p, rho, ux, uy):
    out = np.zeros(9)
    lib().or_feq(p, rho, ux, uy, _p(out))
    return out


def geq(phi, mu, alpha):
    out = np.zeros(9)
    lib().or_geq(phi, mu, alpha, _p(out))
    return out


def force(tau_f, ux, uy, drx, dry, Fx, Fy):
    out = np.zeros(9)
    lib().or_force(tau_f, ux, uy, drx, dry, Fx, Fy, _p(out))
    return out


def source(s):
    out = np.zeros(9)
    lib().or_source(s, _p(out))
    return out


def velocity_pressure(f, rho, drx, dry, Fx, Fy):
    f = np.ascontiguousarray(f, dtype=np.float64)
    ux, uy, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_velocity_pressure(_p(f), rho, drx, dry, Fx, Fy,
                               ctypes.byref(ux), ctypes.byref(uy), ctypes.byref(p))
    return ux.value, uy.value, p.value


def stencil(v3x3):
    v = np.ascontiguousarray(v3x3, dtype=np.float64)
    gx, gy, lap = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_stencil(_p(v), ctypes.byref(gx), ctypes.byref(gy), ctypes.byref(lap))
    return gx.value, gy.value, lap.value


def droplet_phi(x, y, x0, y0, R, W, nx_period=0, out=None):
    """Eq. initialphi at points (x, y) (arrays of one shape), x-periodic with
    nx_period; with ``out`` given, the pointwise maximum with ``out``."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.shape == y.shape
    combine = out is not None
    if out is None:
        out = np.empty(x.shape)
    assert out.flags["C_CONTIGUOUS"] and out.dtype == np.float64
    lib().or_droplet_phi_points(_p(x), _p(y), x.size, x0, y0, R, W, int(nx_period),
                                int(combine), _p(out))
    return out


def circle_fit(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    c = np.zeros(3)
    rc = lib().or_circle_fit(_p(x), _p(y), len(x), _p(c))
    if rc:
        raise ValueError("circle fit failed")
    return c


def contact_angle(phi, cls, wall: dict):
    """Fit the phi = 1/2 contour and return (theta_deg, circle, n_points)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    ny, nx = phi.shape
    w = Wall(type=wall.get("type", 0), px=wall.get("px", 0.0), py=wall.get("py", 0.0),
             nx_=wall.get("nx", 0.0), ny_=wall.get("ny", 1.0), r=wall.get("r", 0.0),
             x_lo=wall.get("x_lo", -1e300), x_hi=wall.get("x_hi", 1e300),
             exclude=wall.get("exclude", 0.0))
    th = ctypes.c_double()
    c = np.zeros(3)
    n = lib().or_contact_angle(_p(phi), _p(cls, _u8p), nx, ny, ctypes.byref(w),
                               ctypes.byref(th), _p(c))
    return th.value, c, n


class Oracle:
    """Whole-domain FP64 solver (see pflbm_oracle.h)."""

    def __init__(self, solid, theta_deg=90.0, sigma=0.01, W=4.0, M=0.1, tau_f=0.8,
                 rho_l=1.0, rho_g=0.1, tau_g=0.0, theta_field=None, wrap_y=False):
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.ny, self.nx = solid.shape
        self.W = W
        tf = None
        if theta_field is not None:
            tf = np.ascontiguousarray(theta_field, dtype=np.float64)
            assert tf.shape == solid.shape
        self._h = lib().or_create(self.nx, self.ny, int(wrap_y), _p(solid, _u8p),
                                  float(theta_deg), _p(tf), sigma, W, M, tau_f,
                                  rho_l, rho_g, tau_g)
        if not self._h:
            raise ValueError("or_create rejected the arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    @property
    def params(self):
        out = np.zeros(4)
        lib().or_params(self._h, _p(out))
        return dict(beta=out[0], kappa=out[1], tau_g=out[2], alpha=out[3])

    def geometry(self):
        shp = (self.ny, self.nx)
        cls = np.zeros(shp, np.uint8)
        zeta = np.zeros(shp, np.uint8)
        eps = np.zeros(shp)
        av = np.zeros(shp)
        un = np.zeros(shp, np.uint16)
        db = np.zeros(shp, np.uint16)
        lib().or_geometry(self._h, _p(cls, _u8p), _p(zeta, _u8p), _p(eps), _p(av),
                          _p(un, _u16p), _p(db, _u16p))
        return dict(cls=cls, zeta=zeta, eps=eps, av=av, unknown=un, doubly=db)

    def set_viscosity(self, nu_l, nu_g):
        lib().or_set_viscosity(self._h, nu_l, nu_g)

    def set_body_force(self, gx, gy):
        lib().or_set_body_force(self._h, gx, gy)

    def set_dgdt(self, mode):
        lib().or_set_dgdt(self._h, int(mode))

    def set_chi_case(self, chi_case):
        lib().or_set_chi_case(self._h, int(chi_case))

    def init_droplet(self, x0, y0, R):
        lib().or_init_droplet(self._h, x0, y0, R)

    def init_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        lib().or_init_phi(self._h, _p(phi))

    def step(self, n=1):
        lib().or_step(self._h, int(n))

    def get(self):
        shp = (self.ny, self.nx)
        phi = np.zeros(shp)
        u = np.zeros(shp + (2,))
        p = np.zeros(shp)
        lib().or_get(self._h, _p(phi), _p(u), _p(p))
        return phi, u, p

    def mass(self):
        return lib().or_mass(self._h)

    def budget(self):
        out = np.zeros(4)
        lib().or_budget(self._h, _p(out))
        return out

    def state(self):
        N = self.nx * self.ny
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((9, self.ny, self.nx))
        sp = np.zeros((self.ny, self.nx))
        lib().or_state(self._h, _p(f), _p(g), _p(sp))
        return f, g, sp

    def set_state(self, f, g):
        """Overwrite the post-streaming f, g (arrays [9, ny, nx], paper order);
        the u.grad(phi) history and the first-step flag are kept."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == g.shape == (9, self.ny, self.nx)
        lib().or_set_state(self._h, _p(f), _p(g))

    @property
    def steps(self):
        return lib().or_steps(self._h)


# ------------------------------------------------------------------ 3D --
_3d_ready = False


def _lib3d():
    global _3d_ready
    L = lib()
    if not _3d_ready:
        vp = ctypes.c_void_p
        L.or3_lattices.argtypes = [_ip, _dp, _ip, _dp]
        L.or3_feq.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.or3_geq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.or3_force.argtypes = [ctypes.c_double, _dp, _dp, _dp, _dp]
        L.or3_source.argtypes = [ctypes.c_double, _dp]
        L.or3_velocity_pressure.argtypes = [_dp, ctypes.c_double, _dp, _dp, _dp, _dp]
        L.or3_stencil.argtypes = [_dp, _dp, _dp]
        L.or3_create.restype = vp
        L.or3_create.argtypes = [ctypes.c_int] * 4 + [_u8p] + [ctypes.c_double] * 8
        L.or3_destroy.argtypes = [vp]
        L.or3_params.argtypes = [vp, _dp]
        L.or3_geometry.argtypes = [vp, _u8p, _dp]
        L.or3_init_droplet.argtypes = [vp] + [ctypes.c_double] * 4
        L.or3_init_phi.argtypes = [vp, _dp]
        L.or3_step.argtypes = [vp, ctypes.c_long]
        L.or3_get.argtypes = [vp, _dp, _dp, _dp]
        L.or3_mass.restype = ctypes.c_double
        L.or3_mass.argtypes = [vp]
        L.or3_budget.argtypes = [vp, _dp]
        L.or3_set_dgdt.restype = None
        L.or3_set_dgdt.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or3_contact_angle.restype = ctypes.c_int
        L.or3_contact_angle.argtypes = [_dp, _u8p] + [ctypes.c_int] * 3 + [ctypes.POINTER(Wall3), _dp, _dp]
        L.or3_contact_angle_flat.restype = ctypes.c_int
        L.or3_contact_angle_flat.argtypes = [_dp, _u8p] + [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_dp, _dp]
        _3d_ready = True
    return L


def lattices3d():
    c19 = np.zeros((19, 3), np.int32)
    w19 = np.zeros(19)
    c7 = np.zeros((7, 3), np.int32)
    w7 = np.zeros(7)
    _lib3d().or3_lattices(_p(c19, _ip), _p(w19), _p(c7, _ip), _p(w7))
    return c19, w19, c7, w7


def feq3(p, rho, u):
    out = np.zeros(19)
    _lib3d().or3_feq(p, rho, _p(np.ascontiguousarray(u, dtype=np.float64)), _p(out))
    return out


def geq3(phi, mu, alpha):
    out = np.zeros(7)
    _lib3d().or3_geq(phi, mu, alpha, _p(out))
    return out


def force3(tau_f, u, drho, F):
    out = np.zeros(19)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (u, drho, F)]
    _lib3d().or3_force(tau_f, _p(a[0]), _p(a[1]), _p(a[2]), _p(out))
    return out


def source3(s):
    out = np.zeros(7)
    _lib3d().or3_source(s, _p(out))
    return out


def velocity_pressure3(f, rho, drho, F):
    f = np.ascontiguousarray(f, dtype=np.float64)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (drho, F)]
    u = np.zeros(3)
    p = ctypes.c_double()
    _lib3d().or3_velocity_pressure(_p(f), rho, _p(a[0]), _p(a[1]), _p(u), ctypes.byref(p))
    return u, p.value


def stencil3(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    g = np.zeros(3)
    lap = ctypes.c_double()
    _lib3d().or3_stencil(_p(v), _p(g), ctypes.byref(lap))
    return g, lap.value


class Wall3(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("p", ctypes.c_double * 3), ("n", ctypes.c_double * 3),
                ("r", ctypes.c_double), ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
                ("y_lo", ctypes.c_double), ("y_hi", ctypes.c_double), ("exclude", ctypes.c_double)]


def wall3(wall: dict) -> Wall3:
    w = Wall3()
    w.type = int(wall.get("type", 0))
    for i, v in enumerate(wall.get("p", (0.0, 0.0, 0.0))):
        w.p[i] = float(v)
    for i, v in enumerate(wall.get("n", (0.0, 0.0, 1.0))):
        w.n[i] = float(v)
    w.r = float(wall.get("r", 0.0))
    w.x_lo, w.x_hi = float(wall.get("x_lo", -1e300)), float(wall.get("x_hi", 1e300))
    w.y_lo, w.y_hi = float(wall.get("y_lo", -1e300)), float(wall.get("y_hi", 1e300))
    w.exclude = float(wall.get("exclude", 0.0))
    return w


def contact_angle3(phi, cls, wall: dict):
    """Sphere fit of the phi = 1/2 crossings and the contact angle against a
    plane or a solid sphere (see or3_contact_angle). Returns (theta_deg,
    [cx, cy, cz, R], n_points)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    nz, ny, nx = phi.shape
    th = ctypes.c_double()
    sph = np.zeros(4)
    w = wall3(wall)
    n = _lib3d().or3_contact_angle(_p(phi), _p(cls, _u8p), nx, ny, nz, ctypes.byref(w), ctypes.byref(th), _p(sph))
    return th.value, sph, n


def contact_angle_flat3(phi, cls, zw, exclude):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    nz, ny, nx = phi.shape
    th = ctypes.c_double()
    sph = np.zeros(4)
    n = _lib3d().or3_contact_angle_flat(_p(phi), _p(cls, _u8p), nx, ny, nz, zw, exclude,
                                        ctypes.byref(th), _p(sph))
    return th.value, sph, n


class Oracle3D:
    """Whole-domain FP64 3D solver (see pflbm_oracle3d.h); arrays are [nz, ny, nx]."""

    def __init__(self, solid, theta_deg=90.0, sigma=0.01, W=4.0, M=0.1, tau_f=0.8,
                 rho_l=1.0, rho_g=0.1, tau_g=0.0, wrap_z=False):
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.nz, self.ny, self.nx = solid.shape
        L = _lib3d()
        self._h = L.or3_create(self.nx, self.ny, self.nz, int(wrap_z), _p(solid, _u8p), float(theta_deg),
                               sigma, W, M, tau_f, rho_l, rho_g, tau_g)
        if not self._h:
            raise ValueError("or3_create rejected the arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib3d().or3_destroy(h)
            self._h = None

    @property
    def params(self):
        out = np.zeros(4)
        _lib3d().or3_params(self._h, _p(out))
        return dict(beta=out[0], kappa=out[1], tau_g=out[2], alpha=out[3])

    def geometry(self):
        shp = (self.nz, self.ny, self.nx)
        cls = np.zeros(shp, np.uint8)
        av = np.zeros(shp)
        _lib3d().or3_geometry(self._h, _p(cls, _u8p), _p(av))
        return dict(cls=cls, av=av)

    def init_droplet(self, x0, y0, z0, R):
        _lib3d().or3_init_droplet(self._h, x0, y0, z0, R)

    def init_phi(self, phi):
        _lib3d().or3_init_phi(self._h, _p(np.ascontiguousarray(phi, dtype=np.float64)))

    def set_dgdt(self, mode):
        _lib3d().or3_set_dgdt(self._h, int(mode))

    def step(self, n=1):
        _lib3d().or3_step(self._h, int(n))

    def get(self):
        shp = (self.nz, self.ny, self.nx)
        phi = np.zeros(shp)
        u = np.zeros(shp + (3,))
        p = np.zeros(shp)
        _lib3d().or3_get(self._h, _p(phi), _p(u), _p(p))
        return phi, u, p

    def mass(self):
        return _lib3d().or3_mass(self._h)

    def budget(self):
        out = np.zeros(4)
        _lib3d().or3_budget(self._h, _p(out))
        return out
