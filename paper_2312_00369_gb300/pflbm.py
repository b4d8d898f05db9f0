"""ctypes binding of libpflbm.so (include/pflbm.h) with the same names.

Argument marshalling only: every step of the computation runs in the CUDA
library. PyTorch supplies device memory (its caching allocator, through the
library's allocator callbacks) and streams. If the library is missing or
cannot be loaded, every call raises: there is no fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import re
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PFLBM_LIBRARY selects another build of the same library (the index-checked
# libpflbm_bounds.so beside it); the default is libpflbm.so
LIB_PATH = os.environ.get("PFLBM_LIBRARY") or os.path.join(HERE, "libpflbm.so")
BOUNDS_LIB_PATH = os.path.join(HERE, "libpflbm_bounds.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pflbm.h")

OK, EINVAL, ENOMEM, EBADMASK, ENUMERIC, ETIMEOUT, ECUDA = 0, -1, -2, -3, -4, -5, -6
FP64, FP32, BF16, FP16 = 0, 1, 2, 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16}
FLUID, BOUNDARY, GHOST, INTERIOR = 0, 1, 2, 3

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class PflbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pflbm error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("solid_mask", ctypes.POINTER(ctypes.c_uint8)),
                ("theta_deg", ctypes.c_double),
                ("theta_field_deg", ctypes.POINTER(ctypes.c_float)),
                ("sigma", ctypes.c_double), ("W", ctypes.c_double), ("M", ctypes.c_double),
                ("tau_f", ctypes.c_double), ("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
                ("tau_g", ctypes.c_double), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("alloc", _ALLOC), ("free", _FREE),
                ("alloc_ctx", ctypes.c_void_p), ("nu_l", ctypes.c_double), ("nu_g", ctypes.c_double),
                ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("dgdt_mode", ctypes.c_int),
                ("chi_case", ctypes.c_int), ("step_kernel", ctypes.c_int), ("step_chunk", ctypes.c_int)]


class Params3D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("solid_mask", ctypes.POINTER(ctypes.c_uint8)),
                ("theta_deg", ctypes.c_double), ("sigma", ctypes.c_double), ("W", ctypes.c_double),
                ("M", ctypes.c_double), ("tau_f", ctypes.c_double), ("rho_l", ctypes.c_double),
                ("rho_g", ctypes.c_double), ("tau_g", ctypes.c_double), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("step_path", ctypes.c_int),
                ("fused_zc", ctypes.c_int), ("dgdt_mode", ctypes.c_int),
                ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", ctypes.c_void_p)]


class Wall3D(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int)] + [(k, ctypes.c_double) for k in
                                            ("px", "py", "pz", "nx", "ny", "nz", "r", "x_lo", "x_hi", "y_lo",
                                             "y_hi", "exclude")]


class Schedule(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("tiles_per_item", ctypes.c_int),
                ("order", ctypes.c_int), ("use_graph", ctypes.c_int), ("kernel", ctypes.c_int),
                ("n_classes", ctypes.c_int), ("class_max_nodes", ctypes.c_int64 * 8),
                ("class_shape", ctypes.c_int * 8), ("class_tiles", ctypes.c_int * 8)]


# step kernels (pflbm_params_t.step_kernel)
STEP_KERNELS = {"default": 0, "global": 1, "staged32x8": 2, "staged64x4": 3, "pair": 4}


class Wall(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("px", ctypes.c_double), ("py", ctypes.c_double),
                ("nx", ctypes.c_double), ("ny", ctypes.c_double), ("r", ctypes.c_double),
                ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
                ("exclude", ctypes.c_double)]


_lib = None
_H = ctypes.c_void_p
# live handles, closed before the interpreter (and PyTorch, whose allocator
# the handles call back into) shuts down
_LIVE_BATCHES = weakref.WeakSet()
_LIVE_SOLVERS = weakref.WeakSet()


@atexit.register
def _close_all():
    for b in list(_LIVE_BATCHES):
        try:
            b.close()
        except Exception:
            pass
    for s in list(_LIVE_SOLVERS):
        try:
            s.close()
        except Exception:
            pass
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u16p = ctypes.POINTER(ctypes.c_uint16)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "pflbm_params_default": (None, [ctypes.POINTER(Params)]),
    "pflbm_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.c_int, ctypes.c_int, _u8p]
                     + [ctypes.c_double] * 7),
    "pflbm_create_ex": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(Params)]),
    "pflbm_destroy": (None, [_H]),
    "pflbm_set_theta_field": (ctypes.c_int, [_H, _fp]),
    "pflbm_set_step_kernel": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_int]),
    "pflbm_debug_bounds": (ctypes.c_int, [_ip, ctypes.POINTER(ctypes.c_uint)]),
    "pflbm_get_step_kernel": (ctypes.c_int, [_H]),
    "pflbm_init_droplet": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "pflbm_init_phi": (ctypes.c_int, [_H, _dp]),
    "pflbm_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "pflbm_get": (ctypes.c_int, [_H, _dp, _dp, _dp]),
    "pflbm_get_device": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pflbm_get_f32": (ctypes.c_int, [_H, _fp, _fp, _fp]),
    "pflbm_mass": (ctypes.c_int, [_H, _dp]),
    "pflbm_phi_mass_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "pflbm_contact_angle": (ctypes.c_int, [_H, ctypes.POINTER(Wall), _dp, _dp, _ip]),
    "pflbm_geometry": (ctypes.c_int, [_H, _u8p, _u16p, _u16p, _dp]),
    "pflbm_lattice": (None, [_ip, _ip]),
    "pflbm_check": (ctypes.c_int, [_H]),
    "pflbm_steps": (ctypes.c_int64, [_H]),
    "pflbm_status": (ctypes.c_int, [_H]),
    "pflbm_footprint_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pflbm_save": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "pflbm_load": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "pflbm_last_error": (ctypes.c_char_p, []),
    "pflbm_schedule_default": (None, [ctypes.POINTER(Schedule)]),
    "pflbm_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_H),
                                          ctypes.c_int, ctypes.POINTER(Schedule)]),
    "pflbm_batch_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(_H), ctypes.c_int]),
    "pflbm_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pflbm_batch_info": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip, ctypes.POINTER(ctypes.c_int64)]),
    "pflbm_batch_kernel": (ctypes.c_int, [ctypes.c_void_p]),
    "pflbm_batch_destroy": (None, [ctypes.c_void_p]),
    "pflbm3d_params_default": (None, [ctypes.POINTER(Params3D)]),
    "pflbm3d_create": (ctypes.c_int, [ctypes.POINTER(_H), ctypes.POINTER(Params3D)]),
    "pflbm3d_destroy": (None, [_H]),
    "pflbm3d_init_droplet": (ctypes.c_int, [_H] + [ctypes.c_double] * 4),
    "pflbm3d_init_phi": (ctypes.c_int, [_H, _dp]),
    "pflbm3d_step": (ctypes.c_int, [_H, ctypes.c_int64]),
    "pflbm3d_get": (ctypes.c_int, [_H, _dp, _dp, _dp]),
    "pflbm3d_get_f32": (ctypes.c_int, [_H, _fp, _fp, _fp]),
    "pflbm3d_mass": (ctypes.c_int, [_H, _dp]),
    "pflbm3d_geometry": (ctypes.c_int, [_H, _u8p, _dp]),
    "pflbm3d_check": (ctypes.c_int, [_H]),
    "pflbm3d_contact_angle": (ctypes.c_int, [_H, ctypes.POINTER(Wall3D), _dp, _dp, _ip]),
    "pflbm3d_steps": (ctypes.c_int64, [_H]),
    "pflbm3d_save": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "pflbm3d_load": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
}


def declared_functions(header: str = HEADER):
    """Names of the functions include/pflbm.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pflbm(?:3d)?_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libpflbm.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2312_00369_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise PflbmError(rc, lib().pflbm_last_error().decode())
    return rc


def _p(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def pflbm_lattice():
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    lib().pflbm_lattice(cx, cy)
    return np.array(cx[:]), np.array(cy[:])


def debug_bounds():
    """(enabled, violations) of the index-checked build (see pflbm.h)."""
    e, v = ctypes.c_int(), ctypes.c_uint()
    _check(lib().pflbm_debug_bounds(ctypes.byref(e), ctypes.byref(v)))
    return bool(e.value), int(v.value)


def pflbm_footprint_bytes(nx, ny, precision="fp32"):
    return int(lib().pflbm_footprint_bytes(nx, ny, PRECISIONS.get(precision, precision)))


def pflbm_phi_mass_noalloc(d_phi, d_zeta, nx, ny, d_out, stream=None):
    """Allocation-free FP64 sum of a device phi field (raw device pointers as
    ints; d_zeta may be None). Asynchronous on ``stream`` (a cudaStream_t
    handle as int, or None for the default stream)."""
    _check(lib().pflbm_phi_mass_noalloc(ctypes.c_void_p(d_phi),
                                        None if d_zeta is None else ctypes.c_void_p(d_zeta),
                                        int(nx), int(ny), ctypes.c_void_p(d_out),
                                        None if stream is None else ctypes.c_void_p(stream)))


# One pair of allocator callbacks for the whole process (ctypes thunks must
# outlive every handle that may call them); ctx selects (device, stream).
_ALLOC_CTX = {}


def _torch_alloc(nbytes, ctx):
    try:
        import torch
        dev, stream = _ALLOC_CTX[int(ctx or 0)]
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream))
    except Exception:
        return None


def _torch_free(ptr, nbytes, ctx):
    if ptr:
        try:
            import torch
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


_TORCH_ALLOC = _ALLOC(_torch_alloc)
_TORCH_FREE = _FREE(_torch_free)


def _alloc_ctx(device, stream):
    key = len(_ALLOC_CTX) + 1
    for k, v in _ALLOC_CTX.items():
        if v == (device, stream):
            return k
    _ALLOC_CTX[key] = (device, stream)
    return key


class Solver:
    """One lattice (``pflbm_t``) owned from Python.

    ``solid``: uint8 [ny, nx] mask (1 = solid). ``precision``: "fp64",
    "fp32", "bf16" or "fp16". ``stream``: a ``torch.cuda.Stream`` (default:
    the current stream of ``device``). Memory comes from PyTorch's caching
    allocator unless ``torch_memory=False``.
    """

    def __init__(self, solid, theta_deg=90.0, sigma=0.01, W=4.0, M=0.1, tau_f=0.8,
                 rho_l=1.0, rho_g=0.1, tau_g=0.0, theta_field=None, precision="fp32",
                 device=None, stream=None, torch_memory=True, nu_l=0.0, nu_g=0.0, gx=0.0, gy=0.0,
                 dgdt_mode=0, chi_case=2, step_kernel="default", step_chunk=0):
        import torch
        L = lib()
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.ny, self.nx = solid.shape
        self.precision = precision
        dev = torch.cuda.current_device() if device is None else int(device)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        self.device = dev
        p = Params()
        L.pflbm_params_default(ctypes.byref(p))
        p.nx, p.ny = self.nx, self.ny
        p.solid_mask = _p(solid, _u8p)
        p.theta_deg = float(theta_deg)
        self._theta_field = None
        if theta_field is not None:
            self._theta_field = np.ascontiguousarray(theta_field, dtype=np.float32)
            p.theta_field_deg = _p(self._theta_field, _fp)
        p.sigma, p.W, p.M, p.tau_f = sigma, W, M, tau_f
        p.rho_l, p.rho_g, p.tau_g = rho_l, rho_g, tau_g
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.nu_l, p.nu_g, p.gx, p.gy = float(nu_l), float(nu_g), float(gx), float(gy)
        p.dgdt_mode = int(dgdt_mode)
        p.chi_case = int(chi_case)
        p.step_kernel = STEP_KERNELS.get(step_kernel, step_kernel) if isinstance(step_kernel, str) \
            else int(step_kernel)
        p.step_chunk = int(step_chunk)
        p.device = dev
        p.stream = ctypes.c_void_p(stream.cuda_stream)
        if torch_memory:
            p.alloc = _TORCH_ALLOC
            p.free = _TORCH_FREE
            p.alloc_ctx = ctypes.c_void_p(_alloc_ctx(dev, stream.cuda_stream))
        h = _H()
        _check(L.pflbm_create_ex(ctypes.byref(h), ctypes.byref(p)))
        self._h = h
        self.W = W
        _LIVE_SOLVERS.add(self)

    # -- lifetime ------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pflbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- the API ---------------------------------------------------------------
    def init_droplet(self, x0, y0, R):
        _check(lib().pflbm_init_droplet(self._h, float(x0), float(y0), float(R)))

    def init_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        assert phi.shape == (self.ny, self.nx)
        _check(lib().pflbm_init_phi(self._h, _p(phi)))

    def set_step_kernel(self, step_kernel, step_chunk=0):
        """Switch the step kernel ("default", "global", "staged32x8",
        "staged64x4", "pair" or 0..4); results are the same bit for bit."""
        k = STEP_KERNELS.get(step_kernel, step_kernel) if isinstance(step_kernel, str) else int(step_kernel)
        _check(lib().pflbm_set_step_kernel(self._h, int(k), int(step_chunk)))

    @property
    def step_kernel(self):
        return {v: k for k, v in STEP_KERNELS.items()}[lib().pflbm_get_step_kernel(self._h)]

    def set_theta_field(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().pflbm_set_theta_field(self._h, _p(theta, _fp)))

    def step(self, n=1):
        _check(lib().pflbm_step(self._h, int(n)))

    def get(self, out=None):
        """(phi [ny, nx], u [ny, nx, 2], p [ny, nx]) as float64 host arrays.
        ``out``: three C-contiguous float64 arrays of those shapes to fill
        (for example views of pinned memory, which copy faster)."""
        if out is None:
            out = (np.empty((self.ny, self.nx)), np.empty((self.ny, self.nx, 2)), np.empty((self.ny, self.nx)))
        phi, u, p = out
        for a, shp in zip(out, ((self.ny, self.nx), (self.ny, self.nx, 2), (self.ny, self.nx))):
            if a.shape != shp or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError(f"output array must be C-contiguous float64 {shp}")
        _check(lib().pflbm_get(self._h, _p(phi), _p(u), _p(p)))
        return phi, u, p

    def get_f32(self, out=None):
        """As get(), rounded to float32 on the device (half the bytes)."""
        shapes = ((self.ny, self.nx), (self.ny, self.nx, 2), (self.ny, self.nx))
        if out is None:
            out = tuple(np.empty(sh, np.float32) for sh in shapes)
        for a, sh in zip(out, shapes):
            if a.shape != sh or a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError(f"output array must be C-contiguous float32 {sh}")
        phi, u, p = out
        _check(lib().pflbm_get_f32(self._h, _p(phi, _fp), _p(u, _fp), _p(p, _fp)))
        return phi, u, p

    def get_device(self, phi=None, u=None, p=None):
        """Fill caller-owned torch float64 CUDA tensors (any may be None)."""
        ptr = (lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
        _check(lib().pflbm_get_device(self._h, ptr(phi), ptr(u), ptr(p)))

    def mass(self):
        out = ctypes.c_double()
        _check(lib().pflbm_mass(self._h, ctypes.byref(out)))
        return out.value

    def contact_angle(self, wall: dict, exclude=None):
        w = Wall(type=int(wall.get("type", 0)), px=wall.get("px", 0.0), py=wall.get("py", 0.0),
                 nx=wall.get("nx", 0.0), ny=wall.get("ny", 1.0), r=wall.get("r", 0.0),
                 x_lo=wall.get("x_lo", -1e300), x_hi=wall.get("x_hi", 1e300),
                 exclude=wall.get("exclude", 1.5 * self.W if exclude is None else exclude))
        th = ctypes.c_double()
        circ = (ctypes.c_double * 3)()
        n = ctypes.c_int()
        _check(lib().pflbm_contact_angle(self._h, ctypes.byref(w), ctypes.byref(th), circ,
                                         ctypes.byref(n)))
        return th.value, np.array(circ[:]), n.value

    def geometry(self):
        shp = (self.ny, self.nx)
        cls = np.empty(shp, np.uint8)
        un = np.empty(shp, np.uint16)
        db = np.empty(shp, np.uint16)
        av = np.empty(shp)
        _check(lib().pflbm_geometry(self._h, _p(cls, _u8p), _p(un, _u16p), _p(db, _u16p), _p(av)))
        return dict(cls=cls, unknown=un, doubly=db, av=av)

    def check(self):
        _check(lib().pflbm_check(self._h))

    def status(self, wait=False):
        """Status code (0 or ENUMERIC) without raising; wait=True synchronises
        first, otherwise the last value copied back is returned."""
        if wait:
            return int(lib().pflbm_check(self._h))
        return int(lib().pflbm_status(self._h))

    @property
    def steps(self):
        return int(lib().pflbm_steps(self._h))

    def save(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(lib().pflbm_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().pflbm_save(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().pflbm_load(self._h, buf, len(blob)))


def schedule(ctas_per_sm=0, tiles_per_item=1, order=0, use_graph=1, kernel=0, classes=()):
    """A ``pflbm_schedule_t``. ``classes``: up to 8 (max_nodes, shape,
    tiles_per_item) entries of the staged kernel, by lattice size."""
    s = Schedule()
    lib().pflbm_schedule_default(ctypes.byref(s))
    s.ctas_per_sm, s.tiles_per_item, s.order, s.use_graph = (int(ctas_per_sm), int(tiles_per_item),
                                                             int(order), int(use_graph))
    s.kernel = int(kernel)
    classes = list(classes)[:8]
    s.n_classes = len(classes)
    for k, (mx, shape, tiles) in enumerate(classes):
        s.class_max_nodes[k], s.class_shape[k], s.class_tiles[k] = int(mx), int(shape), int(tiles)
    return s


class Batch:
    """Several Solvers advanced together (``pflbm_batch_t``). The solvers must
    share precision, device and stream; they stay alive while the batch
    uses them."""

    def __init__(self, solvers, sched=None):
        self._solvers = list(solvers)
        arr = (_H * len(self._solvers))(*[s.handle for s in self._solvers])
        self._arr = arr
        b = ctypes.c_void_p()
        sc = sched if sched is not None else schedule()
        _check(lib().pflbm_batch_create(ctypes.byref(b), arr, len(self._solvers), ctypes.byref(sc)))
        self._b = b
        self.sched = sc
        _LIVE_BATCHES.add(self)

    def set(self, solvers):
        self._solvers = list(solvers)
        self._arr = (_H * len(self._solvers))(*[s.handle for s in self._solvers])
        _check(lib().pflbm_batch_set(self._b, self._arr, len(self._solvers)))

    def step(self, n=1):
        _check(lib().pflbm_batch_step(self._b, int(n)))

    @property
    def kernel(self):
        """1: global-load kernel, 2: staged kernel, 3: two-node kernel."""
        return lib().pflbm_batch_kernel(self._b)

    def info(self):
        nw, grid, nodes = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().pflbm_batch_info(self._b, ctypes.byref(nw), ctypes.byref(grid),
                                      ctypes.byref(nodes)))
        return dict(n_work=nw.value, grid=grid.value, nodes=nodes.value)

    def close(self):
        b = getattr(self, "_b", None)
        if b:
            lib().pflbm_batch_destroy(b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3D:
    """One three-dimensional lattice (``pflbm3d_t``): f on D3Q19, g on D3Q7.

    ``solid``: uint8 [nz, ny, nx] mask (1 = solid; planes z = 0, 1, nz-2,
    nz-1 solid). ``precision``: "fp64" or "fp32". ``step_path``: "auto",
    "fused" (one launch per step) or "three_pass". Work runs on ``stream``
    (default: the current stream). Memory comes from PyTorch's caching
    allocator unless ``torch_memory=False`` (then cudaMalloc).
    """

    def __init__(self, solid, theta_deg=90.0, sigma=0.01, W=4.0, M=0.1, tau_f=0.8,
                 rho_l=1.0, rho_g=0.1, tau_g=0.0, precision="fp32", device=None, stream=None,
                 step_path="auto", fused_zc=0, dgdt_mode=0, torch_memory=True):
        import torch
        L = lib()
        solid = np.ascontiguousarray(solid, dtype=np.uint8)
        self.nz, self.ny, self.nx = solid.shape
        self.precision = precision
        dev = torch.cuda.current_device() if device is None else int(device)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        p = Params3D()
        L.pflbm3d_params_default(ctypes.byref(p))
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.solid_mask = _p(solid, _u8p)
        p.theta_deg, p.sigma, p.W, p.M, p.tau_f = float(theta_deg), sigma, W, M, tau_f
        p.rho_l, p.rho_g, p.tau_g = rho_l, rho_g, tau_g
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.device = dev
        p.stream = ctypes.c_void_p(stream.cuda_stream)
        p.step_path = {"auto": 0, "fused": 1, "three_pass": 2}[step_path]
        p.fused_zc = int(fused_zc)
        p.dgdt_mode = int(dgdt_mode)
        if torch_memory:
            p.alloc = _TORCH_ALLOC
            p.free = _TORCH_FREE
            p.alloc_ctx = ctypes.c_void_p(_alloc_ctx(dev, stream.cuda_stream))
        h = _H()
        _check(L.pflbm3d_create(ctypes.byref(h), ctypes.byref(p)))
        self._h = h
        self.W = W
        _LIVE_SOLVERS.add(self)

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pflbm3d_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_droplet(self, x0, y0, z0, R):
        _check(lib().pflbm3d_init_droplet(self._h, float(x0), float(y0), float(z0), float(R)))

    def init_phi(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        assert phi.shape == (self.nz, self.ny, self.nx)
        _check(lib().pflbm3d_init_phi(self._h, _p(phi)))

    def step(self, n=1):
        _check(lib().pflbm3d_step(self._h, int(n)))

    def get(self, out=None):
        """(phi, u [..., 3], p) as float64 host arrays [nz, ny, nx]; ``out``
        as for Solver.get."""
        shp = (self.nz, self.ny, self.nx)
        if out is None:
            out = (np.empty(shp), np.empty(shp + (3,)), np.empty(shp))
        phi, u, p = out
        for a, sh in zip(out, (shp, shp + (3,), shp)):
            if a.shape != sh or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError(f"output array must be C-contiguous float64 {sh}")
        _check(lib().pflbm3d_get(self._h, _p(phi), _p(u), _p(p)))
        return phi, u, p

    def get_f32(self, out=None):
        """As get(), rounded to float32 on the device (half the bytes)."""
        shp = (self.nz, self.ny, self.nx)
        shapes = (shp, shp + (3,), shp)
        if out is None:
            out = tuple(np.empty(sh, np.float32) for sh in shapes)
        for a, sh in zip(out, shapes):
            if a.shape != sh or a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError(f"output array must be C-contiguous float32 {sh}")
        phi, u, p = out
        _check(lib().pflbm3d_get_f32(self._h, _p(phi, _fp), _p(u, _fp), _p(p, _fp)))
        return phi, u, p

    def mass(self):
        m = ctypes.c_double()
        _check(lib().pflbm3d_mass(self._h, ctypes.byref(m)))
        return m.value

    def geometry(self):
        shp = (self.nz, self.ny, self.nx)
        cls, av = np.empty(shp, np.uint8), np.empty(shp)
        _check(lib().pflbm3d_geometry(self._h, _p(cls, _u8p), _p(av)))
        return {"cls": cls, "av": av}

    def check(self):
        _check(lib().pflbm3d_check(self._h))

    @property
    def steps(self):
        return lib().pflbm3d_steps(self._h)

    def save(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().pflbm3d_save(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().pflbm3d_save(self._h, buf, ctypes.byref(n)))
        return buf.raw[:n.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().pflbm3d_load(self._h, buf, len(blob)))

    def contact_angle(self, wall: dict, exclude=None):
        """``wall``: dict(type=0, p=(x, y, z), n=(nx, ny, nz)) for a plane or
        dict(type=1, p=centre, r=radius) for a solid sphere; optional x_lo,
        x_hi, y_lo, y_hi window and ``exclude`` (default 1.5 W). Returns
        (theta_deg, [cx, cy, cz, R], n_points)."""
        p = wall.get("p", (0.0, 0.0, 0.0))
        n = wall.get("n", (0.0, 0.0, 1.0))
        w = Wall3D(type=int(wall.get("type", 0)), px=p[0], py=p[1], pz=p[2], nx=n[0], ny=n[1], nz=n[2],
                   r=float(wall.get("r", 0.0)), x_lo=wall.get("x_lo", -1e300), x_hi=wall.get("x_hi", 1e300),
                   y_lo=wall.get("y_lo", -1e300), y_hi=wall.get("y_hi", 1e300),
                   exclude=wall.get("exclude", 1.5 * self.W if exclude is None else exclude))
        th = ctypes.c_double()
        sph = (ctypes.c_double * 4)()
        npts = ctypes.c_int()
        _check(lib().pflbm3d_contact_angle(self._h, ctypes.byref(w), ctypes.byref(th), sph, ctypes.byref(npts)))
        return th.value, np.array(sph[:]), npts.value
