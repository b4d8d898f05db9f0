"""The C-ABI library builds for sm_103a and exports every declared symbol
(no GPU needed: nothing is called that touches the device)."""
import ctypes

from paper_2312_00369_gb300 import build as libbuild
from paper_2312_00369_gb300 import pflbm


def test_library_builds_and_exports_header():
    path = libbuild.build()
    L = ctypes.CDLL(path)
    names = pflbm.declared_functions()
    assert "pflbm_create" in names and "pflbm_step" in names and "pflbm_get" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding declares a signature for every header function
    assert set(names) <= set(pflbm._SIGS)


def test_host_only_entry_points():
    L = pflbm.lib()
    cx, cy = pflbm.pflbm_lattice()
    assert cx[0] == 0 and cy[0] == 0
    vecs = set(zip(cx.tolist(), cy.tolist()))
    assert vecs == {(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    # footprint grows with the lattice and the storage precision
    f64 = pflbm.pflbm_footprint_bytes(128, 64, "fp64")
    f32 = pflbm.pflbm_footprint_bytes(128, 64, "fp32")
    assert f64 > f32 > 0
    assert pflbm.pflbm_footprint_bytes(256, 64, "fp32") > f32
    # argument checks that fail before any CUDA call
    h = pflbm._H()
    P = pflbm.Params()
    L.pflbm_params_default(ctypes.byref(P))
    assert L.pflbm_create_ex(ctypes.byref(h), ctypes.byref(P)) == pflbm.EINVAL
    assert L.pflbm_step(None, 1) == pflbm.EINVAL
    assert b"NULL handle" in L.pflbm_last_error()


def test_host_only_checks_3d():
    L = pflbm.lib()
    h = pflbm._H()
    P = pflbm.Params3D()
    L.pflbm3d_params_default(ctypes.byref(P))
    assert P.precision == pflbm.FP32 and P.tau_f == 0.8 and P.device == -1
    # nx = 0 and no mask: refused before any CUDA call
    assert L.pflbm3d_create(ctypes.byref(h), ctypes.byref(P)) == pflbm.EINVAL
    assert L.pflbm3d_step(None, 1) == pflbm.EINVAL
    assert L.pflbm3d_mass(None, None) == pflbm.EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no CPU fallback: without libpflbm.so every entry point raises
    monkeypatch.setattr(pflbm, "_lib", None)
    monkeypatch.setattr(pflbm, "LIB_PATH", str(tmp_path / "libpflbm.so"))
    import pytest
    with pytest.raises(RuntimeError, match="missing"):
        pflbm.lib()
    with pytest.raises(RuntimeError):
        pflbm.pflbm_footprint_bytes(64, 32)


def test_sizes_beyond_the_launch_grid_are_refused():
    # refused by the argument checks, before any CUDA call
    import numpy as np
    L = pflbm.lib()
    ny = 524288 + 8
    mask = np.ones((ny, 3), np.uint8)
    P = pflbm.Params()
    L.pflbm_params_default(ctypes.byref(P))
    P.nx, P.ny = 3, ny
    P.solid_mask = mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    h = pflbm._H()
    assert L.pflbm_create_ex(ctypes.byref(h), ctypes.byref(P)) == pflbm.EINVAL
    assert b"ny too large" in L.pflbm_last_error()
    nz = 65536 + 2
    mask3 = np.ones((nz, 3, 3), np.uint8)
    P3 = pflbm.Params3D()
    L.pflbm3d_params_default(ctypes.byref(P3))
    P3.nx, P3.ny, P3.nz = 3, 3, nz
    P3.solid_mask = mask3.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    assert L.pflbm3d_create(ctypes.byref(h), ctypes.byref(P3)) == pflbm.EINVAL
    assert b"65535" in L.pflbm_last_error()
