"""Pins of the oracle's geometry pre-processing (Sec. 2.2.2, Sec. 2.2.3)."""
import numpy as np

import oracle
from tests.oracle_fixtures import read_geometry


def make(solid, **kw):
    return oracle.Oracle(solid, **kw)


def test_hand_classified_block():
    mask, cls_expected, links = read_geometry("geometry_block.txt")
    o = make(mask)
    g = o.geometry()
    assert np.array_equal(g["cls"], cls_expected)
    zeta = ((cls_expected == oracle.FLUID) | (cls_expected == oracle.BOUNDARY)).astype(np.uint8)
    assert np.array_equal(g["zeta"], zeta)
    assert np.array_equal(g["eps"], (cls_expected == oracle.FLUID).astype(float))
    cx, cy, _, _ = oracle.lattice()
    x, y = links["node"]
    un, db = int(g["unknown"][y, x]), int(g["doubly"][y, x])
    got_un = {(int(cx[i]), int(cy[i])) for i in range(1, 9) if un >> i & 1}
    got_db = {(int(cx[i]), int(cy[i])) for i in range(1, 9) if db >> i & 1}
    assert got_un == links["unknown"]
    assert got_db == links["doubly"]


def test_flat_wall_effective_surface_area():
    # Sec. 2.2.3: for a flat boundary a_v equals 1/dx. With a_v = |grad eps|
    # the unit is spread over two layers: the boundary row and the first fluid
    # row carry 1/2 each, every other node 0.
    nx, ny = 16, 12
    s = np.zeros((ny, nx), np.uint8)
    s[:3] = 1
    s[-2:] = 1
    g = make(s).geometry()
    av = g["av"]
    assert np.allclose(av[2], 0.5, atol=1e-15) and np.allclose(av[3], 0.5, atol=1e-15)
    assert np.allclose(av[-2], 0.5, atol=1e-15) and np.allclose(av[-3], 0.5, atol=1e-15)
    assert np.allclose(av.sum(axis=0), 2.0, atol=1e-14)   # 1/dx per wall, two walls
    assert np.count_nonzero(av) == 4 * nx


def test_flat_wall_links():
    # On a flat floor the boundary row misses exactly the three populations
    # arriving from below (c_y = +1); none is doubly unknown.
    nx, ny = 8, 8
    s = np.zeros((ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    g = make(s).geometry()
    cx, cy, _, _ = oracle.lattice()
    from_below = sum(1 << i for i in range(1, 9) if cy[i] == 1)
    from_above = sum(1 << i for i in range(1, 9) if cy[i] == -1)
    assert np.all(g["unknown"][1] == from_below)
    assert np.all(g["unknown"][ny - 2] == from_above)
    assert np.all(g["unknown"][2:ny - 2] == 0)
    assert np.all(g["doubly"] == 0)
    assert np.all(g["cls"][0] == oracle.GHOST) and np.all(g["cls"][1] == oracle.BOUNDARY)


def test_thin_plate_has_zero_av():
    # A one-node-thick plate has fluid on both sides: the isotropic gradient of
    # eps cancels there (the two layers of opposite normal overlap).
    nx, ny = 10, 12
    s = np.zeros((ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    s[6] = 1
    g = make(s).geometry()
    assert np.all(g["cls"][6] == oracle.BOUNDARY)
    assert np.allclose(g["av"][6], 0.0)


def test_wrap_in_x():
    # x is periodic: a solid column at x = 0 has boundary neighbours at x = nx-1
    nx, ny = 9, 8
    s = np.zeros((ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    s[:, 0] = 1
    g = make(s).geometry()
    assert g["cls"][4, 0] == oracle.BOUNDARY
    cx, cy, _, _ = oracle.lattice()
    i_east = [i for i in range(9) if cx[i] == 1 and cy[i] == 0][0]
    assert g["unknown"][4, 1] >> i_east & 1 == 0     # (0,4) is a zeta=1 boundary node
    assert g["av"][4, nx - 1] > 0 and g["av"][4, 1] > 0
