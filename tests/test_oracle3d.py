"""Pins of the 3D oracle (D3Q19 hydrodynamics, D3Q7 phase lattice)."""
import math
import os

import numpy as np
import pytest

import oracle

rng = np.random.default_rng(11)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def mom(v, c):
    return v.sum(), np.einsum("i,ia->a", v, c), np.einsum("i,ia,ib->ab", v, c, c)


def test_lattices():
    c19, w19, c7, w7 = oracle.lattices3d()
    rows = np.array([[int(t) for t in ln.split()] for ln in open(os.path.join(GOLDEN, "d3q7_paper_matrix.txt"))
                     if ln.strip() and not ln.startswith("#")])
    assert np.array_equal(c7, rows[:, 1:4]) and np.allclose(w7, rows[:, 4] / rows[:, 5])
    d = np.eye(3)
    c = c19.astype(float)
    assert abs(w19.sum() - 1) < 1e-15 and abs(w7.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w19, c, c), d / 3, atol=1e-16)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w19, c, c, c, c), iso, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w7, c7.astype(float), c7.astype(float)), d / 4, atol=1e-16)
    # D3Q19 = rest, 6 axes, 12 edges, each with its opposite
    norms = sorted((c19 ** 2).sum(1).tolist())
    assert norms == [0] + [1] * 6 + [2] * 12
    assert {tuple(v) for v in c19} == {tuple(-v) for v in c19}


@pytest.mark.parametrize("trial", range(10))
def test_equilibria_and_sources(trial):
    c19, w19, c7, w7 = oracle.lattices3d()
    c, cg = c19.astype(float), c7.astype(float)
    p, rho = rng.normal() * 1e-3, rng.uniform(0.1, 5)
    u = rng.normal(size=3) * 0.05
    m0, m1, m2 = mom(oracle.feq3(p, rho, u), c)
    assert abs(m0) < 1e-14 and np.allclose(m1, rho * u, atol=1e-15)
    assert np.allclose(m2, p * np.eye(3) + rho * np.outer(u, u), atol=1e-15)
    phi, mu, al = rng.uniform(0, 1), rng.normal() * 1e-3, rng.uniform(0.2, 2)
    m0, m1, m2 = mom(oracle.geq3(phi, mu, al), cg)
    assert abs(m0 - phi) < 1e-15 and np.allclose(m1, 0, atol=1e-18)
    assert np.allclose(m2, al * mu * 0.25 * np.eye(3), atol=1e-18)        # D3Q7: c_s^2 = 1/4
    tau = rng.uniform(0.55, 1.5)
    dr, F = rng.normal(size=3) * 0.1, rng.normal(size=3) * 1e-3
    P = 1 - 1 / (2 * tau)
    m0, m1, m2 = mom(oracle.force3(tau, u, dr, F), c)
    assert abs(m0 - P * u @ dr) < 1e-16 and np.allclose(m1, P * F, atol=1e-17)
    assert np.allclose(m2, P / 3 * ((u @ dr) * np.eye(3) + np.outer(u, dr) + np.outer(dr, u)), atol=1e-16)
    s = rng.normal() * 1e-3
    m0, m1, _ = mom(oracle.source3(s), cg)
    assert abs(m0 + s) < 1e-18 and np.allclose(m1, 0, atol=1e-19)
    # pressure/velocity round trip with the half-force shift
    f = oracle.feq3(p, rho, u) - 0.5 * 3 * w19 * (c @ F)
    uu, pp = oracle.velocity_pressure3(f, rho, np.zeros(3), F)
    assert np.allclose(uu, u, atol=1e-15) and abs(pp - p) < 1e-16


def test_stencils_exact_on_polynomials():
    a = rng.normal(size=20)
    x0 = rng.normal(size=3)

    def q(x, y, z, cubic=True):
        v = (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * x + a[5] * y * y + a[6] * z * z
             + a[7] * x * y + a[8] * x * z + a[9] * y * z)
        if cubic:
            v += a[10] * x ** 3 + a[11] * y ** 3 + a[12] * z ** 3 + a[13] * x * y * z + a[14] * x * x * y
        return v

    grid = lambda cubic: np.array([[[q(x0[0] + dx, x0[1] + dy, x0[2] + dz, cubic) for dx in (-1, 0, 1)]
                                    for dy in (-1, 0, 1)] for dz in (-1, 0, 1)])
    _, lap = oracle.stencil3(grid(True))
    x, y, z = x0
    exact = (2 * a[4] + 2 * a[5] + 2 * a[6] + 6 * a[10] * x + 6 * a[11] * y + 6 * a[12] * z + 2 * a[14] * y)
    assert abs(lap - exact) < 1e-11
    g, _ = oracle.stencil3(grid(False))
    exg = [a[1] + 2 * a[4] * x + a[7] * y + a[8] * z, a[2] + 2 * a[5] * y + a[7] * x + a[9] * z,
           a[3] + 2 * a[6] * z + a[8] * x + a[9] * y]
    assert np.allclose(g, exg, atol=1e-11)


def box(nx, ny, nz):
    s = np.zeros((nz, ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    return s


def test_flat_wall_classes_and_av():
    o = oracle.Oracle3D(box(6, 5, 10))
    g = o.geometry()
    assert np.all(g["cls"][0] == 2) and np.all(g["cls"][1] == 1) and np.all(g["cls"][2:-2] == 0)
    # Sec. 2.2.3: a_v = 1/dx on a flat wall, spread over two layers of 1/2
    assert np.allclose(g["av"][1], 0.5) and np.allclose(g["av"][2], 0.5) and np.allclose(g["av"][3], 0)
    assert np.allclose(g["av"].sum(0), 2.0)


def test_budget_and_phase_swap_symmetry():
    s = box(12, 10, 12)
    o = oracle.Oracle3D(s, theta_deg=70.0)
    o.init_droplet(6, 5, 1.5, 5.0)
    for _ in range(20):
        o.step(1)
        m0, src, lost, bb = o.budget()
        assert abs(o.mass() - (m0 + src - lost + bb)) < 1e-12 * m0
    kw = dict(sigma=0.01, W=4.0, M=0.1, tau_f=0.8, rho_l=1.0, rho_g=1.0)
    a = oracle.Oracle3D(s, theta_deg=55.0, **kw)
    b = oracle.Oracle3D(s, theta_deg=125.0, **kw)
    z, y, x = np.mgrid[0:12, 0:10, 0:12]
    phi0 = 0.5 + 0.5 * np.tanh(2 * (5 - np.sqrt((x - 6) ** 2 + (y - 5) ** 2 + (z - 1.5) ** 2)) / 4)
    a.init_phi(phi0)
    b.init_phi(1 - phi0)
    a.step(40)
    b.step(40)
    pa, ua, qa = a.get()
    pb, ub, qb = b.get()
    zeta = s == 0
    zeta[1] = True
    zeta[-2] = True
    assert np.max(np.abs(pa[zeta] + pb[zeta] - 1)) < 1e-12
    assert np.max(np.abs(ua - ub)) < 1e-13 and np.max(np.abs(qa - qb)) < 1e-13


@pytest.mark.slow
def test_laplace_law_3d():
    # sphere: p_in - p_out = 2 sigma / R (the deviation, 8.4 % at R = 8 with
    # W = 4, shrinks with R: 18 % at R = 6)
    n, sigma, R = 24, 0.01, 8.0
    o = oracle.Oracle3D(np.zeros((n, n, n), np.uint8), sigma=sigma, tau_f=1.0, wrap_z=True)
    o.init_droplet(12, 12, 12, R)
    o.step(1200)
    phi, u, p = o.get()
    Re = (3 * phi.sum() / (4 * math.pi)) ** (1 / 3)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    r = np.sqrt((x - 12) ** 2 + (y - 12) ** 2 + (z - 12) ** 2)
    dp = p[r < R - 3].mean() - p[r > R + 4].mean()
    assert abs(dp / (2 * sigma / Re) - 1) < 0.12


def _cap_field(shape, c, R, W=4.0):
    z, y, x = np.mgrid[0:shape[0], 0:shape[1], 0:shape[2]]
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    return 0.5 + 0.5 * np.tanh(2 * (R - r) / W)


@pytest.mark.parametrize("theta", [40.0, 90.0, 130.0])
def test_contact_angle_fit_exact_caps(theta):
    # tanh spheres placed where a cap of angle theta meets (a) a plane tilted
    # by 20 deg and (b) a solid sphere: the fit returns theta (closed-form
    # geometry: centre at -R cos(theta) n from the plane; at distance
    # sqrt(R^2 + r^2 - 2 R r cos(theta)) from the sphere's centre)
    shape, R = (48, 64, 64), 14.0
    cls = np.zeros(shape, np.uint8)
    n = np.array([-math.sin(math.radians(20)), 0.0, math.cos(math.radians(20))])
    p0 = np.array([32.0, 32.0, 16.0])
    c = p0 - R * math.cos(math.radians(theta)) * n
    th, sph, npts = oracle.contact_angle3(_cap_field(shape, c, R), cls, dict(type=0, p=p0, n=n, exclude=1.0))
    assert npts > 200 and abs(th - theta) < 0.1 and abs(sph[3] - R) < 0.02
    rs, cs = 10.0, np.array([32.0, 32.0, 14.0])
    D = math.sqrt(R * R + rs * rs - 2 * R * rs * math.cos(math.radians(theta)))
    c2 = cs + np.array([0.0, 0.0, D])
    th, sph, npts = oracle.contact_angle3(_cap_field(shape, c2, R), cls, dict(type=1, p=cs, r=rs, exclude=1.0))
    assert npts > 1000 and abs(th - theta) < 0.1
    # the flat-wall form is the plane form with n = +z
    field = _cap_field(shape, (30.0, 31.0, 10.0 - R * math.cos(math.radians(theta))), R)
    th1, _, n1 = oracle.contact_angle_flat3(field, cls, 10.0, 1.0)
    th2, _, n2 = oracle.contact_angle3(field, cls, dict(type=0, p=(0, 0, 10.0), n=(0, 0, 1), exclude=1.0))
    assert n1 == n2 and th1 == th2 and abs(th1 - theta) < 0.1


def test_dgdt_omitted_changes_only_the_source():
    # with the (1/2) dG/dt term omitted the first step is unchanged (the
    # backward difference starts from a zero derivative) and later steps differ
    s = box(12, 10, 12)
    a = oracle.Oracle3D(s, theta_deg=70.0)
    b = oracle.Oracle3D(s, theta_deg=70.0)
    b.set_dgdt(1)
    for o in (a, b):
        o.init_droplet(6, 5, 1.5, 5.0)
        o.step(1)
    assert np.array_equal(a.get()[0], b.get()[0])
    a.step(5)
    b.step(5)
    assert np.max(np.abs(a.get()[0] - b.get()[0])) > 0
    m0, src, lost, bb = b.budget()
    assert abs(b.mass() - (m0 + src - lost + bb)) < 1e-12 * m0
