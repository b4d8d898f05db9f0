"""Pins of the oracle's single-node pieces against identities the paper fixes.

Every expected value below is a closed form (a moment of the lattice or of an
equilibrium), not a retyped copy of the oracle's formula; a dropped term, a
wrong sign or a transposed operand in the oracle changes at least one moment.
"""
import numpy as np
import pytest

import oracle
from tests.oracle_fixtures import read_lattice

CS2 = 1.0 / 3.0
rng = np.random.default_rng(7)


def moments(v, cx, cy):
    m0 = v.sum()
    m1 = np.array([(cx * v).sum(), (cy * v).sum()])
    m2 = np.array([[(cx * cx * v).sum(), (cx * cy * v).sum()],
                   [(cy * cx * v).sum(), (cy * cy * v).sum()]])
    return m0, m1, m2


def test_lattice_matches_paper_listing():
    cx, cy, w, opp = oracle.lattice()
    gx, gy, gw = read_lattice()          # Eq. ci evaluated by hand
    assert np.array_equal(cx, gx) and np.array_equal(cy, gy)
    assert np.allclose(w, gw, rtol=0, atol=1e-16)
    for i in range(9):
        assert cx[opp[i]] == -cx[i] and cy[opp[i]] == -cy[i]


def test_lattice_isotropy():
    # sum w = 1, sum w c = 0, sum w c c = cs2 I, sum w cccc = cs2^2 (dd + dd + dd)
    cx, cy, w, _ = oracle.lattice()
    c = np.stack([cx, cy], 1).astype(float)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(2), atol=1e-16)
    d = np.eye(2)
    iso4 = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)


@pytest.mark.parametrize("trial", range(20))
def test_feq_moments(trial):
    # Eq. feq_i: sum f = 0, sum c f = rho u, sum cc f = p I + rho u u
    cx, cy, _, _ = oracle.lattice()
    p, rho = rng.normal() * 1e-3, rng.uniform(0.1, 10)
    ux, uy = rng.normal(size=2) * 0.05
    f = oracle.feq(p, rho, ux, uy)
    m0, m1, m2 = moments(f, cx, cy)
    u = np.array([ux, uy])
    assert abs(m0) < 1e-15 * (1 + rho)
    assert np.allclose(m1, rho * u, atol=1e-15 * rho)
    assert np.allclose(m2, p * np.eye(2) + rho * np.outer(u, u), atol=1e-15 * (1 + rho))


@pytest.mark.parametrize("trial", range(20))
def test_geq_moments(trial):
    # Eq. H_i: sum g = phi, sum c g = 0, sum cc g = alpha mu cs2 I
    cx, cy, _, _ = oracle.lattice()
    phi, mu, alpha = rng.uniform(-0.1, 1.1), rng.normal() * 1e-3, rng.uniform(0.1, 2)
    g = oracle.geq(phi, mu, alpha)
    m0, m1, m2 = moments(g, cx, cy)
    assert abs(m0 - phi) < 1e-15
    assert np.allclose(m1, 0, atol=1e-18)
    assert np.allclose(m2, alpha * mu * CS2 * np.eye(2), atol=1e-18)


@pytest.mark.parametrize("trial", range(20))
def test_force_moments(trial):
    # Eq. GGi with prefactor P = 1 - 1/(2 tau_f): sum F_i = P u.grad(rho),
    # sum c F_i = P F, sum cc F_i = P cs2 (u.grad(rho) I + u grad(rho) + grad(rho) u)
    cx, cy, _, _ = oracle.lattice()
    tau = rng.uniform(0.51, 2.0)
    ux, uy, drx, dry, Fx, Fy = rng.normal(size=6) * np.array([.05, .05, .2, .2, 1e-3, 1e-3])
    Fi = oracle.force(tau, ux, uy, drx, dry, Fx, Fy)
    P = 1 - 1 / (2 * tau)
    u, dr = np.array([ux, uy]), np.array([drx, dry])
    m0, m1, m2 = moments(Fi, cx, cy)
    assert abs(m0 - P * u @ dr) < 1e-16
    assert np.allclose(m1, P * np.array([Fx, Fy]), atol=1e-17)
    exp2 = P * CS2 * ((u @ dr) * np.eye(2) + np.outer(u, dr) + np.outer(dr, u))
    assert np.allclose(m2, exp2, atol=1e-16)


@pytest.mark.parametrize("s", [-3e-3, 0.0, 1e-4, 2.5e-2])
def test_source_moments(s):
    # Eq. F_i: sum G = -s (the -u.grad(phi) of the CH equation), sum c G = 0,
    # sum cc G = 0 (no spurious flux or stress), G_0 = -2 w_0 s
    cx, cy, w, _ = oracle.lattice()
    G = oracle.source(s)
    m0, m1, m2 = moments(G, cx, cy)
    tol = 1e-15 * abs(s) + 1e-20
    assert abs(m0 + s) < tol
    assert np.allclose(m1, 0, atol=tol) and np.allclose(m2, 0, atol=tol)
    assert abs(G[0] + 2 * w[0] * s) < tol


@pytest.mark.parametrize("trial", range(10))
def test_velocity_pressure_round_trip(trial):
    # f = f^eq(p, rho, u) shifted by -F/2 in its first moment must return u and p
    # (the half-force correction of the velocity, Sec. 2.1.2); with grad(rho) = 0.
    cx, cy, w, _ = oracle.lattice()
    p, rho = rng.normal() * 1e-3, rng.uniform(0.1, 10)
    ux, uy = rng.normal(size=2) * 0.05
    Fx, Fy = rng.normal(size=2) * 1e-3
    f = oracle.feq(p, rho, ux, uy) - 0.5 * 3 * w * (cx * Fx + cy * Fy)
    vx, vy, pp = oracle.velocity_pressure(f, rho, 0.0, 0.0, Fx, Fy)
    assert abs(vx - ux) < 1e-15 and abs(vy - uy) < 1e-15
    assert abs(pp - p) < 1e-16


def test_pressure_density_gradient_term():
    # with grad(rho) != 0 the pressure gains cs2/(1 - w0) * u.grad(rho)/2
    p, rho, ux, uy = 2e-4, 3.0, 0.02, -0.01
    drx, dry = 0.3, -0.2
    f = oracle.feq(p, rho, ux, uy)
    vx, vy, pp = oracle.velocity_pressure(f, rho, drx, dry, 0.0, 0.0)
    assert abs(pp - (p + CS2 / (1 - 4 / 9) * 0.5 * (ux * drx + uy * dry))) < 1e-16


@pytest.mark.parametrize("trial", range(10))
def test_stencils_exact_on_polynomials(trial):
    # Eq. gradient is exact for degree <= 2, Eq. Laplace for degree <= 3.
    a = rng.normal(size=10)

    def poly(x, y):
        return (a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y
                + a[6] * x ** 3 + a[7] * x * x * y + a[8] * x * y * y + a[9] * y ** 3)

    x0, y0 = rng.normal(size=2)
    v = np.array([[poly(x0 + dx, y0 + dy) for dx in (-1, 0, 1)] for dy in (-1, 0, 1)])
    gx, gy, lap = oracle.stencil(v)
    lap_exact = (2 * a[3] + 2 * a[5] + 6 * a[6] * x0 + 2 * a[7] * y0 + 2 * a[8] * x0
                 + 6 * a[9] * y0)
    assert abs(lap - lap_exact) < 1e-12
    a2 = a.copy()
    a2[6:] = 0

    def poly2(x, y):
        return (a2[0] + a2[1] * x + a2[2] * y + a2[3] * x * x + a2[4] * x * y
                + a2[5] * y * y)

    v2 = np.array([[poly2(x0 + dx, y0 + dy) for dx in (-1, 0, 1)] for dy in (-1, 0, 1)])
    gx, gy, _ = oracle.stencil(v2)
    assert abs(gx - (a2[1] + 2 * a2[3] * x0 + a2[4] * y0)) < 1e-12
    assert abs(gy - (a2[2] + a2[4] * x0 + 2 * a2[5] * y0)) < 1e-12


def test_circle_fit_recovers_circle():
    t = np.linspace(0.3, 2.6, 40)
    a, b, R = 12.3, -4.5, 17.0
    c = oracle.circle_fit(a + R * np.cos(t), b + R * np.sin(t))
    assert np.allclose(c, [a, b, R], atol=1e-9)
