"""Pins of the variable-viscosity and body-force extension of the oracle
(Sec. 2.1.1: nu(phi) linear in phi, F = F_s + F_b; Sec. 2.1.2: nu =
c_s^2 (tau_f - 1/2)) and of the option that omits (1/2) dt^2 dG/dt."""
import numpy as np

import oracle
from paper_2312_00369_gb300 import workloads as wl


def channel(nx, ny):
    s = np.zeros((ny, nx), np.uint8)
    s[:2] = 1
    s[-2:] = 1
    return s


def test_poiseuille_curvature_fixes_viscosity():
    # single phase (phi = 1), body acceleration g along x between two walls:
    # rho nu u'' = -rho g, so the profile is a parabola of curvature -g / nu
    nx, ny, nu, g = 4, 34, 0.3, 1e-6
    o = oracle.Oracle(channel(nx, ny), theta_deg=90, tau_f=3 * nu + 0.5, rho_l=1.0, rho_g=0.1)
    o.set_body_force(g, 0.0)
    o.init_phi(np.ones((ny, nx)))
    o.step(4000)
    _, u, _ = o.get()
    ux = u[:, 1, 0]
    ys = np.arange(3, ny - 3)
    c = np.polyfit(ys, ux[ys], 2)
    assert abs(2 * c[0] / (-g / nu) - 1) < 1e-4
    assert np.allclose(ux, ux[::-1], rtol=1e-9, atol=1e-15)          # symmetric
    assert np.max(np.abs(u[..., 1])) < 1e-12                          # no cross flow


def test_two_layer_channel_curvature_per_phase():
    # liquid (nu_l) below, gas (nu_g) above; in each bulk layer u'' = -g / nu
    nx, ny, nl, ng, g = 4, 50, 0.3, 0.1, 1e-6
    o = oracle.Oracle(channel(nx, ny), theta_deg=90, tau_f=0.8, rho_l=1.0, rho_g=0.1)
    o.set_viscosity(nl, ng)
    o.set_body_force(g, 0.0)
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    o.init_phi(0.5 + 0.5 * np.tanh(2 * (25.0 - y) / 4))
    o.step(10000)
    _, u, _ = o.get()
    ux = u[:, 1, 0]
    lo, hi = np.arange(3, 17), np.arange(33, ny - 3)
    assert abs(2 * np.polyfit(lo, ux[lo], 2)[0] / (-g / nl) - 1) < 0.01
    assert abs(2 * np.polyfit(hi, ux[hi], 2)[0] / (-g / ng) - 1) < 0.01


def test_equal_viscosities_reduce_to_uniform_tau():
    case = wl.droplet_on_flat_wall(nx=60, ny=30, R=10.0, theta=70.0)
    a = oracle.Oracle(case.solid, theta_deg=70.0, **case.physical())
    b = oracle.Oracle(case.solid, theta_deg=70.0, **case.physical())
    nu = (case.tau_f - 0.5) / 3.0
    b.set_viscosity(nu, nu)
    for o in (a, b):
        o.init_droplet(30.0, 0.5, 10.0)
        o.step(200)
    pa, ua, _ = a.get()
    pb, ub, _ = b.get()
    assert np.max(np.abs(pa - pb)) < 1e-13 and np.max(np.abs(ua - ub)) < 1e-15


def test_budget_closes_without_dgdt_term():
    case = wl.droplet_on_flat_wall(theta=60.0)
    o = oracle.Oracle(case.solid, theta_deg=case.theta_deg, **case.physical())
    o.set_dgdt(1)
    o.init_droplet(*case.droplets[0])
    for _ in range(50):
        o.step(1)
        m_before, src, lost, bb = o.budget()
        assert abs(o.mass() - (m_before + src - lost + bb)) < 1e-12 * m_before
