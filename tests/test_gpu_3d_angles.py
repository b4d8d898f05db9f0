"""Equilibrium contact angles of the 3D path (the 3D form of Secs. 3.1-3.3).

Resolved droplets (radius 16-20 lattice units, W = 4) on a flat wall, a
30 deg staircase plane and a solid sphere, 20000 steps in FP32 with the
(1/2) dG/dt term omitted, fitted on the device. The bars are regression
bounds a little above the errors this discretisation gives (measured: flat
1.1-2.7 deg, incline 0.4-1.3 deg, sphere 1.7-1.9 deg); at theta = 30 the
droplet is still spreading at 20000 steps and at theta = 150 (contact radius
~2 W) it leaves the wall, so those are reported by bench.py --workload
angles3d but not asserted here.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [("flat", 60.0, 2.5), ("flat", 90.0, 2.0), ("flat", 120.0, 3.5),
         ("incline", 60.0, 1.5), ("incline", 90.0, 1.5), ("incline", 120.0, 2.0),
         ("sphere", 60.0, 3.0), ("sphere", 90.0, 3.0)]


@pytest.mark.parametrize("kind,theta,bar", CASES)
def test_equilibrium_angle_3d(kind, theta, bar):
    from paper_2312_00369_gb300 import pflbm
    from paper_2312_00369_gb300 import workloads as wl
    c = {"flat": lambda: wl.droplet_on_flat_wall_3d(nx=96, ny=96, nz=56, R=20.0, theta=theta),
         "incline": lambda: wl.droplet_on_incline_3d(nx=128, ny=64, nz=112, gamma=30.0, R=20.0, theta=theta),
         "sphere": lambda: wl.droplet_on_sphere_3d(n=128, Rs=24.0, R=16.0, theta=theta)}[kind]()
    s = pflbm.Solver3D(c.solid, theta_deg=theta, precision="fp32", dgdt_mode=1, **c.physical())
    for d in c.droplets:
        s.init_droplet(*d)
    s.step(20000)
    s.check()
    fit, _, n = s.contact_angle(dict(dict(exclude=1.5 * c.W), **c.wall))
    s.close()
    assert n > 500
    assert abs(fit - theta) <= bar, fit
