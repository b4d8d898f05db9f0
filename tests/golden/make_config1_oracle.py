"""Write tests/golden/config1_oracle.npz: FP64 oracle results for the
inclined-wall and cylinder cases at their full length (20000 steps).

The runs omit the (1/2) dG/dt term (dgdt mode 1): with the backward
difference the period-2 mode has grown by 20000 steps (theta = 150 deg fits
as 180 deg, |u| reaches 0.14), so those states are not equilibria.

Calls only the oracle and the seeded input generators. Each case runs in its
own process. Stored per case: the contact angle and fitted circle, the mass,
and phi on every 4th node in x and y (as written, float64).

    python tests/golden/make_config1_oracle.py [--steps 20000]
"""
import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = [("incline", th) for th in (30.0, 60.0, 90.0, 120.0, 150.0)] + [("cylinder", 90.0)]


def run(args):
    kind, theta, steps, dgdt = args
    import oracle
    from paper_2312_00369_gb300 import workloads as wl
    c = (wl.droplet_on_incline(theta=theta, steps=steps) if kind == "incline"
         else wl.droplet_on_cylinder(theta=theta, steps=steps))
    o = oracle.Oracle(c.solid, theta_deg=c.theta_deg, **c.physical())
    o.set_dgdt(dgdt)
    for d in c.droplets:
        o.init_droplet(*d)
    o.step(steps)
    phi, u, p = o.get()
    th, circ, n = oracle.contact_angle(phi, o.geometry()["cls"], dict(c.wall, exclude=1.5 * c.W))
    return f"{kind}_{int(theta)}", dict(theta=th, circle=circ, npts=n, mass=o.mass(),
                                         phi_sub=phi[::4, ::4].copy(), umax=float(np.abs(u).max()),
                                         steps=steps, dgdt=dgdt)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--dgdt", type=int, default=1, choices=[0, 1])
    ap.add_argument("--out", default=os.path.join(HERE, "config1_oracle.npz"))
    a = ap.parse_args()
    with mp.get_context("spawn").Pool(len(CASES)) as pool:
        res = pool.map(run, [(k, t, a.steps, a.dgdt) for k, t in CASES])
    flat = {}
    for name, d in res:
        for k, v in d.items():
            flat[f"{name}:{k}"] = np.asarray(v)
        print(name, "theta", d["theta"], "npts", d["npts"], "umax", d["umax"], flush=True)
    np.savez_compressed(a.out, **flat)


if __name__ == "__main__":
    main()
