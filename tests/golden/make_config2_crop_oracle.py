"""Write tests/golden/config2_crop_oracle.npz: the FP64 oracle run of the
512 x 256 crop of the many-droplet flat-wall workload (8 droplets of radius
U[30, 60] at x ~ U[0, 512), per-node angle of the droplet nearest in x,
rho_l / rho_g = 10, seed 2312) for 10000 steps with the (1/2) dG/dt term
omitted (dgdt mode 1). With the backward difference the merged droplets'
flow grows from 7000 steps on (max |u| 0.007 at 7000, 0.017 at 8000, 0.17 at
10000; omitted: 0.0065 at 10000), so the states at 10000 steps are not
comparable between precisions.

Calls only the oracle, the seeded input generator and the window helper.
Stored at 2000, 5000 and 10000 steps (keys prefixed "t<steps>:"): phi and u
on every 4th node in x and y, the mass, max |u|, and for each droplet region
(droplets that touched are one region) its x window and the oracle's fitted
contact angle.

    python tests/golden/make_config2_crop_oracle.py [--steps 10000]
"""
import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


SNAPSHOTS = (2000, 5000, 10000)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=SNAPSHOTS[-1])
    ap.add_argument("--dgdt", type=int, default=1, choices=[0, 1])
    ap.add_argument("--out", default=os.path.join(HERE, "config2_crop_oracle.npz"))
    a = ap.parse_args()
    import oracle
    from paper_2312_00369_gb300 import workloads as wl
    from tests.droplet_windows import regions
    c = wl.many_droplets_flat(nx=512, ny=256, n_drops=8, seed=2312, steps=a.steps)
    o = oracle.Oracle(c.solid, theta_deg=c.theta_deg, theta_field=c.theta_field.astype(np.float64),
                      **c.physical())
    o.set_dgdt(a.dgdt)
    for d in c.droplets:
        o.init_droplet(*d)
    cls = o.geometry()["cls"]
    out = dict(steps=a.steps, dgdt=a.dgdt, snapshots=np.array(SNAPSHOTS, dtype=np.int64))
    done = 0
    for t in SNAPSHOTS:
        o.step(t - done)
        done = t
        phi, u, _ = o.get()
        wins, thetas, npts = [], [], []
        for x_lo, x_hi in regions(phi, c.solid):
            th, circ, n = oracle.contact_angle(phi, cls, dict(c.wall, x_lo=x_lo, x_hi=x_hi, exclude=1.5 * c.W))
            wins.append((x_lo, x_hi))
            thetas.append(th)
            npts.append(n)
            print(f"t={t}: region x [{x_lo}, {x_hi}): theta {th:.3f} deg from {n} points", flush=True)
        umax = float(np.sqrt((u ** 2).sum(-1)).max())
        print(f"t={t}: mass {o.mass()} max|u| {umax}", flush=True)
        p = f"t{t}:"
        out.update({p + "phi_sub": phi[::4, ::4].copy(), p + "u_sub": u[::4, ::4].copy(), p + "mass": o.mass(),
                    p + "umax": umax, p + "windows": np.array(wins, dtype=np.int64).reshape(-1, 2),
                    p + "theta": np.array(thetas), p + "npts": np.array(npts)})
    np.savez_compressed(a.out, **out)


if __name__ == "__main__":
    main()
