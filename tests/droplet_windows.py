"""Contact-angle windows of a multi-droplet field on a flat floor.

Measurement helper shared by the tests and the scripts that write their
stored oracle values: it finds the connected regions of phi > 1/2 (droplets
that touched have merged into one region) and returns, for each region that
does not cross the periodic seam, the x window [x_lo, x_hi) that holds it.
The contact angle of each region is then fitted inside its window (the
oracle's fit on the oracle's field, the library's device fit on the GPU
field), with the same wall and exclusion band on both sides. Pure numpy; no
arithmetic of the scheme.
"""
import numpy as np


def regions(phi, solid, margin=6):
    """[(x_lo, x_hi), ...] of the phi > 1/2 regions of the fluid, left to
    right; regions touching x = 0 or x = nx - 1 are left out."""
    ny, nx = phi.shape
    wet = (phi > 0.5) & (solid == 0)
    cols = wet.any(axis=0)
    out = []
    x = 0
    while x < nx:
        if not cols[x]:
            x += 1
            continue
        x0 = x
        while x < nx and cols[x]:
            x += 1
        if x0 > 0 and x < nx:
            out.append((max(0, x0 - margin), min(nx, x + margin)))
    return out
