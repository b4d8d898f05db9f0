"""Small parity cases run with the index-checked build (libpflbm_bounds.so).

Run as a script in its own process (the library is loaded once per process):
    PFLBM_LIBRARY=.../libpflbm_bounds.so python tests/bounds_cases.py
Every step kernel (global loads; staged, both tile shapes; two nodes per
thread) and the batched kernels step the cases; the script prints one JSON line with the number of
refused accesses and the FP32 error against the FP64 oracle, and exits 1 if
the build is not the index-checked one.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

CASES = ["tiny", "block", "incline45_ragged", "flat60_short", "cylinder"]


def main():
    import torch
    from tests import oracle_jobs as oj
    from paper_2312_00369_gb300 import pflbm, workloads as wl
    enabled, _ = pflbm.debug_bounds()
    if not enabled:
        print(json.dumps({"error": "not the index-checked build"}))
        return 1
    out = {"cases": {}}
    for name in CASES:
        case = oj.case_by_name(name)
        steps = min(case.steps, 120)
        ref = oj.run_case(name, steps)
        errs = {}
        for prec in ("fp32", "bf16"):
            for kernel in ("global", "staged32x8", "staged64x4", "pair"):
                s = pflbm.Solver(case.solid, theta_deg=case.theta_deg, theta_field=case.theta_field,
                                 precision=prec, step_kernel=kernel, step_chunk=3, **case.physical(),
                                 **oj.solver_options(case))
                for d in case.droplets:
                    s.init_droplet(*d)
                s.step(steps)
                phi, _, _ = s.get()
                s.mass()
                s.close()
                errs[f"{prec}/{kernel}"] = float(np.max(np.abs(phi - ref["phi"])))
        out["cases"][name] = errs
    # batches of uneven lattices, every batched kernel
    stream = torch.cuda.Stream()
    cases = wl.batched_instances(count=6, seed=11)
    for kernel in (1, 2, 3):
        members = []
        for c in cases:
            s = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision="bf16", stream=stream, **c.physical())
            for d in c.droplets:
                s.init_droplet(*d)
            members.append(s)
        b = pflbm.Batch(members, pflbm.schedule(tiles_per_item=2, kernel=kernel,
                                                classes=[(64 * 32, 1, 2), (256 * 128, 0, 3)]))
        b.step(31)
        torch.cuda.synchronize()
        b.close()
        for s in members:
            s.check()
            s.close()
    torch.cuda.synchronize()
    out["violations"] = pflbm.debug_bounds()[1]
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
