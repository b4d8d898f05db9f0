"""Schedule autotuner for batched steps (``pflbm_batch_t``).

The batched step has three knobs (``pflbm_schedule_t``): persistent CTAs per
SM, the work-item shape (how many 32 x 8 tiles of one tile column a CTA takes
per item) and the item order (lattice by lattice, or largest lattices first
and interleaved). The best choice depends on the mix of lattice sizes and on
the GPU, so it is measured: every candidate runs a few batched steps on
scratch copies of the lattices (same geometry and parameters, so the real
solves are not advanced), timed with CUDA events, and the fastest is cached
per (GPU, precision, size mix) in a JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import pflbm

CANDIDATES = [dict(ctas_per_sm=c, tiles_per_item=g, order=o, use_graph=1)
              for c in (0, 4) for g in (1, 2, 4, 8) for o in (0, 1)]


def cache_path():
    return os.environ.get("PFLBM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pflbm", "schedules.json"))


def signature(cases, precision, device_name):
    sizes = sorted((int(c.nx), int(c.ny)) for c in cases)
    h = hashlib.sha1(json.dumps(sizes).encode()).hexdigest()[:16]
    return f"{device_name}|{precision}|{len(sizes)}|{h}"


def _load_cache():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass


def tune(cases, precision="bf16", stream=None, steps=12, warmup=4, candidates=None,
         use_cache=True, verbose=False):
    """Return (best schedule dict, {candidate: ms per step}) for the cases."""
    import torch
    dev = torch.cuda.current_device()
    key = signature(cases, precision, torch.cuda.get_device_name(dev))
    cache = _load_cache() if use_cache else {}
    if use_cache and key in cache:
        return cache[key]["schedule"], cache[key].get("timings", {})
    if stream is None:
        stream = torch.cuda.Stream()
    scratch = []
    with torch.cuda.stream(stream):
        for c in cases:
            s = pflbm.Solver(c.solid, theta_deg=c.theta_deg, theta_field=c.theta_field,
                             precision=precision, stream=stream, **c.physical())
            for d in c.droplets:
                s.init_droplet(*d)
            scratch.append(s)
    timings = {}
    best, best_ms = None, float("inf")
    for cand in (candidates or CANDIDATES):
        b = pflbm.Batch(scratch, pflbm.schedule(**cand))
        b.step(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        b.close()
        name = "c{ctas_per_sm}_g{tiles_per_item}_o{order}".format(**cand)
        timings[name] = ms
        if verbose:
            print(f"autotune {name}: {ms:.4f} ms/step")
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    for s in scratch:
        s.close()
    if use_cache:
        cache = _load_cache()
        cache[key] = {"schedule": best, "timings": timings, "when": time.time()}
        _save_cache(cache)
    return best, timings
