"""Schedule autotuner for batched steps (``pflbm_batch_t``).

The batched step has three kernels and several knobs (``pflbm_schedule_t``):

* the global-load kernel (32 x 8 tiles): persistent CTAs per SM, tiles of one
  tile column per work item, item order;
* the two-node kernel (64 x 8 tiles, two x-adjacent nodes per thread in
  packed FP32x2 arithmetic; one launch per group of same-size lattices,
  side by side): no knobs, one candidate;
* the staged kernel (TMA ring): per size class of the mix, the tile shape
  (32 x 8 or 64 x 4) and the tiles a CTA marches down per work item.

The best choice depends on the mix of lattice sizes and on the GPU, so it is
measured. Every candidate runs a few batched steps on scratch copies of the
lattices (same geometry and parameters, so the real solves are not
advanced), timed with CUDA events. The global-load kernel's knobs are
swept as a grid; the staged kernel's per-class shape and item length are
chosen by coordinate descent over the classes, largest total node count
first. The fastest schedule is cached per (GPU, precision, size mix) in a
JSON file.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import pflbm

GLOBAL_CANDIDATES = [dict(kernel=1, ctas_per_sm=c, tiles_per_item=g, order=o, use_graph=1)
                     for c in (0, 4) for g in (1, 2, 4, 8) for o in (0, 1)]
PAIR_CANDIDATES = [dict(kernel=3, ctas_per_sm=0, tiles_per_item=1, order=0, use_graph=1)]
STAGED_OPTIONS = [(shape, tiles) for shape in (0, 1) for tiles in (2, 4, 8, 16)]


def cache_path():
    return os.environ.get("PFLBM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pflbm", "schedules.json"))


def signature(cases, precision, device_name):
    sizes = sorted((int(c.nx), int(c.ny)) for c in cases)
    h = hashlib.sha1(json.dumps(sizes).encode()).hexdigest()[:16]
    return f"v4|{device_name}|{precision}|{len(sizes)}|{h}"


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


def name_of(sched):
    if sched.get("kernel", 1) == 3:
        return "pair_by_size"
    if sched.get("kernel", 1) == 2:
        cls = ",".join(f"{m}:{'32x8' if s == 0 else '64x4'}/{t}" for m, s, t in sched["classes"])
        return f"staged[{cls}]"
    return "global_c{ctas_per_sm}_g{tiles_per_item}_o{order}".format(**sched)


def to_schedule(sched):
    """A ``pflbm_schedule_t`` from a schedule dict."""
    kw = {k: sched[k] for k in ("ctas_per_sm", "tiles_per_item", "order", "use_graph", "kernel") if k in sched}
    return pflbm.schedule(classes=[tuple(c) for c in sched.get("classes", [])], **kw)


def tune(cases, precision="bf16", stream=None, steps=12, warmup=4, candidates=None,
         use_cache=True, verbose=False, staged=True):
    """Return (best schedule dict, {candidate name: ms per step}) for the cases."""
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
    explicit = candidates is not None

    def measure(sched):
        b = pflbm.Batch(scratch, to_schedule(sched))
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
        timings[name_of(sched)] = ms
        if verbose:
            print(f"autotune {name_of(sched)}: {ms:.4f} ms/step")
        return ms

    best, best_ms = None, float("inf")
    if candidates is None:
        candidates = GLOBAL_CANDIDATES + (PAIR_CANDIDATES if precision != "fp64" else [])
    for cand in candidates:
        ms = measure(cand)
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    if staged and precision != "fp64" and not explicit:
        # size classes: the distinct lattice sizes, by node count
        nodes = {}
        for c in cases:
            n = int(c.nx) * int(c.ny)
            nodes[n] = nodes.get(n, 0) + n
        classes = sorted(nodes)                             # max_nodes of each class, ascending
        order = sorted(classes, key=lambda n: -nodes[n])    # tuned largest total first
        choice = {n: (0, 4) for n in classes}

        def sched_of(ch):
            return dict(kernel=2, ctas_per_sm=0, tiles_per_item=4, order=0, use_graph=1,
                        classes=[[n, ch[n][0], ch[n][1]] for n in classes])

        cur_ms = measure(sched_of(choice))
        for n in order[:8]:
            for opt in STAGED_OPTIONS:
                if opt == choice[n]:
                    continue
                trial = dict(choice)
                trial[n] = opt
                ms = measure(sched_of(trial))
                if ms < cur_ms:
                    choice, cur_ms = trial, ms
        if cur_ms < best_ms:
            best, best_ms = sched_of(choice), cur_ms
    for s in scratch:
        s.close()
    if use_cache:
        cache = _load_cache()
        cache[key] = {"schedule": best, "timings": timings, "when": time.time()}
        _save_cache(cache)
    return best, timings
