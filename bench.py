"""Benchmark: MLUPS and fraction of the HBM roofline of the fused time step.

Workload (default): 4096 x 2048 lattice, flat bottom wall, 64 droplets of
radius U[30, 60] at random x, per-node contact angle U[30, 150] deg (seed
2312), rho_l / rho_g = 10, FP32 storage and arithmetic. One bench step is one
time step of the whole lattice (all of: order parameter, ghost fill,
stencils, chemical potential with the wetting term, forces, moments, both
collisions, streaming with bounce-back). The state (1.2 GB) is far larger
than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--precision fp32|fp64] [--workload many_flat|flat|incline|cylinder|
                     batched|serving|wsweep|many_flat3d|angles3d]

Prints one JSON line (rank 0). Under torchrun each rank runs an independent
replica of the workload (the solver does not shard: replicas only).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# algorithmic bytes per lattice update of the fused step: every f_i and g_i
# read once and written once, the u.grad(phi) history read and written once,
# one node byte (the wetting coefficient is read on wall layers only)
BYTES_PER_LU = {"fp64": 2 * 9 * 2 * 8 + 2 * 8 + 1, "fp32": 2 * 9 * 2 * 4 + 2 * 4 + 1,
                # 17 populations in 16 bits, g_0 in 32 bits, FP32 history
                "bf16": 2 * (17 * 2 + 4) + 2 * 4 + 1, "fp16": 2 * (17 * 2 + 4) + 2 * 4 + 1}


def max_over_ranks(x, device, world):
    """The largest value of x over all ranks (x itself when world == 1).
    Every rank calls it; the barrier makes the slowest rank decide."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def pinned(torch, shape, dtype):
    """A numpy view of page-locked host memory (allocated outside timed regions)."""
    tdt = {np.float64: torch.float64, np.float32: torch.float32, np.uint8: torch.uint8}[np.dtype(dtype).type]
    return torch.empty(tuple(shape), dtype=tdt, pin_memory=True).numpy()


def whole_job_mlups(world, nodes, steps, seconds):
    """Lattice updates of all replicas (world x nodes x steps) per second, in millions."""
    return world * nodes * steps / seconds / 1e6


def step_source_sha256(files=("step.cu", "step2.cu", "step_core.cuh", "storage.cuh", "pflbm_internal.cuh")):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2312_00369_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_case(name):
    from paper_2312_00369_gb300 import workloads as wl
    if name == "many_flat":
        return wl.many_droplets_flat(nx=4096, ny=2048, n_drops=64, seed=2312)
    if name == "flat":
        return wl.droplet_on_flat_wall()
    if name == "incline":
        return wl.droplet_on_incline(theta=60.0)
    if name == "cylinder":
        return wl.droplet_on_cylinder()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def wait_first(self, timeout=3.0):
        """Block until nvidia-smi has printed its first sample (its start-up
        takes longer than a short timed region)."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(case, seconds=12.0):
    """Time the FP64 CPU oracle (single thread, as it stands) on a bounded
    512 x 256 sample of the workload; returns (MLUPS, description)."""
    import oracle
    from paper_2312_00369_gb300 import workloads as wl
    if case.name == "many_flat":
        sub = wl.many_droplets_flat(nx=512, ny=256, n_drops=8, seed=2312)
    else:
        sub = case
    o = oracle.Oracle(sub.solid, theta_deg=sub.theta_deg, theta_field=sub.theta_field,
                      **sub.physical())
    for d in sub.droplets:
        o.init_droplet(*d)
    n = sub.nx * sub.ny
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(5)
        steps += 5
    dt = time.perf_counter() - t0
    return n * steps / dt / 1e6, f"{sub.nx}x{sub.ny} lattice of the same generator, {steps} steps"


def _oracle_worker(job):
    """One host core's share of the CPU baseline: the oracle, as it stands, on
    the bounded sample of a workload. Returns (lattice updates, seconds, text)."""
    kind, workload, seconds = job
    if kind == "3d":
        mlups, desc = oracle_sample_3d(seconds)
    else:
        mlups, desc = oracle_sample(make_case(workload), seconds)
    return mlups * 1e6 * seconds, seconds, desc


def oracle_baseline(kind, workload, seconds):
    """The CPU baseline on all host cores: one independent copy of the oracle
    sample per core (the oracle itself is single-threaded and unchanged), in a
    spawn pool. Returns (MLUPS of all copies, cores, description)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    jobs = [(kind, workload, seconds)] * cores
    if cores == 1:
        res = [_oracle_worker(jobs[0])]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    lu = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    return lu / wall / 1e6, cores, f"{cores} independent copies (one per host core) of: {res[0][2]}"


def run_reference(args, rank, world):
    if rank != 0:
        return
    secs = max(3.0, min(20.0, 2.0 * args.steps))
    if args.workload == "many_flat3d":
        mlups, cores, desc = oracle_baseline("3d", "many_flat3d", secs)
        cfg = {"workload": "many_flat3d", "nx": 512, "ny": 512, "nz": 128}
    else:
        case = make_case(args.workload)
        mlups, cores, desc = oracle_baseline("2d", args.workload, secs)
        cfg = {"workload": case.name, "nx": case.nx, "ny": case.ny}
    line = {
        "impl": "reference", "metric": "MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, torch, rank, world, local):
    line = batched_line(args, torch, world, local, args.steps, args.warmup, plain=True)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batched_line(args, torch, world, local, steps, warmup, plain=True, precision=None):
    """256 uneven lattices (sizes from {64x32 .. 512x256}, flat / 30 deg
    incline / cylinder walls, theta ~ U[30, 150], seed 369), advanced by one
    persistent launch per step with the autotuned schedule, replayed from a
    CUDA graph. Also times the plain path: the same lattices in FP32, one
    launch per lattice per step."""
    from paper_2312_00369_gb300 import autotune, workloads as wl
    from paper_2312_00369_gb300.pflbm import Batch, Solver
    cases = wl.batched_instances(256, seed=369, steps=5000)
    nodes = sum(c.nx * c.ny for c in cases)
    stream = torch.cuda.Stream(device=local)

    def build(precision):
        out = []
        with torch.cuda.stream(stream):
            for c in cases:
                sv = Solver(c.solid, theta_deg=c.theta_deg, precision=precision, device=local,
                            stream=stream, **c.physical())
                for d in c.droplets:
                    sv.init_droplet(*d)
                out.append(sv)
        return out

    precision = args.precision if precision is None else precision
    sched, timings = autotune.tune(cases, precision, stream=stream)
    solvers = build(precision)
    b = Batch(solvers, autotune.to_schedule(sched))
    b.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    sampler.wait_first()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    for sv in solvers:
        sv.check()
    info = b.info()
    kernel = b.kernel
    b.close()
    for sv in solvers:
        sv.close()
    value = nodes * steps / (ms * 1e-3) / 1e6

    plain_mlups = None
    if plain:
        # the plain path: FP32, one launch per lattice per step
        ps = build("fp32")
        k_plain = max(3, steps // 4)
        for sv in ps:
            sv.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(k_plain):
            for sv in ps:
                sv.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_plain = e0.elapsed_time(e1)
        for sv in ps:
            sv.close()
        plain_mlups = nodes * k_plain / (ms_plain * 1e-3) / 1e6
    peak, peak_kind = load_peaks()
    bpl = BYTES_PER_LU[precision]
    achieved = bpl * nodes / (ms / steps * 1e-3) / 1e9
    return {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": precision + " storage", "data": "synthetic",
        "config": {"workload": "batched", "lattices": len(cases), "nodes": nodes,
                   "precision": precision, "schedule": sched, "kernel": kernel, "work_items": info["n_work"],
                   "grid": info["grid"], "l2": "state of all lattices > L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "bytes_per_lu": bpl},
        "plain_fp32_one_launch_per_lattice_mlups": plain_mlups,
        "speedup_vs_plain": (value / plain_mlups) if plain_mlups else None,
        "autotune_ms_per_step": timings,
        # the two-node batched kernel runs one launch per group of same-size
        # lattices each step (batch info's grid); the others one launch
        "gpu_launches": (info["grid"] if kernel == 3 else 1) * steps, "clocks": clocks,
    }


def run_serving(args, torch, rank, world, local):
    line = serving_line(args, torch, world, args.serve_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_line(args, torch, world, T, prec=None, dgdt=None):
    """Poisson request stream (2000 requests/s, sizes 128x64 .. 1024x512
    log-uniform, steps U[1000, 20000], random wall and theta, seed 2024)
    served by continuous batching with 16-bit storage (FP16 unless --precision
    bf16) and, unless --dgdt 0, the (1/2) dG/dt term omitted. The offered load is far
    beyond one GPU (about 2.6e12 lattice updates per second), so this run is
    bounded in wall time and reports completed / admitted / queued counts; a
    second pair of runs at a sustainable rate (70 % of the measured capacity)
    compares the batched server with the plain FP32 one-launch-per-solve path."""
    from paper_2312_00369_gb300 import workloads as wl
    from paper_2312_00369_gb300.serve import PlainServer, Server, requests_from_stream
    # FP16 (scaled) storage by default: as fast as BF16 and about 100x closer to
    # the FP64 oracle in phi, which keeps the served angles within 0.5 deg
    if prec is None:
        prec = args.precision if "--precision" in sys.argv and args.precision in ("bf16", "fp16") else "fp16"
    budget = int(args.hbm_budget_gb * (1 << 30))
    over = requests_from_stream(wl.request_stream(rate=2000.0, duration=T, seed=2024))

    def serve(cls, reqs, drain, **kw):
        srv = cls(hbm_budget=budget, max_slots=args.max_slots, tick=args.tick,
                  dgdt_mode=args.dgdt if dgdt is None else dgdt, **kw)
        try:
            st = srv.run(reqs, duration=T, drain=drain, max_wall=(4 * T if drain else T))
            return st.summary(), st.results
        finally:
            srv.close()

    # saturated: both servers under the stated (overloaded) stream
    s_over, _ = serve(Server, over, False, precision=prec)
    s_over_plain, _ = serve(PlainServer, over, False)
    # a sustainable rate: 70 % of the batched server's measured capacity
    mean_lu = float(np.mean([r.nx * r.ny * r.steps for r in over]))
    rate = 0.7 * s_over["processed_mlups"] * 1e6 / mean_lu
    sus = requests_from_stream(wl.request_stream(rate=rate, duration=T, seed=2025))
    sb, rb = serve(Server, sus, True, precision=prec)
    sp, rp = serve(PlainServer, sus, True)
    # the plain path at 70 % of its own capacity (its p99 without the queue
    # the batched server's rate builds up)
    rate_plain = 0.7 * s_over_plain["processed_mlups"] * 1e6 / mean_lu
    sus_p = requests_from_stream(wl.request_stream(rate=rate_plain, duration=T, seed=2026))
    spp, _ = serve(PlainServer, sus_p, True)
    # the same requests served both ways: contact angle of the batched 16-bit
    # result against the plain FP32 one
    tb = {r.rid: r.theta_fit for r in rb if not r.failed and np.isfinite(r.theta_fit)}
    tp = {r.rid: r.theta_fit for r in rp if not r.failed and np.isfinite(r.theta_fit)}
    common = sorted(set(tb) & set(tp))
    dth = np.array([abs(tb[i] - tp[i]) for i in common]) if common else np.array([np.nan])
    angle = {"requests_compared": len(common), "max_abs_deg": float(np.max(dth)),
             "p99_abs_deg": float(np.percentile(dth, 99)), "within_0_5_deg": int(np.sum(dth < 0.5)),
             "reference": "the same request served by the plain FP32 path"}
    line = {
        "metric": "MLUPS", "value": s_over["processed_mlups"], "unit": "MLUPS", "n_gpus": world,
        "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec + " storage", "data": "synthetic",
        "config": {"workload": "serving", "seconds": T, "hbm_budget_gb": args.hbm_budget_gb,
                   "max_slots": args.max_slots, "tick": args.tick, "precision": prec,
                   "dgdt_mode": args.dgdt if dgdt is None else dgdt},
        "value_is": "lattice updates per second processed by the batched server under the stated stream",
        "overloaded_2000_per_s": s_over,
        "overloaded_2000_per_s_plain_fp32": s_over_plain,
        "sustainable_rate_per_s": rate,
        "sustainable_batched": sb,
        "sustainable_plain_fp32_one_launch_per_solve": sp,
        "plain_fp32_rate_per_s_at_70pct_own_capacity": rate_plain,
        "plain_fp32_at_70pct_own_capacity": spp,
        "sustainable_angle_batched_vs_plain": angle,
        "p99_ratio_plain_over_batched": sp["p99_s"] / sb["p99_s"] if sb["p99_s"] > 0 else None,
        "throughput_ratio_batched_over_plain_saturated":
            s_over["processed_mlups"] / max(s_over_plain["processed_mlups"], 1e-9),
    }
    return line


def run_wsweep(args, torch, rank, world, local):
    """Interface-width sweep of Sec. 3.2: droplet of radius 50 on the staircase
    wall y = x/4 (gamma = atan 0.25) of a 256 x 256 lattice, theta = 90 and
    120 deg, W = 4, 6, 8 (sigma, M, densities as elsewhere; FP32). All six
    solves advance in one batch; the measured angle and its error are
    reported per (W, theta)."""
    import math
    from paper_2312_00369_gb300 import workloads as wl
    from paper_2312_00369_gb300.pflbm import Batch, Solver
    gamma = math.degrees(math.atan(0.25))
    stream = torch.cuda.Stream(device=local)
    runs = []
    with torch.cuda.stream(stream):
        for W in (4.0, 6.0, 8.0):
            for th in (90.0, 120.0):
                c = wl.droplet_on_incline(nx=256, ny=256, gamma=gamma, R=50.0, theta=th, W=W)
                sv = Solver(c.solid, theta_deg=th, precision=args.precision, device=local, stream=stream,
                            dgdt_mode=args.dgdt, **c.physical())
                for d in c.droplets:
                    sv.init_droplet(*d)
                runs.append((W, th, c, sv))
    b = Batch([r[3] for r in runs])
    steps = long_solve_steps(args)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    table = {}
    for W, th, c, sv in runs:
        fit, circ, n = sv.contact_angle(dict(c.wall, exclude=1.5 * W))
        table.setdefault(f"W={W:g}", {})[f"theta={th:g}"] = {"measured": fit, "error": fit - th, "points": n}
    b.close()
    for r in runs:
        r[3].close()
    nodes = sum(r[3].nx * r[3].ny for r in runs)
    line = {"metric": "MLUPS", "value": nodes * steps / dt / 1e6, "unit": "MLUPS", "n_gpus": world,
            "steps": steps, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "wsweep", "lattice": "256x256", "gamma_deg": gamma, "R": 50,
                       "dgdt_mode": args.dgdt},
            "contact_angle": table}
    if rank == 0:
        print(json.dumps(line), flush=True)


def angle_cases_3d():
    """The 3D contact-angle table: flat wall (96 x 96 x 56, R = 20), 30 deg
    staircase plane (128 x 64 x 112, R = 20) and solid sphere of radius 24
    (128^3, R = 16)."""
    from paper_2312_00369_gb300 import workloads as wl
    out = [("flat", th, wl.droplet_on_flat_wall_3d(nx=96, ny=96, nz=56, R=20.0, theta=th))
           for th in (30.0, 60.0, 90.0, 120.0, 150.0)]
    out += [("incline30", th, wl.droplet_on_incline_3d(nx=128, ny=64, nz=112, gamma=30.0, R=20.0, theta=th))
            for th in (60.0, 90.0, 120.0)]
    out += [("sphere", th, wl.droplet_on_sphere_3d(n=128, Rs=24.0, R=16.0, theta=th)) for th in (60.0, 90.0, 120.0)]
    return out


def long_solve_steps(args, default=20000):
    """Steps of a workload that runs solves to equilibrium: --steps when given
    on the command line, else `default` (the timed-step default is far too
    short for an equilibrium angle)."""
    given = any(a == "--steps" or a.startswith("--steps=") for a in sys.argv[1:])
    return args.steps if given else default


def run_angles3d(args, torch, rank, world, local):
    """Equilibrium contact angles in 3D (the 3D column of the paper's angle
    comparison, Secs. 3.1-3.3): every case of angle_cases_3d() run for
    `steps` (default 20000) with the (1/2) dG/dt term as --dgdt (default for
    this workload: omitted), FP32; the fitted angle and its error per case."""
    from paper_2312_00369_gb300.pflbm import PflbmError, Solver3D
    steps = long_solve_steps(args)
    stream = torch.cuda.Stream(device=local)
    table, lu, busy = {}, 0, 0.0
    for kind, th, c in angle_cases_3d():
        with torch.cuda.stream(stream):
            sv = Solver3D(c.solid, theta_deg=th, precision="fp32", device=local, stream=stream,
                          dgdt_mode=args.dgdt, **c.physical())
            for d in c.droplets:
                sv.init_droplet(*d)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv.step(steps)
            torch.cuda.synchronize()
            busy += time.perf_counter() - t0
            lu += int(np.prod(c.shape)) * steps
            try:
                sv.check()
                fit, sph, n = sv.contact_angle(dict(dict(exclude=1.5 * c.W), **c.wall))
                row = {"measured": fit, "error": fit - th, "points": n}
            except PflbmError as e:
                row = {"failed": str(e)}
            sv.close()
        table.setdefault(kind, {})[f"theta={th:g}"] = row
    line = {"metric": "MLUPS", "value": lu / busy / 1e6, "unit": "MLUPS", "n_gpus": world, "steps": steps,
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
            "data": "synthetic",
            "config": {"workload": "angles3d", "dgdt_mode": args.dgdt,
                       "cases": "flat 96x96x56 R=20; incline30 128x64x112 R=20; sphere Rs=24 128^3 R=16"},
            "contact_angle": table}
    if rank == 0:
        print(json.dumps(line), flush=True)


# three dimensions (D3Q19 f, D3Q7 g): every f_i and g_i read and written
# once, the history read and written once, one node byte
BYTES_PER_LU_3D = {"fp64": 2 * (19 + 7) * 8 + 2 * 8 + 1, "fp32": 2 * (19 + 7) * 4 + 2 * 4 + 1}


def oracle_sample_3d(seconds=10.0):
    """Time the FP64 3D CPU oracle (single thread, as it stands) on a bounded
    sample: a 64 x 64 x 32 box with 4 droplets of the same generator."""
    import oracle
    from paper_2312_00369_gb300 import workloads as wl
    sub = wl.many_droplets_3d(nx=64, ny=64, nz=32, n_drops=4, r_lo=6.0, r_hi=10.0)
    o = oracle.Oracle3D(sub.solid, theta_deg=sub.theta_deg, **sub.physical())
    for d in sub.droplets:
        o.init_droplet(*d)
    n = int(np.prod(sub.shape))
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(2)
        steps += 2
    dt = time.perf_counter() - t0
    return n * steps / dt / 1e6, f"64x64x32 box of the same generator (4 droplets), {steps} steps"


def run_3d(args, torch, rank, world, local):
    """512 x 512 x 128 box, flat bottom wall, 64 droplets of radius U[12, 24],
    theta = 60 deg; one bench step = one time step (3 launches: order
    parameter, ghost fill, fused collide-and-stream)."""
    import torch.distributed as dist
    from paper_2312_00369_gb300 import workloads as wl
    from paper_2312_00369_gb300.pflbm import Solver3D, lib
    prec = args.precision if args.precision in ("fp32", "fp64") else "fp32"
    nx, ny, nz = (int(v) for v in args.size3d.split("x"))
    case = wl.many_droplets_3d(nx=nx, ny=ny, nz=nz)
    N = int(np.prod(case.shape))
    stream = torch.cuda.Stream(device=local)
    lib()
    with torch.cuda.stream(stream):
        s = Solver3D(case.solid, theta_deg=case.theta_deg, precision=prec, device=local, stream=stream,
                     step_path=args.path3d, **case.physical())
        for d in case.droplets:
            s.init_droplet(*d)
        s.step(args.warmup)
        s.check()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # the K-step region is repeated until it has run for at least 300 ms
        # (clock samples need that long); each repeat is bracketed by a
        # barrier and a synchronize, and the repeat count is the same on
        # every rank (from the slowest rank's first region)
        sampler = ClockSampler(local)
        sampler.start()
        sampler.wait_first()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def region():
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0.record(stream)
            s.step(args.steps)          # K launches of the fused step kernel
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        times = [region()]
        first = max_over_ranks(times[0], f"cuda:{local}", world)
        repeats = max(1, min(1000, int(math.ceil(300.0 / max(first, 1e-3)))))
        while len(times) < repeats:
            times.append(region())
        clocks = sampler.stop()
        ms = sum(times) / len(times)
        s.check()
    ms = max_over_ranks(ms, f"cuda:{local}", world)
    ms_per_step = ms / args.steps
    value = whole_job_mlups(world, N, args.steps, ms * 1e-3)
    peak, peak_kind = load_peaks()
    bpl = BYTES_PER_LU_3D[prec]
    achieved = bpl * N / (ms_per_step * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile) and case.shape == (128, 512, 512):
        try:
            t = json.load(open(tfile)).get(f"many_flat3d:{prec}:{args.path3d}")
            if t and t.get("step_source_sha256") == step_source_sha256(
                    ("step3d.cu", "storage.cuh", "pflbm_internal.cuh")):
                traffic = t["bytes_per_launch"]
        except Exception:
            traffic = None

    e2e_steps = args.e2e_steps
    solid_h = pinned(torch, case.solid.shape, np.uint8)
    solid_h[...] = case.solid
    rb = np.float64 if prec == "fp64" else np.float32
    outs = (pinned(torch, case.shape, rb), pinned(torch, case.shape + (3,), rb), pinned(torch, case.shape, rb))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s2 = Solver3D(solid_h, theta_deg=case.theta_deg, precision=prec, device=local, stream=stream,
                      step_path=args.path3d, **case.physical())
        for d in case.droplets:
            s2.init_droplet(*d)
        s2.step(e2e_steps)
        phi, u, p = s2.get(out=outs) if rb is np.float64 else s2.get_f32(out=outs)
        s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, f"cuda:{local}", world)
    extra = None
    if rank == 0 and world == 1 and not args.no_extra and case.name == "many_flat" and args.precision == "fp32":
        extra = extra_block(args, torch, world, local, case, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc = oracle_baseline("3d", "many_flat3d", 10.0)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64"}[prec], "data": "synthetic",
            "config": {"workload": case.name, "nx": case.shape[2], "ny": case.shape[1], "nz": case.shape[0],
                       "droplets": len(case.droplets), "precision": prec, "step_path": args.path3d,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state %.1f GB > L2, no flush needed" % (2 * 26 * (4 if prec == "fp32" else 8) * N / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "bytes_per_lu": bpl,
                         "kernel": "whole step (k3_fused, 1 launch)" if args.path3d == "fused"
                         else "whole step (k3_phi, k3_ghost, k3_step: 3 launches)"},
            "hbm_roofline_mlups": peak * 1e9 / bpl / 1e6,
            "e2e": {"value": whole_job_mlups(world, N, e2e_steps, e2e_s), "unit": "MLUPS",
                    "h2d_bytes_per_step": case.solid.nbytes / e2e_steps,
                    "d2h_bytes_per_step": (phi.nbytes + u.nbytes + p.nbytes) / e2e_steps,
                    "steps_per_solve": e2e_steps,
                    "includes": "create (mask upload, geometry), droplet init, steps, get (float64 for "
                                "FP64 solves, float32 otherwise)",
                    "host_buffers": "pinned"},
            "gpu_launches": (1 if args.path3d == "fused" else 3) * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def extra_block(args, torch, world, local, case, stream):
    """The other paths, measured in the same run: the 16-bit step on the same
    lattice, the batched config-3 workload with the autotuned schedule, and
    short serving runs (capacity, a sustainable rate, each path at 70 % of its
    own capacity)."""
    from paper_2312_00369_gb300.pflbm import Solver
    out = {}
    N = case.nx * case.ny
    with torch.cuda.stream(stream):
        s = Solver(case.solid, theta_deg=case.theta_deg, theta_field=case.theta_field, precision="bf16",
                   device=local, stream=stream, **case.physical())
        for d in case.droplets:
            s.init_droplet(*d)
        kernel16 = s.step_kernel
        s.step(20)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        k = 1000
        e0.record(stream)
        s.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        s.check()
        s.close()
    ms = e0.elapsed_time(e1) / k
    peak, peak_kind = load_peaks()
    achieved = BYTES_PER_LU["bf16"] * N / (ms * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            t = json.load(open(tfile)).get(f"many_flat:bf16:{kernel16}")
            if t and t.get("step_source_sha256") == step_source_sha256():
                traffic = t["bytes_per_launch"]
        except Exception:
            traffic = None
    out["bf16_many_flat"] = {"value": N / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": k,
                             "step_kernel": kernel16,
                             "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                          "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                                          "bytes_per_lu": BYTES_PER_LU["bf16"]}}
    b = batched_line(args, torch, world, local, 400, 5, plain=False, precision="bf16")
    out["batched_bf16_config3"] = {kk: b[kk] for kk in ("value", "unit", "ms_per_step", "steps", "config",
                                                        "roofline", "clocks")}
    out["batched_bf16_config3"]["autotune_candidates"] = len(b["autotune_ms_per_step"])
    # the serving defaults: FP16 storage, the (1/2) dG/dt term omitted (long
    # solves at these parameters are not stable with the backward difference)
    sv = serving_line(args, torch, world, 5.0, prec="fp16", dgdt=1)
    keep = ("sustainable_rate_per_s", "sustainable_batched", "sustainable_plain_fp32_one_launch_per_solve",
            "plain_fp32_rate_per_s_at_70pct_own_capacity", "plain_fp32_at_70pct_own_capacity",
            "sustainable_angle_batched_vs_plain", "p99_ratio_plain_over_batched",
            "throughput_ratio_batched_over_plain_saturated")
    out["serving_fp16_5s"] = {kk: sv[kk] for kk in keep}
    out["serving_fp16_5s"]["config"] = sv["config"]
    out["serving_fp16_5s"]["capacity_mlups"] = {"batched": sv["overloaded_2000_per_s"]["processed_mlups"],
                                                "plain_fp32": sv["overloaded_2000_per_s_plain_fp32"]["processed_mlups"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16", "fp16"])
    ap.add_argument("--workload", default="many_flat")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra block (BF16 step, batched config 3, short serving runs)")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--hbm-budget-gb", type=float, default=64.0)
    ap.add_argument("--max-slots", type=int, default=512)
    ap.add_argument("--tick", type=int, default=200)
    ap.add_argument("--size3d", default="512x512x128", help="nx x ny x nz of many_flat3d")
    ap.add_argument("--path3d", default="auto", choices=["auto", "fused", "three_pass"],
                    help="3D step: one fused launch or three launches")
    ap.add_argument("--kernel", default="default", choices=["default", "global", "staged32x8", "staged64x4", "pair"],
                    help="2D step kernel (results identical; speed differs)")
    ap.add_argument("--chunk", type=int, default=0, help="staged kernel: tiles per work item (0: library default)")
    ap.add_argument("--dgdt", type=int, default=0, choices=[0, 1],
                    help="(1/2) dG/dt: 0 backward difference, 1 omitted")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2312_00369_gb300.pflbm import Solver, lib

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    if args.workload in ("batched", "serving", "wsweep", "many_flat3d", "angles3d"):
        if args.workload in ("angles3d", "serving", "wsweep") and "--dgdt" not in sys.argv:
            # long solves: the (1/2) dG/dt term omitted unless asked for (the
            # backward difference is not at equilibrium by 1e4-2e4 steps, and
            # on the shallow staircase of the W sweep it goes unstable)
            args.dgdt = 1
        {"batched": run_batched, "serving": run_serving, "wsweep": run_wsweep,
         "many_flat3d": run_3d, "angles3d": run_angles3d}[args.workload](
            args, torch, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return
    case = make_case(args.workload)
    N = case.nx * case.ny
    stream = torch.cuda.Stream(device=local)
    lib()

    # ---------------- device-resident throughput ----------------
    with torch.cuda.stream(stream):
        s = Solver(case.solid, theta_deg=case.theta_deg, theta_field=case.theta_field,
                   precision=args.precision, device=local, stream=stream, step_kernel=args.kernel,
                   step_chunk=args.chunk, **case.physical())
        for d in case.droplets:
            s.init_droplet(*d)
        s.step(args.warmup)
        s.check()
        step_kernel_used = s.step_kernel
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # the K-step region is repeated until it has run for at least 300 ms
        # (clock samples need that long); each repeat is bracketed by a
        # barrier and a synchronize, and the repeat count is the same on
        # every rank (from the slowest rank's first region)
        sampler = ClockSampler(local)
        sampler.start()
        sampler.wait_first()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)

        def region():
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e0.record(stream)
            s.step(args.steps)          # K launches of the fused step kernel
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        times = [region()]
        first = max_over_ranks(times[0], f"cuda:{local}", world)
        repeats = max(1, min(1000, int(math.ceil(300.0 / max(first, 1e-3)))))
        while len(times) < repeats:
            times.append(region())
        clocks = sampler.stop()
        ms = sum(times) / len(times)
        s.check()
    ms = max_over_ranks(ms, f"cuda:{local}", world)
    ms_per_step = ms / args.steps
    value = whole_job_mlups(world, N, args.steps, ms * 1e-3)

    peak, peak_kind = load_peaks()
    bpl = BYTES_PER_LU[args.precision]
    achieved = bpl * N / (ms_per_step * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        # DRAM bytes per launch from one ncu capture of the step kernel this
        # run used; null once the step sources differ from the captured ones
        try:
            t = json.load(open(tfile)).get(f"{args.workload}:{args.precision}:{step_kernel_used}")
            if t and t.get("step_source_sha256") == step_source_sha256():
                traffic = t["bytes_per_launch"]
        except Exception:
            traffic = None
    s.close()

    # ---------------- end to end through the C ABI with host buffers --------
    # inputs and outputs in pinned host memory, allocated before the timed region
    e2e_steps = args.e2e_steps
    solid_h = pinned(torch, case.solid.shape, np.uint8)
    solid_h[...] = case.solid
    theta_h = None
    if case.theta_field is not None:
        theta_h = pinned(torch, case.theta_field.shape, np.float32)
        theta_h[...] = case.theta_field
    # read-back in the solve's own precision class: float64 for FP64 solves,
    # float32 (pflbm_get_f32) for FP32 and 16-bit solves
    rb = np.float64 if args.precision == "fp64" else np.float32
    outs = (pinned(torch, (case.ny, case.nx), rb), pinned(torch, (case.ny, case.nx, 2), rb),
            pinned(torch, (case.ny, case.nx), rb))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        s2 = Solver(solid_h, theta_deg=case.theta_deg, theta_field=theta_h,
                    precision=args.precision, device=local, stream=stream, step_kernel=args.kernel,
                    step_chunk=args.chunk, **case.physical())
        for d in case.droplets:
            s2.init_droplet(*d)
        s2.step(e2e_steps)
        phi, u, p = s2.get(out=outs) if rb is np.float64 else s2.get_f32(out=outs)
        s2.close()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, f"cuda:{local}", world)
    h2d = case.solid.nbytes + (case.theta_field.nbytes if case.theta_field is not None else 0)
    d2h = phi.nbytes + u.nbytes + p.nbytes

    extra = None
    if rank == 0 and world == 1 and not args.no_extra and case.name == "many_flat" and args.precision == "fp32":
        extra = extra_block(args, torch, world, local, case, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups_cpu, cores, desc = oracle_baseline("2d", args.workload, 12.0)
        cpu = {"value": mlups_cpu, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16 storage, f32 arithmetic",
                      "fp16": "f16 storage, f32 arithmetic"}[args.precision], "data": "synthetic",
            "config": {"workload": case.name, "nx": case.nx, "ny": case.ny,
                       "droplets": len(case.droplets), "precision": args.precision,
                       "step_kernel": step_kernel_used,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state 1.2 GB > L2, no flush needed" if case.name == "many_flat"
                       else "small lattice: L2-resident"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_kind": peak_kind, "bytes_per_lu": bpl},
            "hbm_roofline_mlups": peak * 1e9 / bpl / 1e6,
            "e2e": {"value": whole_job_mlups(world, N, e2e_steps, e2e_s), "unit": "MLUPS",
                    "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                    "steps_per_solve": e2e_steps,
                    "includes": "create (mask upload, geometry), droplet init, steps, get (float64 for "
                                "FP64 solves, float32 otherwise)",
                    "host_buffers": "pinned"},
            "gpu_launches": args.steps,
            "timing": {"repeats": len(times), "note": "each repeat times exactly K steps, bracketed by a "
                       "barrier and synchronize; ms_per_step is the mean over repeats (max over ranks)",
                       "ms_per_repeat": [round(t, 4) for t in times[:50]]},
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        if extra is not None:
            line["extra"] = extra
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
