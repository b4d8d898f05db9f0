"""Continuous-batching request server for droplet-spreading solves.

Requests (grid size, wall type, contact angle, step count) arrive over time.
The server keeps every admitted solve resident on the device and admits
queued requests, first come first served, as soon as their HBM footprint
(``pflbm_footprint_bytes``) fits the budget and a slot is free. All resident
solves advance together in ticks of up to ``tick`` steps: one persistent
launch per step over every resident lattice (``pflbm_batch_t``), so requests
that arrive while others run share the device with them. A solve whose
remaining steps are fewer than a tick takes exactly those steps on its own
and finishes in that tick. Finished solves are read back (FP64 contact-angle
fit and mass on the device), their memory is released, and the latency
(finish - arrival) is recorded.

``PlainServer`` is the comparison path: the same admission and ticks, but
FP32 storage and one launch per solve per step.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import pflbm, workloads


@dataclass
class Request:
    rid: int
    t_arrival: float          # seconds after the stream starts
    nx: int
    ny: int
    wall_type: int
    theta: float
    steps: int


@dataclass
class Result:
    rid: int
    t_arrival: float
    t_admit: float
    t_done: float
    steps: int
    nodes: int
    theta_fit: float
    npoints: int
    mass: float
    failed: bool = False      # the solve reported a NaN or |u| >= 0.3

    @property
    def latency(self):
        return self.t_done - self.t_arrival


@dataclass
class _Slot:
    req: Request
    case: workloads.Case
    solver: pflbm.Solver
    left: int
    t_admit: float


def requests_from_stream(stream_dicts):
    return [Request(i, d["t"], d["nx"], d["ny"], d["wall_type"], d["theta"], d["steps"])
            for i, d in enumerate(stream_dicts)]


def case_of(req: Request) -> workloads.Case:
    return workloads.batch_instance(None, req.nx, req.ny, req.wall_type, req.theta, req.steps)


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    admitted: int = 0
    offered: int = 0
    wall_s: float = 0.0
    ticks: int = 0
    peak_slots: int = 0
    peak_bytes: int = 0
    processed_lu: int = 0     # lattice updates done, finished or not

    def summary(self):
        ok = [r for r in self.results if not r.failed]
        lat = np.array([r.latency for r in ok]) if ok else np.array([np.nan])
        lu = sum(r.nodes * r.steps for r in ok)
        return {
            "offered": self.offered, "admitted": self.admitted, "completed": len(ok),
            "failed": len(self.results) - len(ok),
            "queued_at_end": self.offered - self.admitted,
            "in_flight_at_end": self.admitted - len(self.results),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)),
            "completed_mlups": lu / self.wall_s / 1e6 if self.wall_s > 0 else 0.0,
            "processed_mlups": self.processed_lu / self.wall_s / 1e6 if self.wall_s > 0 else 0.0,
            "wall_s": self.wall_s, "ticks": self.ticks, "peak_slots": self.peak_slots,
            "peak_bytes": self.peak_bytes,
        }


class Server:
    """Continuous batching over resident solves (see the module docstring).
    ``precision``: storage of the resident solves; FP16 (scaled) by default,
    as fast as BF16 and about 100x closer to FP64 in phi. ``dgdt_mode`` as in
    pflbm_params_t (1 omits the (1/2) dG/dt term, stable for long solves)."""

    batched = True

    def __init__(self, precision="fp16", hbm_budget=32 << 30, max_slots=512, tick=200,
                 schedule=None, device=None, exclude_w=1.5, dgdt_mode=0):
        import torch
        self.torch = torch
        self.precision = precision
        self.budget = int(hbm_budget)
        self.max_slots = int(max_slots)
        self.tick = int(tick)
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = torch.cuda.Stream(device=self.device)
        self.schedule = schedule
        self.exclude_w = exclude_w
        self.slots: list[_Slot] = []
        self.used = 0
        self.batch = None
        self.processed_lu = 0
        self.dgdt_mode = dgdt_mode

    # -- admission ---------------------------------------------------------
    def footprint(self, req):
        return pflbm.pflbm_footprint_bytes(req.nx, req.ny, self.precision)

    def fits(self, req):
        return len(self.slots) < self.max_slots and self.used + self.footprint(req) <= self.budget

    def admit(self, req, now):
        case = case_of(req)
        with self.torch.cuda.stream(self.stream):
            s = pflbm.Solver(case.solid, theta_deg=case.theta_deg, precision=self.precision,
                             device=self.device, stream=self.stream, dgdt_mode=self.dgdt_mode,
                             **case.physical())
            for d in case.droplets:
                s.init_droplet(*d)
        self.slots.append(_Slot(req, case, s, req.steps, now))
        self.used += self.footprint(req)

    # -- one tick ----------------------------------------------------------
    def _advance(self, full, short):
        """Advance `full` slots by one tick together, `short` slots by their
        remaining steps."""
        if full:
            solvers = [sl.solver for sl in full]
            if self.batch is None:
                self.batch = pflbm.Batch(solvers, self.schedule if self.schedule is not None
                                         else pflbm.schedule())
            else:
                self.batch.set(solvers)
            self.batch.step(self.tick)
        for sl in short:
            sl.solver.step(sl.left)

    def _finish(self, sl, now_fn, failed):
        if failed:
            th, npts, m = float("nan"), 0, float("nan")
        else:
            w = dict(sl.case.wall, exclude=self.exclude_w * sl.case.W)
            try:
                th, _, npts = sl.solver.contact_angle(w)
            except pflbm.PflbmError:
                th, npts = float("nan"), 0
            m = sl.solver.mass()          # synchronises the stream
        res = Result(sl.req.rid, sl.req.t_arrival, sl.t_admit, now_fn(), sl.req.steps,
                     sl.req.nx * sl.req.ny, th, npts, m, failed)
        sl.solver.close()
        self.used -= self.footprint(sl.req)
        return res

    def _evict_failed(self, now_fn, out):
        failed = [sl for sl in self.slots if sl.solver.status() == pflbm.ENUMERIC]
        for sl in failed:
            out.append(self._finish(sl, now_fn, True))
        self.slots = [sl for sl in self.slots if sl not in failed]

    def step_tick(self, now_fn):
        with self.torch.cuda.nvtx.range(f"serve tick ({len(self.slots)} solves)"):
            return self._step_tick(now_fn)

    def _step_tick(self, now_fn):
        out = []
        # solves that reported a NaN or |u| >= 0.3 leave as failed requests
        # (the flag is read without waiting; a refused step did no work)
        self._evict_failed(now_fn, out)
        for _ in range(3):
            full = [sl for sl in self.slots if sl.left >= self.tick]
            try:
                self._advance(full, [])
                break
            except pflbm.PflbmError as e:
                if e.code != pflbm.ENUMERIC:
                    raise
                self._evict_failed(now_fn, out)
        else:
            full = []
        for sl in full:
            sl.left -= self.tick
            self.processed_lu += self.tick * sl.req.nx * sl.req.ny
        for sl in [sl for sl in self.slots if 0 < sl.left < self.tick]:
            try:
                self._advance([], [sl])
                self.processed_lu += sl.left * sl.req.nx * sl.req.ny
                sl.left = 0
            except pflbm.PflbmError as e:
                if e.code != pflbm.ENUMERIC:
                    raise
                sl.left = -1          # finished as failed below
        for sl in [sl for sl in self.slots if sl.left <= 0]:
            st = sl.solver.status(wait=True)
            out.append(self._finish(sl, now_fn, sl.left < 0 or st == pflbm.ENUMERIC))
        self.slots = [sl for sl in self.slots if sl.left > 0]
        return out

    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        for sl in self.slots:
            sl.solver.close()
        self.slots = []

    # -- the loop ------------------------------------------------------------
    def run(self, requests, duration=None, drain=False, max_wall=None):
        """Serve `requests` (sorted by arrival) against the wall clock.
        Stops accepting arrivals after `duration` seconds; with drain=True
        it then finishes the admitted work; max_wall bounds the whole run."""
        stats = ServeStats()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        queue = []
        nxt = 0
        horizon = duration if duration is not None else math.inf
        while True:
            t = now()
            if max_wall is not None and t >= max_wall:
                break
            while nxt < len(requests) and requests[nxt].t_arrival <= min(t, horizon):
                queue.append(requests[nxt])
                nxt += 1
                stats.offered += 1
            while queue and self.fits(queue[0]):
                self.admit(queue.pop(0), now())
                stats.admitted += 1
            stats.peak_slots = max(stats.peak_slots, len(self.slots))
            stats.peak_bytes = max(stats.peak_bytes, self.used)
            if self.slots:
                stats.results.extend(self.step_tick(now))
                stats.ticks += 1
            else:
                if t >= horizon or nxt >= len(requests):
                    if not queue:
                        break
                # idle until the next arrival
                if nxt < len(requests):
                    wait = requests[nxt].t_arrival - now()
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
            if t >= horizon and not drain:
                break
            if t >= horizon and drain and not self.slots and not queue:
                break
        self.torch.cuda.synchronize()
        stats.wall_s = now()
        stats.processed_lu = self.processed_lu
        return stats


class PlainServer(Server):
    """Comparison path: FP32 storage, one launch per solve per step."""

    batched = False

    def __init__(self, **kw):
        kw = dict(kw)
        kw["precision"] = "fp32"
        super().__init__(**kw)

    def _advance(self, full, short):
        # each solve's steps are issued back to back by the library, one
        # launch per step, without Python in between
        for sl in full:
            sl.solver.step(self.tick)
        for sl in short:
            sl.solver.step(sl.left)
