"""Batched lattices (one persistent launch per step, CUDA-graph replay).

Each lattice's result must be the same alone and in the mix: the batched
kernel runs the very same per-tile code, so the fields are compared bit for
bit. A member stepped on its own between batched steps, odd step counts and
membership changes must keep that property. One member is also checked
against the FP64 oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mix(seed=5, n=9):
    from paper_2312_00369_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    sizes = [(64, 32), (128, 64), (96, 48), (256, 128), (100, 50)]
    out = []
    for i in range(n):
        nx, ny = sizes[i % len(sizes)]
        out.append(wl.batch_instance(rng, nx, ny, i % 3, float(rng.uniform(30, 150)), 200))
    return out


def make(cases, precision, stream):
    from paper_2312_00369_gb300.pflbm import Solver
    out = []
    for c in cases:
        s = Solver(c.solid, theta_deg=c.theta_deg, precision=precision, stream=stream, **c.physical())
        for d in c.droplets:
            s.init_droplet(*d)
        out.append(s)
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp64"])
@pytest.mark.parametrize("sched", [dict(tiles_per_item=1, order=0, use_graph=1),
                                   dict(tiles_per_item=4, order=1, use_graph=0, ctas_per_sm=2)])
def test_batch_equals_alone_bitwise(precision, sched):
    from paper_2312_00369_gb300.pflbm import Batch, schedule
    cases = mix()
    stream = torch.cuda.Stream()
    alone = make(cases, precision, stream)
    for s in alone:
        s.step(37)
    together = make(cases, precision, stream)
    b = Batch(together, schedule(**sched))
    b.step(37)
    for a, t in zip(alone, together):
        pa, ua, qa = a.get()
        pt, ut, qt = t.get()
        assert np.array_equal(pa, pt) and np.array_equal(ua, ut) and np.array_equal(qa, qt)
    b.close()


def test_batch_phase_membership_and_individual_steps():
    from paper_2312_00369_gb300.pflbm import Batch
    cases = mix(seed=9, n=5)
    stream = torch.cuda.Stream()
    ref = make(cases, "fp32", stream)
    runs = make(cases, "fp32", stream)
    b = Batch(runs)
    b.step(3)                       # odd: the batch phase flips
    runs[2].step(1)                 # a member moves on its own
    b.step(2)
    b.set([runs[0], runs[2], runs[4]])
    b.step(5)
    counts = [10, 5, 11, 5, 10]
    for s, n in zip(ref, counts):
        s.step(n)
    for s, r, n in zip(runs, ref, counts):
        assert s.steps == n
        assert np.array_equal(s.get()[0], r.get()[0])
    b.close()


def test_batch_member_matches_oracle():
    import oracle
    from paper_2312_00369_gb300.pflbm import Batch
    cases = mix(seed=3, n=4)
    stream = torch.cuda.Stream()
    runs = make(cases, "fp32", stream)
    b = Batch(runs)
    b.step(150)
    for c, s in zip(cases[:2], runs[:2]):
        o = oracle.Oracle(c.solid, theta_deg=c.theta_deg, **c.physical())
        for d in c.droplets:
            o.init_droplet(*d)
        o.step(150)
        assert np.max(np.abs(s.get()[0] - o.get()[0])) <= 1e-5
    b.close()


def test_autotune_picks_a_measured_schedule(tmp_path, monkeypatch):
    from paper_2312_00369_gb300 import autotune
    monkeypatch.setenv("PFLBM_TUNE_CACHE", str(tmp_path / "sched.json"))
    cases = mix(seed=1, n=6)
    cands = [dict(ctas_per_sm=0, tiles_per_item=1, order=0, use_graph=1),
             dict(ctas_per_sm=2, tiles_per_item=2, order=1, use_graph=1)]
    best, timings = autotune.tune(cases, "bf16", steps=4, warmup=2, candidates=cands)
    assert best in cands and len(timings) == 2 and all(t > 0 for t in timings.values())
    again, _ = autotune.tune(cases, "bf16", candidates=cands)      # served from the cache
    assert again == best
