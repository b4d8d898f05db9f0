"""The other step kernels -- the staged kernel (populations brought to shared
memory by TMA, two tile shapes) and the two-node kernel (two x-adjacent
nodes per thread in packed FP32x2 arithmetic) -- against the global-load
kernel: the arithmetic is shared, so the fields must agree bit for bit after
any number of steps, for every storage precision that has these paths, every
geometry class (fluid-only tiles, walls, ghosts, bounce-back corners,
lattices narrower than a tile, ragged and odd widths) and in batches whose
lattices run with different tile shapes.
"""
import numpy as np
import pytest

from tests import oracle_jobs as oj

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = ["flat60_short", "incline45_ragged", "block", "tiny", "cylinder", "crop", "flat_visc_force", "flat_chi1",
         "incline_nodgdt", "odd_wide"]
KERNELS = [("staged32x8", 16), ("staged64x4", 16), ("staged32x8", 3), ("staged64x4", 1), ("pair", 0)]


def _solver(case, precision, kernel, chunk=0):
    from paper_2312_00369_gb300.pflbm import Solver
    s = Solver(case.solid, theta_deg=case.theta_deg, theta_field=case.theta_field, precision=precision,
               step_kernel=kernel, step_chunk=chunk, **case.physical(), **oj.solver_options(case))
    for d in case.droplets:
        s.init_droplet(*d)
    return s


def _state(s):
    phi, u, p = s.get()
    return phi, u, p, s.mass()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("name", CASES)
def test_staged_equals_global(name, precision):
    case = oj.case_by_name(name)
    steps = 37   # odd: both population copies serve as input
    ref = _solver(case, precision, "global")
    assert ref.step_kernel == "global"
    ref.step(steps)
    want = _state(ref)
    ref.close()
    for kernel, chunk in KERNELS:
        s = _solver(case, precision, kernel, chunk)
        assert s.step_kernel == kernel
        s.step(steps)
        got = _state(s)
        s.close()
        for a, b, what in zip(want, got, ("phi", "u", "p", "mass")):
            assert np.array_equal(a, b), (name, precision, kernel, chunk, what, np.max(np.abs(np.asarray(a) - b)))


def test_kernel_is_switchable_between_steps():
    from paper_2312_00369_gb300.pflbm import PflbmError, EINVAL
    case = oj.case_by_name("flat60_short")
    s = _solver(case, "fp32", "default")
    assert s.step_kernel == "global"
    s.step(10)
    s.set_step_kernel("staged32x8")
    s.step(10)
    s.set_step_kernel("staged64x4", 2)
    s.step(11)
    got = _state(s)
    r = _solver(case, "fp32", "global")
    r.step(31)
    want = _state(r)
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    f64 = _solver(case, "fp64", "default")
    assert f64.step_kernel == "global"
    with pytest.raises(PflbmError) as e:
        f64.set_step_kernel("staged32x8")
    assert e.value.code == EINVAL
    for x in (s, r, f64):
        x.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_staged_batch_with_mixed_shapes_equals_single(precision):
    # lattices of several sizes, the small ones with 64 x 4 tiles and short
    # items, the others with 32 x 8 tiles: each member equals its own
    # single-lattice run with the global-load kernel
    from paper_2312_00369_gb300 import pflbm, workloads as wl
    cases = wl.batched_instances(count=12, seed=7)
    classes = [(64 * 32, 1, 2), (128 * 64, 1, 5), (256 * 128, 0, 3)]
    stream = torch.cuda.Stream()
    members = []
    for c in cases:
        s = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, stream=stream, **c.physical())
        for d in c.droplets:
            s.init_droplet(*d)
        members.append(s)
    b = pflbm.Batch(members, pflbm.schedule(tiles_per_item=4, kernel=2, classes=classes))
    assert b.kernel == 2
    b.step(23)
    for c, s in zip(cases, members):
        r = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, step_kernel="global",
                         **c.physical())
        for d in c.droplets:
            r.init_droplet(*d)
        r.step(23)
        for x, y in zip(_state(r), _state(s)):
            assert np.array_equal(x, y), (c.nx, c.ny)
        r.close()
    b.close()
    for s in members:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_pair_batch_equals_single(precision):
    # the two-node batched kernel over a mix of lattice sizes and wall types
    # (flat, inclined, cylinder), one launch per size, the launches side by
    # side: each member equals its own single-lattice run with the
    # global-load kernel
    from paper_2312_00369_gb300 import pflbm, workloads as wl
    cases = wl.batched_instances(count=12, seed=11)
    stream = torch.cuda.Stream()
    members = []
    for c in cases:
        s = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, stream=stream, **c.physical())
        for d in c.droplets:
            s.init_droplet(*d)
        members.append(s)
    b = pflbm.Batch(members, pflbm.schedule(kernel=3))
    assert b.kernel == 3
    b.step(23)
    for c, s in zip(cases, members):
        r = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, step_kernel="global",
                         **c.physical())
        for d in c.droplets:
            r.init_droplet(*d)
        r.step(23)
        for x, y in zip(_state(r), _state(s)):
            assert np.array_equal(x, y), (c.nx, c.ny)
        r.close()
    b.close()
    for s in members:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pair_batch_groups_by_size_and_viscosity(precision):
    # the two-node batched kernel groups lattices by size and viscosity mode,
    # one launch per group of at most one launch's descriptor capacity: 300
    # lattices of one size (more than one launch holds), same-size lattices
    # with and without variable viscosity and a body force, and a lone size;
    # every member equals its own single-lattice run with the global-load kernel
    from paper_2312_00369_gb300 import pflbm, workloads as wl
    rng = np.random.default_rng(5)
    specs = [(64, 32, 0, 0.0)] * 300 + [(128, 64, 1, 0.0), (128, 64, 1, 0.3), (128, 64, 2, 0.3), (256, 128, 0, 0.0)]
    stream = torch.cuda.Stream()
    members, refs = [], []
    for i, (nx, ny, wt, nu) in enumerate(specs):
        c = wl.batch_instance(rng, nx, ny, wt, float(rng.uniform(30.0, 150.0)), 100)
        extra = dict(nu_l=nu, nu_g=nu / 6.0, gx=1e-6, gy=-2e-6) if nu else {}
        s = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, stream=stream, **c.physical(), **extra)
        for d in c.droplets:
            s.init_droplet(*d)
        members.append(s)
        if i % 50 == 0 or i >= 300:     # check a sample of the large group and every other member
            r = pflbm.Solver(c.solid, theta_deg=c.theta_deg, precision=precision, step_kernel="global",
                             **c.physical(), **extra)
            for d in c.droplets:
                r.init_droplet(*d)
            refs.append((i, r))
    b = pflbm.Batch(members, pflbm.schedule(kernel=3))
    assert b.kernel == 3 and b.info()["grid"] >= 5     # launches: the large group takes at least two
    b.step(17)
    for i, r in refs:
        r.step(17)
        for x, y in zip(_state(r), _state(members[i])):
            assert np.array_equal(x, y), specs[i]
        r.close()
    b.close()
    for s in members:
        s.close()


@pytest.mark.parametrize("precision,nx,ny,want", [
    ("fp32", 1024, 1023, "global"), ("fp32", 2048, 1024, "pair"),
    ("bf16", 1024, 511, "global"), ("bf16", 1024, 512, "pair"),
    ("fp16", 512, 512, "global"), ("fp16", 2048, 256, "pair"),
    ("fp64", 4096, 1024, "global")])
def test_default_kernel_by_lattice_size(precision, nx, ny, want):
    # the default step kernel: the two-node kernel from 2^19 nodes (16-bit
    # storage) and 2^21 nodes (FP32), else the one-node kernel
    from paper_2312_00369_gb300 import workloads as wl
    from paper_2312_00369_gb300.pflbm import Solver
    solid, _ = wl.flat_channel(nx, ny)
    s = Solver(solid, theta_deg=60.0, precision=precision)
    assert s.step_kernel == want
    s.set_step_kernel("default")
    assert s.step_kernel == want
    s.close()
