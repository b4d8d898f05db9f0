"""GPU parity of the three-dimensional path (D3Q19 f, D3Q7 g, 27-neighbour
ghost average) against the FP64 3D oracle, through the C ABI.

Bars: node classes bit-exact, a_v to rounding; phi within 1e-10 (FP64) and
1e-5 (FP32) after the stated steps; mass as the oracle's.
"""
import multiprocessing as mp

import numpy as np
import pytest

from tests import oracle_jobs as oj

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": dict(phi=1e-10, u=1e-12, p=1e-12, mass=1e-9), "fp32": dict(phi=1e-5, u=1e-6, p=1e-6, mass=1e-4)}
CASES = ["flat3d", "flat3d_two", "sphere3d", "tiny3d", "incline3d", "flat3d_nodgdt"]

_pool = None
_fut = {}


# the benchmark box (512 x 512 x 128, 64 droplets) compared on columns with
# oracle windows of the same input
FULL3 = dict(nx=512, ny=512, nz=128)
WIN3_STEPS, WIN3_HALF = 8, 18


def _win_centres():
    from paper_2312_00369_gb300 import workloads as wl
    c = wl.many_droplets_3d(**FULL3)
    return [(int(round(d[0] + 0.5 * d[3])) % 512, int(round(d[1])) % 512) for d in c.droplets[:4]]


@pytest.fixture(scope="module", autouse=True)
def oracle_pool():
    global _pool
    _pool = mp.get_context("spawn").Pool(processes=len(CASES) + 4)
    for name in CASES:
        _fut[name] = _pool.apply_async(oj.run3d_case, (name,))
    for xc, yc in _win_centres():
        _fut[("win3", xc, yc)] = _pool.apply_async(oj.window3d_run, (FULL3, xc, yc, WIN3_HALF, WIN3_STEPS))
    _fut["max3d"] = _pool.apply_async(oj.window3d_run, ("max3d", 507, 500, WIN3_HALF, 8))
    yield
    _pool.close()
    _pool.join()


def ref(name):
    return _fut[name].get(timeout=900)


def gpu_run(name, precision, path="fused", zc=0, steps=None):
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name(name)
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision=precision, step_path=path, fused_zc=zc,
                       dgdt_mode=c.meta.get("dgdt", 0), **c.physical())
    for d in c.droplets:
        s.init_droplet(*d)
    m0 = s.mass()
    s.step(c.steps if steps is None else steps)
    s.check()
    phi, u, p = s.get()
    g = s.geometry()
    out = dict(phi=phi, u=u, p=p, mass0=m0, mass=s.mass(), cls=g["cls"], av=g["av"])
    if c.wall:
        out["theta"], out["sphere"], out["npts"] = s.contact_angle(dict(dict(exclude=1.5 * c.W), **c.wall))
    s.close()
    return out


@pytest.mark.parametrize("name", CASES)
def test_geometry_3d(name):
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name(name)
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp64", **c.physical())
    g = s.geometry()
    s.close()
    r = ref(name)
    assert np.array_equal(g["cls"], r["cls"])
    assert np.max(np.abs(g["av"] - r["av"])) < 1e-15


@pytest.mark.parametrize("path", ["fused", "three_pass"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", CASES)
def test_parity_3d(name, precision, path):
    r = ref(name)
    g = gpu_run(name, precision, path)
    t = TOL[precision]
    zeta = r["cls"] <= 1
    dphi = np.max(np.abs(g["phi"] - r["phi"]))
    assert dphi <= t["phi"], dphi
    assert np.max(np.abs(g["u"] - r["u"])[zeta]) <= t["u"]
    assert np.max(np.abs(g["p"] - r["p"])[zeta]) <= t["p"]
    assert abs(g["mass0"] - r["mass0"]) <= t["mass"] and abs(g["mass"] - r["mass"]) <= t["mass"]
    # the droplet moved: the comparison is not of two initial states
    assert np.max(np.abs(r["u"])) > 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name,zc", [("flat3d", 1), ("flat3d", 0), ("flat3d", 100), ("sphere3d", 3),
                                     ("tiny3d", 2)])
def test_fused_equals_three_pass(name, zc, precision):
    # The two step paths inline the same arithmetic, with every multiply-add
    # explicit: they agree bit for bit, whatever the number of planes each
    # CTA of the fused path marches.
    a = gpu_run(name, precision, "three_pass", steps=40)
    b = gpu_run(name, precision, "fused", zc=zc, steps=40)
    for key in ("phi", "u", "p"):
        assert np.array_equal(a[key], b[key]), key
    assert a["mass"] == b["mass"]


@pytest.mark.parametrize("name", ["flat3d", "incline3d", "sphere3d"])
def test_contact_angle_3d(name):
    import oracle
    c = oj.case3d_by_name(name)
    g = gpu_run(name, "fp64")
    # the device fit against the oracle's fit of the same field (the point
    # order differs, so the FP64 sums agree to round-off)
    th, sph, n = oracle.contact_angle3(g["phi"], g["cls"], dict(dict(exclude=1.5 * c.W), **c.wall))
    assert n == g["npts"] and n >= 20
    assert abs(th - g["theta"]) < 1e-9 and np.allclose(sph, g["sphere"], rtol=0, atol=1e-9)
    # and against the oracle's own run: within 0.5 deg
    r = ref(name)
    assert abs(g["theta"] - r["theta"]) < 0.5


@pytest.mark.parametrize("path", ["auto", "fused"])
def test_full_size_box_sampled_columns(path):
    # the benchmark's box and launch configuration (FP32), columns through
    # the edge of four droplets compared with oracle windows of the same input
    from paper_2312_00369_gb300 import pflbm
    from paper_2312_00369_gb300 import workloads as wl
    c = wl.many_droplets_3d(**FULL3)
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp32", step_path=path, **c.physical())
    for d in c.droplets:
        s.init_droplet(*d)
    s.step(WIN3_STEPS)
    s.check()
    phi, u, p = s.get()
    s.close()
    for xc, yc in _win_centres():
        r = _fut[("win3", xc, yc)].get(timeout=900)
        assert r["phi"].max() > 0.9 and r["phi"].min() < 0.1    # the column crosses the interface
        assert np.max(np.abs(phi[:, yc, xc] - r["phi"])) <= 1e-5
        assert np.max(np.abs(u[:, yc, xc] - r["u"])) <= 1e-6
        assert np.max(np.abs(p[:, yc, xc] - r["p"])) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_3d(precision):
    # save after 25 steps, run 30 more; a fresh handle loaded from the
    # checkpoint runs the same 30 steps to the same state, bit for bit
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name("sphere3d")
    mk = lambda: pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision=precision, **c.physical())
    a = mk()
    for d in c.droplets:
        a.init_droplet(*d)
    a.step(25)
    blob = a.save()
    a.step(30)
    b = mk()
    b.load(blob)
    assert b.steps == 25
    b.step(30)
    for x, y in zip(a.get(), b.get()):
        assert np.array_equal(x, y)
    assert a.mass() == b.mass() and b.steps == 55
    # a checkpoint of another size, other parameters or another wall is refused
    s2, _ = __import__("paper_2312_00369_gb300.workloads", fromlist=["box3d"]).box3d(40, 20, 20)
    bump = c.solid.copy()
    bump[2, 3:6, 3:6] = 1
    others = [pflbm.Solver3D(s2, precision=precision),
              pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision=precision, **{**c.physical(), "tau_f": 0.9}),
              pflbm.Solver3D(c.solid, theta_deg=c.theta_deg + 1.0, precision=precision, **c.physical()),
              pflbm.Solver3D(bump, theta_deg=c.theta_deg, precision=precision, **c.physical())]
    for other in others:
        with pytest.raises(pflbm.PflbmError) as e:
            other.load(blob)
        assert e.value.code == pflbm.EINVAL
    for s in [a, b] + others:
        s.close()


def test_nan_stops_stepping_3d():
    # a NaN in the initial field trips the device status word; the next step
    # after the status has reached the host is refused with ENUMERIC
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name("flat3d")
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp32", **c.physical())
    phi = np.zeros((c.solid.shape))
    phi[10, 10, 20] = np.nan
    s.init_phi(phi)
    s.step(3)
    torch.cuda.synchronize()
    with pytest.raises(pflbm.PflbmError) as e:
        s.step(1)
    assert e.value.code == pflbm.ENUMERIC
    assert s.steps == 3
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_get_f32_is_get_rounded_3d(precision):
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name("sphere3d")
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision=precision, **c.physical())
    for d in c.droplets:
        s.init_droplet(*d)
    s.step(20)
    full = s.get()
    low = s.get_f32()
    s.close()
    for a, b in zip(full, low):
        assert b.dtype == np.float32 and np.array_equal(b, a.astype(np.float32))


def test_init_phi_and_edge_cases_3d():
    # a general initial field (init_phi) against the oracle; step(0) is a
    # no-op; a lattice without liquid stays exactly at rest
    import oracle
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name("incline3d")
    z, y, x = np.mgrid[0:c.shape[0], 0:c.shape[1], 0:c.shape[2]]
    phi0 = 0.5 + 0.5 * np.tanh(2 * (6.0 - np.sqrt((x - 17.3) ** 2 + (y - 9.6) ** 2 + (z - 15.1) ** 2)) / 4.0)
    phi0 = np.maximum(phi0, 0.5 + 0.5 * np.tanh((z - 33.0) / 2.0))      # plus a liquid layer near the top
    o = oracle.Oracle3D(c.solid, theta_deg=c.theta_deg, **c.physical())
    o.init_phi(phi0)
    o.step(60)
    r = o.get()
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp64", **c.physical())
    s.init_phi(phi0)
    before = s.get()
    s.step(0)
    assert s.steps == 0 and all(np.array_equal(a, b) for a, b in zip(before, s.get()))
    s.step(60)
    g = s.get()
    s.close()
    assert np.max(np.abs(g[0] - r[0])) <= 1e-10 and np.max(np.abs(g[1] - r[1])) <= 1e-12
    e = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp32", **c.physical())
    e.init_phi(np.zeros(c.shape))
    e.step(50)
    e.check()
    phi, u, p = e.get()
    assert np.all(phi == 0) and np.all(u == 0) and np.all(p == 0) and e.mass() == 0.0
    e.close()


def test_largest_accepted_box_3d():
    # 512 x 512 x 315 (26 * nz * ny * pitch just below 2^31): the highest
    # population indices; the column through the edge of a droplet hanging
    # from the top wall at the far corner against an oracle window
    from paper_2312_00369_gb300 import pflbm
    c = oj.max3d_case()
    s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp32", **c.physical())
    for d in c.droplets:
        s.init_droplet(*d)
    s.step(c.steps)
    s.check()
    phi, u, p = s.get_f32()
    s.close()
    r = _fut["max3d"].get(timeout=900)
    col = (slice(None), 500, 507)
    assert r["phi"][-20:].max() > 0.9 and r["phi"].min() < 0.1
    assert np.max(np.abs(phi[col] - r["phi"])) <= 1e-5
    assert np.max(np.abs(u[col] - r["u"])) <= 1e-6
    assert np.max(np.abs(p[col] - r["p"])) <= 1e-6


def test_rejects_bad_mask_3d():
    from paper_2312_00369_gb300 import pflbm
    s = np.zeros((12, 8, 8), np.uint8)
    with pytest.raises(pflbm.PflbmError):
        pflbm.Solver3D(s)


@pytest.mark.parametrize("path", ["three_pass", "fused"])
def test_allocator_choice_does_not_change_results_3d(path):
    # the default takes device memory from PyTorch's caching allocator; with
    # torch_memory=False the library calls cudaMalloc. Same state either way.
    from paper_2312_00369_gb300 import pflbm
    c = oj.case3d_by_name("sphere3d")
    outs = []
    for tm in (True, False):
        s = pflbm.Solver3D(c.solid, theta_deg=c.theta_deg, precision="fp32", step_path=path,
                           torch_memory=tm, **c.physical())
        for d in c.droplets:
            s.init_droplet(*d)
        s.step(40)
        s.check()
        outs.append(s.get() + (s.mass(),))
        s.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
