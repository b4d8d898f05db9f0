"""Host-side pieces of the request generator and the serving statistics."""
import numpy as np

from paper_2312_00369_gb300 import workloads as wl
from paper_2312_00369_gb300.serve import Result, ServeStats, requests_from_stream


def test_request_stream_statistics():
    reqs = wl.request_stream(rate=2000.0, duration=2.0, seed=2024)
    assert 3600 < len(reqs) < 4400                          # Poisson, mean 4000
    ts = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(ts) >= 0) and ts[-1] < 2.0
    nx = np.array([r["nx"] for r in reqs])
    assert np.all(nx % 16 == 0) and nx.min() >= 128 and nx.max() <= 1024
    assert all(r["ny"] * 2 == r["nx"] for r in reqs)
    st = np.array([r["steps"] for r in reqs])
    assert st.min() >= 1000 and st.max() <= 20000
    # log-uniform sizes: the median sits near sqrt(128 * 1024) = 362
    assert 300 < np.median(nx) < 430
    again = wl.request_stream(rate=2000.0, duration=2.0, seed=2024)
    assert again == reqs                                    # seeded


def test_serve_stats_summary():
    st = ServeStats(offered=5, admitted=4, wall_s=2.0)
    for i, lat in enumerate([1.0, 2.0, 3.0]):
        st.results.append(Result(i, 0.0, 0.0, lat, 100, 1000, 60.0, 20, 1.0))
    s = st.summary()
    assert s["completed"] == 3 and s["queued_at_end"] == 1 and s["in_flight_at_end"] == 1
    assert s["p50_s"] == 2.0 and abs(s["p99_s"] - 2.98) < 1e-9
    assert abs(s["completed_mlups"] - 3 * 100 * 1000 / 2.0 / 1e6) < 1e-12
    reqs = requests_from_stream([dict(t=0.1, nx=128, ny=64, wall_type=1, theta=50.0, steps=10)])
    assert reqs[0].rid == 0 and reqs[0].nx == 128


def test_batched_instances_mix():
    cases = wl.batched_instances(256, seed=369, steps=5000)
    assert len(cases) == 256
    sizes = {(c.nx, c.ny) for c in cases}
    assert sizes <= set(wl.BATCH_SIZES)
    names = {c.name for c in cases}
    assert names == {"flat", "incline", "cylinder"}
    for c in cases[:20]:
        assert c.solid[:2].all() and c.solid[-2:].all()
        assert 30.0 <= c.theta_deg <= 150.0
