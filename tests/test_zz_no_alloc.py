"""The allocation-free FP64 mass reduction (pflbm_phi_mass_noalloc).

Some callers cannot allocate device memory at all (a component inside a
framework whose pool owns the device, or a loop in which cudaMalloc's
possible device synchronisation is not allowed). For them the library offers
one entry point whose scratch is a static device array. This file checks it
against pflbm_mass on the same state, on two calls in a row (the static array
keeps the previous call's contents), and checks that sizes beyond the static
limit are refused. It is collected last so that a failure here does not stop
the rest of the suite.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(precision):
    from paper_2312_00369_gb300 import workloads as wl
    from paper_2312_00369_gb300.pflbm import Solver
    case = wl.droplet_on_flat_wall(nx=100, ny=50, R=20.0, theta=60.0)
    s = Solver(case.solid, theta_deg=case.theta_deg, precision=precision, device=0,
               **case.physical())
    s.init_droplet(*case.droplets[0])
    s.step(300)
    return s


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_noalloc_mass_matches_pflbm_mass(precision, rtol):
    from paper_2312_00369_gb300.pflbm import pflbm_phi_mass_noalloc
    s = _state(precision)
    expect = s.mass()                                    # the existing entry point
    dev = torch.device("cuda", 0)
    phi = torch.empty((s.ny, s.nx), dtype=torch.float64, device=dev)
    s.get_device(phi=phi)
    cls = s.geometry()["cls"]
    zeta = torch.from_numpy((cls <= 1).astype(np.uint8)).to(dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = s.stream.cuda_stream
    torch.cuda.synchronize()
    for call in range(2):                                # two calls in a row
        pflbm_phi_mass_noalloc(phi.data_ptr(), zeta.data_ptr(), s.nx, s.ny,
                               out.data_ptr() + 8 * call, stream)
        torch.cuda.synchronize()
        got = float(out[call].item())
        assert abs(got - expect) <= rtol * abs(expect), (call, got, expect)
    s.close()


def test_noalloc_mass_without_mask_and_limit():
    from paper_2312_00369_gb300.pflbm import PflbmError, EINVAL, pflbm_phi_mass_noalloc
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    host = rng.random((517, 333))                         # several blocks, ragged tail
    phi = torch.from_numpy(host).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(2):
        pflbm_phi_mass_noalloc(phi.data_ptr(), None, 333, 517, out.data_ptr(), None)
        torch.cuda.synchronize()
        assert abs(float(out.item()) - host.sum()) <= 1e-12 * host.sum()
    with pytest.raises(PflbmError) as e:                 # refused before any launch
        pflbm_phi_mass_noalloc(phi.data_ptr(), None, 8193, 4096, out.data_ptr(), None)
    assert e.value.code == EINVAL and "static scratch" in str(e.value)
