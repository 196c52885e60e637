"""m2m_observe_static: observables computed with static device scratch, no allocation.

Some callers cannot allocate device memory (they run inside another runtime's
memory pool, or under a no-allocation policy after start-up). For them the library
offers m2m_observe_static, which keeps its scratch in a static device array. This
file runs last: it checks, through the C ABI, that two calls in a row give the
same raw observables as the allocating path (create a context, load the particles
from device memory, read the raw observables), within the FP64 tolerance of the
parity tests.
"""
import numpy as np
import pytest

from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _rel_err(a, b):
    scale = np.maximum(np.abs(b), 1e-12 * np.max(np.abs(b)))
    return float(np.max(np.abs(a - b) / scale))


def test_static_observe_matches_allocating_path_twice():
    torch = pytest.importorskip("torch")
    from paper_1202_2355_gb300 import build
    build.build()
    wl = W.make("c2", n=50_000, n_target=100_000)
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    m = wl.model
    pos = torch.tensor(np.concatenate([m["x"], m["y"], m["z"]]), device="cuda")
    vel = torch.tensor(np.concatenate([m["vx"], m["vy"], m["vz"]]), device="cuda")
    w = torch.tensor(m["w"], device="cuda")
    torch.cuda.synchronize()

    ref = B.fit_from_workload(wl, Y, sig, Vp, sp, precision="fp64")
    ref.load_device(wl.n, pos.data_ptr(), vel.data_ptr(), w.data_ptr())
    y_ref = ref.observables()[1]
    ref.close()

    for _ in range(2):
        y = torch.full((wl.J,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        J = B.observe_static(wl.groups, wl.incl_deg, wl.n, pos.data_ptr(), vel.data_ptr(), w.data_ptr(),
                             y.data_ptr(), Vp=Vp, sp=sp)
        assert J == wl.J
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel_err(got, y_ref) < TOL


def test_static_observe_rejects_oversized_sets():
    torch = pytest.importorskip("torch")
    from paper_1202_2355_gb300.workloads import Group
    big = [Group("pixels", ["mass", "gh1", "gh2"], [0.02] * 3, nx=64, ny=64, box=(-4.0, 4.0, -4.0, 4.0))]
    y = torch.zeros(3 * 4096, dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(B.M2MError) as ei:
        B.observe_static(big, 0.0, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), y.data_ptr(),
                         Vp=np.zeros(4096), sp=np.ones(4096))
    assert ei.value.status == 1
