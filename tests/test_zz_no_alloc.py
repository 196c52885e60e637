"""m2m_observe_static: observables computed with static device scratch, no allocation.

Some callers cannot allocate device memory (they run inside another runtime's
memory pool, or under a no-allocation policy after start-up). For them the library
offers m2m_observe_static, which keeps its scratch in a static device array. This
file runs last: it checks, through the C ABI, that two calls in a row give the
same raw observables as the allocating path (create a context, load the particles
from device memory, read the raw observables), within the FP64 tolerance of the
parity tests, on annuli and on a pixel map with Gauss-Hermite kinds; that the
result is the oracle's y_j = sum_i w_i K_j(z_i); and that sets the call cannot take
are rejected with M2M_ERR_ARG.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W
from paper_1202_2355_gb300.workloads import Group

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def _rel_err(a, b):
    scale = np.maximum(np.abs(b), 1e-12 * np.max(np.abs(b)))
    return float(np.max(np.abs(a - b) / scale))


def _device_particles(torch, m):
    pos = torch.tensor(np.concatenate([m["x"], m["y"], m["z"]]), device="cuda")
    vel = torch.tensor(np.concatenate([m["vx"], m["vy"], m["vz"]]), device="cuda")
    w = torch.tensor(m["w"], device="cuda")
    torch.cuda.synchronize()
    return pos, vel, w


def _allocating_path(wl, Y, sig, Vp, sp, pos, vel, w):
    ref = B.fit_from_workload(wl, Y, sig, Vp, sp, precision="fp64")
    ref.load_device(wl.n, pos.data_ptr(), vel.data_ptr(), w.data_ptr())
    y_ref = ref.observables()[1]
    ref.close()
    return y_ref


def _static_twice(torch, wl, Vp, sp, pos, vel, w):
    out = []
    for _ in range(2):
        y = torch.full((wl.J,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        J = B.observe_static(wl.groups, wl.incl_deg, wl.n, pos.data_ptr(), vel.data_ptr(), w.data_ptr(),
                             y.data_ptr(), Vp=Vp, sp=sp)
        assert J == wl.J
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got))
        out.append(got)
    return out


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()
    return t


def test_static_observe_matches_allocating_path_twice(torch):
    wl = W.make("c2", n=50_000, n_target=100_000)
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    pos, vel, w = _device_particles(torch, wl.model)
    y_ref = _allocating_path(wl, Y, sig, Vp, sp, pos, vel, w)
    for got in _static_twice(torch, wl, Vp, sp, pos, vel, w):
        assert _rel_err(got, y_ref) < TOL
    # and the oracle's plain sum over particles and kernels, on the error scale of the fit
    obs = O.ObsSet(wl.groups, wl.incl_deg, Vp=Vp, sp=sp)
    y_ora = O.observe(obs, O.ParticleSet(wl.model))
    assert np.max(np.abs(got - y_ora) / np.maximum(np.abs(y_ora), sig)) < TOL


def test_static_observe_pixel_map_with_gauss_hermite_kinds(torch):
    """A 16 x 16 map of surface mass and h1..h4 seen at 60 degrees: the pixel-area
    normalisation and 1/sigma_p of the pixel path."""
    wl = W.make("c4", n=40_000, n_target=300_000)
    wl.groups = [Group("pixels", ["mass", "gh1", "gh2", "gh3", "gh4"], [0.02] * 5, nx=16, ny=16,
                       box=(-2.0, 2.0, -2.0, 2.0))]
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), None)
    wl.target = None
    pos, vel, w = _device_particles(torch, wl.model)
    y_ref = _allocating_path(wl, Y, sig, Vp, sp, pos, vel, w)
    for got in _static_twice(torch, wl, Vp, sp, pos, vel, w):
        assert _rel_err(got, y_ref) < TOL
    obs = O.ObsSet(wl.groups, wl.incl_deg, Vp=Vp, sp=sp)
    y_ora = O.observe(obs, O.ParticleSet(wl.model))
    # cancelling Gauss-Hermite sums in sparse pixels: the rounding scale of the sum
    kmax = np.concatenate([np.full(256, 1.0 / (0.25 * 0.25))] + [np.full(256, 1.5)] * 4)
    scale = np.maximum(np.maximum(np.abs(y_ora), sig), 1e-3 * kmax * wl.model["w"][0])
    assert np.max(np.abs(got - y_ora) / scale) < TOL


def test_static_observe_rejects_oversized_sets(torch):
    big = [Group("pixels", ["mass", "gh1", "gh2"], [0.02] * 3, nx=64, ny=64, box=(-4.0, 4.0, -4.0, 4.0))]
    y = torch.zeros(3 * 4096, dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(B.M2MError) as ei:
        B.observe_static(big, 0.0, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), y.data_ptr(),
                         Vp=np.zeros(4096), sp=np.ones(4096))
    assert ei.value.status == 1


def test_static_observe_rejects_shells_and_gauss_hermite_without_vp_sp(torch):
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    shells = [Group("shells", ["alm_0_0"], [1.0], edges=np.exp(np.linspace(math.log(0.1), math.log(5.0), 8)))]
    with pytest.raises(B.M2MError) as ei:
        B.observe_static(shells, 0.0, 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), y.data_ptr())
    assert ei.value.status == 1
    # a Gauss-Hermite kind with no V_p, sigma_p pointers in the descriptor
    gh = [Group("annuli", ["gh3"], [0.01], edges=np.exp(np.linspace(math.log(0.1), math.log(5.0), 9)))]
    d = B.ObsDesc(gh, 0.0)
    d.o.groups[0].Vp = None
    d.o.groups[0].sp = None
    st = B.lib().m2m_observe_static(B.C.byref(d.o), 1, x.data_ptr(), x.data_ptr(), x.data_ptr(), y.data_ptr(),
                                    None)
    assert st == 1
    assert "Vp and sp" in B.lib().m2m_last_error(None).decode()
