"""Diagnostics on the GPU (Sec. 4.1: intrinsic kinematics in spherical bins, Delta_grid;
Sec. 5, Fig. res: weight rms in the (E, x) cells) against the oracle on the same particles.

The device sums are exact integer sums in a two-word fixed point, so they are
bit-reproducible whatever the order of the particles, and they match the oracle's ordered
FP64 sums to rounding: counts exactly, sums within 1e-12 of the column scale. The host
arithmetic (moments, Delta_kin, Delta_grid, rms) matches the oracle's to 1e-13."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KG = dict(n_r=21, n_phi=12, n_ct=21, r_min=0.01, r_max=50.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


def _fit(wl, precision, prior=None):
    obs, Y, sig = O.from_workload(wl)
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision=precision, prior=prior)
    f.load(wl.model)
    return f


def _pulled(f):
    """The fit's current particles as the oracle sees them (FP64 copies of the state)."""
    pos, vel = f.state()
    return dict(x=pos[0], y=pos[1], z=pos[2], vx=vel[0], vy=vel[1], vz=vel[2], w=f.weights())


def _assert_sums_close(s_gpu, s_ora, rel=1e-12):
    scale = np.abs(s_ora).max(axis=0) + 1e-300
    assert np.all(np.abs(s_gpu - s_ora) <= rel * scale), np.abs(s_gpu - s_ora).max(axis=0) / scale


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kinematics_of_the_fit_match_oracle(precision):
    wl = W.make("c1", n=20_000)
    f = _fit(wl, precision)
    f.step(30)
    s, c = f.diag_kinematics(KG)
    so, co = O.kin_sums(KG, O.ParticleSet(_pulled(f)))
    f.close()
    assert np.array_equal(c, co) and c.sum() > 19_000
    _assert_sums_close(s, so)


def test_kinematics_of_host_particles_match_oracle():
    """A rotating, flattened target realisation passed from the host: the v_phi streaming
    shows in the bins, and every sum matches the oracle."""
    tg = W.make("c4", n=1000, n_target=100_000).target
    f = _fit(W.make("c1", n=100_000), "mixed")
    s, c = f.diag_kinematics(KG, particles=tg)
    so, co = O.kin_sums(KG, O.ParticleSet(tg))
    assert np.array_equal(c, co) and c.sum() == 100_000 - np.sum(
        np.sqrt(tg["x"] ** 2 + tg["y"] ** 2 + tg["z"] ** 2) >= 50.0)
    _assert_sums_close(s, so)
    mean, disp, valid = B.kin_moments(s, c, 30)
    mo, do, vo = O.kin_moments(so, co, 30)
    assert np.array_equal(valid, vo)
    assert np.allclose(mean, mo, rtol=1e-9, atol=1e-12) and np.allclose(disp, do, rtol=1e-9, atol=1e-12)
    # the target rotates: mass-weighted mean v_phi > 0
    assert np.sum(s[:, 3]) > 0.1 * np.sum(s[:, 0]) * 0.3
    # a non-rotating model against the target
    sm, cm = f.diag_kinematics(KG)
    out, used = B.delta_kin(sm, cm, s, c, 30)
    oo, uo = O.delta_kin(O.kin_sums(KG, O.ParticleSet(_pulled(f)))[0], cm, so, co, 30)
    f.close()
    assert used == uo > 50
    assert np.allclose(out, oo, rtol=1e-9)
    assert out[2] > 0.05  # the missing rotation dominates the mean-velocity differences


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_weights_of_the_fit_match_oracle(precision):
    wl = W.make("c1", n=20_000)
    f = _fit(wl, precision)
    f.step(30)
    ws, wd, cnt = f.diag_grid()
    p = _pulled(f)
    wso, wdo, co = O.grid_weights(wl.potential, wl.prior, O.ParticleSet(p))
    f.close()
    assert np.array_equal(cnt, co)
    assert np.all(np.abs(ws - wso) <= 1e-12 * wso.sum())
    # deviations about the cell means: the means differ by rounding between the two sums
    mean = np.where(co > 0, wso / np.maximum(co, 1), 0)
    tol = 1e-10 * wdo + co * (1e-13 * mean) ** 2 + 1e-13 * np.sqrt(np.maximum(wdo, 0) * co) * mean
    assert np.all(np.abs(wd - wdo) <= tol + 1e-300)
    rms, rmso = B.weight_rms(wd, cnt, 50), O.weight_rms(wdo, co, 50)
    assert rms == pytest.approx(rmso, rel=1e-9) and rms > 0


def test_delta_grid_of_a_gwr_fit_against_the_target():
    """A GWR fit has no grid of its own: the caller passes one. The model's and the
    target's cell weights, and Delta_grid, match the oracle."""
    wl = W.make("c1", n=20_000, n_target=100_000)
    grid = dict(wl.prior)
    obs, Y, sig = O.from_workload(wl)
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="fp64", prior=dict(wl.prior, mode="gwr"))
    f.load(wl.model)
    f.step(40)
    with pytest.raises(B.M2MError, match="GWR fit has no"):
        f.diag_grid()
    wm, _, cm = f.diag_grid(grid)
    wt, _, ct = f.diag_grid(grid, particles=wl.target)
    wmo, _, cmo = O.grid_weights(wl.potential, grid, O.ParticleSet(_pulled(f)))
    wto, _, cto = O.grid_weights(wl.potential, grid, O.ParticleSet(wl.target))
    f.close()
    assert np.array_equal(cm, cmo) and np.array_equal(ct, cto)
    assert np.allclose(wm, wmo, rtol=1e-12, atol=1e-15) and np.allclose(wt, wto, rtol=1e-12, atol=1e-15)
    d, do = B.delta_grid(wm, wt), O.delta_grid(wmo, wto)
    assert d == pytest.approx(do, rel=1e-10)
    # model and target are different realisations of the same sphere: a few percent
    assert 0.0 < d < 0.5


def test_full_size_c2_diagnostics_match_oracle():
    """1M particles of the radially biased C2 model after 20 steps (FP64)."""
    wl = W.make("c2", n_target=200_000)
    f = _fit(wl, "fp64")
    f.step(20)
    p = _pulled(f)
    s, c = f.diag_kinematics(KG)
    so, co = O.kin_sums(KG, O.ParticleSet(p))
    assert np.array_equal(c, co)
    _assert_sums_close(s, so)
    ws, wd, cnt = f.diag_grid()
    wso, wdo, cno = O.grid_weights(wl.potential, wl.prior, O.ParticleSet(p))
    f.close()
    assert np.array_equal(cnt, cno)
    assert np.all(np.abs(ws - wso) <= 1e-12 * wso.sum())
    # the radial bias shows: sigma_r > sigma_theta over the well-populated bins
    mean, disp, valid = B.kin_moments(s, c, 200)
    assert valid.sum() > 100
    assert np.median(disp[valid, 0] / disp[valid, 1]) > 1.3


def test_diagnostic_sums_do_not_depend_on_particle_order():
    """The same particles in reversed and in shuffled order give bit-identical sums (FP64
    atomics would differ in the last bits when the order of the additions changes)."""
    wl = W.make("c2", n=300_000, n_target=100_000)
    f = _fit(W.make("c1", n=2000), "fp64")
    p = wl.model
    rng = np.random.default_rng(3)
    w = p["w"] * rng.uniform(0.2, 3.0, len(p["w"]))
    base = dict(p, w=w)
    s0, c0 = f.diag_kinematics(KG, particles=base)
    g0 = f.diag_grid(wl.prior, particles=base)
    for order in (np.arange(len(w))[::-1], rng.permutation(len(w))):
        q = {k: np.ascontiguousarray(v[order]) for k, v in base.items()}
        s1, c1 = f.diag_kinematics(KG, particles=q)
        g1 = f.diag_grid(wl.prior, particles=q)
        assert np.array_equal(c0, c1) and np.array_equal(s0, s1)
        for a, b in zip(g0, g1):
            assert np.array_equal(a, b)
    so, _ = O.kin_sums(KG, O.ParticleSet(base))
    _assert_sums_close(s0, so)
    f.close()


def test_diagnostics_reject_non_finite_particles():
    wl = W.make("c1", n=2000)
    f = _fit(wl, "fp64")
    bad = dict(wl.model)
    bad["vx"] = bad["vx"].copy()
    bad["vx"][7] = np.nan
    with pytest.raises(B.M2MError, match="finite"):
        f.diag_kinematics(KG, particles=bad)
    f.close()


def test_diagnostics_argument_errors():
    wl = W.make("c1", n=2000)
    f = _fit(wl, "fp64")
    with pytest.raises(B.M2MError, match="n_r >= 2"):
        f.diag_kinematics(dict(KG, n_r=1))
    with pytest.raises(B.M2MError, match="0 < r_min < r_max"):
        f.diag_kinematics(dict(KG, r_min=5.0, r_max=1.0))
    g = B.SphGrid(4, 4, 4, 0.1, 10.0)
    sums = np.zeros(64 * 7)
    cnt = np.zeros(64, np.int64)
    assert B.lib().m2m_diag_kinematics(f.h, g, 0, None, None, None, B._dp(sums), B._i64(cnt), 63) != 0
    with pytest.raises(B.M2MError, match="ncell"):
        f._ck(B.lib().m2m_diag_grid(f.h, None, 0, None, None, None, B._dp(np.zeros(10)), None, None, 10))
    f.close()
