"""Pins of the oracle's diagnostics of a fitted particle model: intrinsic kinematics in
spherical polar bins and their rms difference to the target (Sec. 4.1), Delta_grid, the
mass-weighted relative rms difference of the (E, x) cell weights (Sec. 4.1), and the rms
of the particle weights about their cell means (Sec. 5, Fig. res).

Expected values come from hand-worked bins, closed forms (the Hernquist cumulative mass
and isotropic dispersion, the anisotropy the generator imposes), symmetries of the binning
and small cases worked out by hand."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import synth
from paper_1202_2355_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


# shells a factor of 2 wide: [0, 1), [1, 2), [2, 4), ..., [2^19, 2^20)
G2 = dict(n_r=21, n_phi=12, n_ct=20, r_min=1.0, r_max=2.0 ** 20)


def _bin(ir, ic, ip, g=G2):
    return (ir * g["n_ct"] + ic) * g["n_phi"] + ip


def test_spherical_bins_by_hand():
    # r = 3 is in [2, 4), shell 2; cos(theta) = 0.5 is in [0.5, 0.6), bin 15 of 20;
    # phi = 45 degrees is in [30, 60) degrees, bin 7 of 12 counted from -180
    r, ct, ph = 3.0, 0.5, math.radians(45.0)
    st = math.sqrt(1 - ct * ct)
    p = (r * st * math.cos(ph), r * st * math.sin(ph), r * ct)
    assert O.sph_bin(G2, *p) == _bin(2, 15, 7)
    # inside r_min: shell 0; on the +z axis: cos(theta) = 1 goes to the top bin, phi = 0
    assert O.sph_bin(G2, 0.0, 0.0, 0.5) == _bin(0, 19, 6)
    # the -x axis: phi = pi goes to the last azimuth bin; cos(theta) = 0 to bin 10
    assert O.sph_bin(G2, -5.0, 0.0, 0.0) == _bin(3, 10, 11)
    # -z axis: cos(theta) = -1 is bin 0
    assert O.sph_bin(G2, 0.0, 0.0, -1.5) == _bin(1, 0, 6)
    # the centre: shell 0, cos(theta) taken as 1
    assert O.sph_bin(G2, 0.0, 0.0, 0.0) == _bin(0, 19, 6)
    # r >= r_max is not binned
    assert O.sph_bin(G2, 2.0 ** 20, 0.0, 0.0) == -1
    assert O.sph_bin(G2, 2.0 ** 20 - 1.0, 0.0, 0.0) == _bin(20, 10, 6)


def test_velocity_components():
    rng = np.random.default_rng(5)
    for _ in range(50):
        x = rng.standard_normal(3) * 3
        v = rng.standard_normal(3)
        vr, vt, vp = O.sph_velocity(*x, *v)
        assert vr * vr + vt * vt + vp * vp == pytest.approx(v @ v, rel=1e-13)
        # a velocity along the position vector is purely radial
        u = x / np.linalg.norm(x)
        assert np.allclose(O.sph_velocity(*x, *(2.5 * u)), [2.5, 0, 0], atol=1e-14)
        # a rotation about z leaves all three components unchanged
        a = rng.uniform(0, 2 * math.pi)
        Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
        assert np.allclose(O.sph_velocity(*(Rz @ x), *(Rz @ v)), [vr, vt, vp], atol=1e-13)
    # prograde circular motion in the equatorial plane: v_phi = +v
    assert np.allclose(O.sph_velocity(0.0, 2.0, 0.0, -0.7, 0.0, 0.0), [0, 0, 0.7], atol=1e-15)
    # moving towards -z from the equator is +v_theta (theta grows)
    assert np.allclose(O.sph_velocity(1.0, 0.0, 0.0, 0.0, 0.0, -0.3), [0, 0.3, 0], atol=1e-15)


KG = dict(n_r=21, n_phi=12, n_ct=21, r_min=0.01, r_max=50.0)


def _shell_totals(sums, counts, g):
    s = sums.reshape(g["n_r"], g["n_ct"] * g["n_phi"], O.KIN_SUMS).sum(axis=1)
    c = counts.reshape(g["n_r"], -1).sum(axis=1)
    return s, c


def _edges(g):
    return np.r_[0.0, np.exp(np.linspace(math.log(g["r_min"]), math.log(g["r_max"]), g["n_r"]))]


def test_shell_masses_follow_the_hernquist_profile():
    """Shell masses of a Hernquist realisation (r < 50) against the closed-form enclosed
    mass M(<r) = r^2/(1+r)^2, normalised to the truncation, within 4.5 Poisson sigma."""
    n = 200_000
    ps = O.ParticleSet(synth.realise_spherical(3, n, W.hernquist_sigma2))
    sums, counts = O.kin_sums(KG, ps)
    s, c = _shell_totals(sums, counts, KG)
    e = _edges(KG)
    Mt = synth.hernquist_mass(50.0)
    frac = np.diff(synth.hernquist_mass(e) / Mt)
    assert counts.sum() == n and s[:, 0].sum() == pytest.approx(1.0, rel=1e-12)
    sig = np.sqrt(n * frac * (1 - frac))
    assert np.all(np.abs(c - n * frac) <= 4.5 * sig + 1)
    assert np.allclose(s[:, 0], c / n, rtol=1e-12)


def _shell_dispersions(model, g, lo=0.1, hi=5.0):
    ps = O.ParticleSet(model)
    sums, counts = O.kin_sums(g, ps)
    s, c = _shell_totals(sums, counts, g)
    e = _edges(g)
    keep = (e[:-1] >= lo) & (e[1:] <= hi) & (c > 2000)
    mean = s[keep, 1:4] / s[keep, :1]
    disp = np.sqrt(s[keep, 4:7] / s[keep, :1] - mean ** 2)
    rmid = np.sqrt(e[:-1] * e[1:])[keep]
    return mean, disp, rmid, c[keep]


def test_isotropic_dispersions_match_the_jeans_closed_form():
    """The isotropic Hernquist realisation: each velocity component has the dispersion of
    Hernquist (1990, eq. 10) and zero mean, per shell, within sampling error."""
    mean, disp, rmid, c = _shell_dispersions(synth.realise_spherical(4, 300_000, W.hernquist_sigma2), KG)
    assert len(c) >= 8
    sj = np.sqrt(synth.hernquist_sigma2_iso(rmid))
    # the shell spans a range of radii; compare to within 4 % plus 5 sampling sigmas
    tol = 0.04 + 5.0 / np.sqrt(2.0 * c)
    for k in range(3):
        assert np.all(np.abs(disp[:, k] / sj - 1) < tol), (k, disp[:, k] / sj)
        assert np.all(np.abs(mean[:, k]) < 5.0 * disp[:, k] / np.sqrt(c))


def test_radial_anisotropy_is_recovered():
    """A realisation with sigma_r/sigma_t = 1.5 at every radius: the r, theta and phi
    dispersions of each shell show that ratio (a mixed-up basis would not)."""
    mean, disp, rmid, c = _shell_dispersions(
        synth.realise_spherical(6, 300_000, W.hernquist_sigma2, anisotropy=1.5), KG)
    tol = 6.0 / np.sqrt(c)
    assert np.all(np.abs(disp[:, 0] / disp[:, 1] - 1.5) < 1.5 * tol)
    assert np.all(np.abs(disp[:, 0] / disp[:, 2] - 1.5) < 1.5 * tol)
    assert np.all(np.abs(disp[:, 1] / disp[:, 2] - 1.0) < tol)


def test_rotation_and_reflection_move_the_bins():
    """A rotation about z by one azimuth bin (30 degrees) moves every sum one bin up in
    phi; the reflection z -> -z reverses the cos(theta) bins and flips sum w v_theta."""
    g = dict(n_r=6, n_phi=12, n_ct=5, r_min=0.3, r_max=20.0)
    m = synth.realise_spherical(8, 20_000, W.hernquist_sigma2)
    rng = np.random.default_rng(2)
    m["w"] = rng.uniform(0.5, 1.5, len(m["w"])) / len(m["w"])
    # keep particles off the azimuth edges so that the rotated ones cannot round across
    ph = np.arctan2(m["y"], m["x"])
    f = (ph + math.pi) / (2 * math.pi) * 12
    keep = np.abs(f - np.round(f)) > 1e-6
    m = {k: v[keep] for k, v in m.items()}
    s0, c0 = O.kin_sums(g, O.ParticleSet(m))
    a = 2 * math.pi / 12
    r = dict(m)
    r["x"], r["y"] = m["x"] * math.cos(a) - m["y"] * math.sin(a), m["x"] * math.sin(a) + m["y"] * math.cos(a)
    r["vx"], r["vy"] = m["vx"] * math.cos(a) - m["vy"] * math.sin(a), m["vx"] * math.sin(a) + m["vy"] * math.cos(a)
    s1, c1 = O.kin_sums(g, O.ParticleSet(r))
    shape = (g["n_r"], g["n_ct"], g["n_phi"])
    assert np.array_equal(np.roll(c0.reshape(shape), 1, axis=2), c1.reshape(shape))
    assert np.allclose(np.roll(s0.reshape(shape + (7,)), 1, axis=2), s1.reshape(shape + (7,)), rtol=1e-9, atol=1e-14)
    z = dict(m)
    z["z"], z["vz"] = -m["z"], -m["vz"]
    s2, c2 = O.kin_sums(g, O.ParticleSet(z))
    assert np.array_equal(c0.reshape(shape)[:, ::-1, :], c2.reshape(shape))
    flip = np.array([1, 1, -1, 1, 1, 1, 1.0])
    assert np.allclose(s0.reshape(shape + (7,))[:, ::-1, :] * flip, s2.reshape(shape + (7,)), rtol=1e-9, atol=1e-14)


def test_moments_and_delta_kin_small_cases():
    nb = 3
    sums = np.zeros((nb, 7))
    # bin 0: weights 1 and 3 with v_r = +2 and -2: mean -1, dispersion sqrt(4 - 1)
    sums[0] = [4, 2 - 6, 0, 0, 4 + 12, 0, 0]
    # bin 1: one particle (below min_count 2); bin 2: empty
    sums[1] = [1, 1, 1, 1, 1, 1, 1]
    counts = np.array([2, 1, 0], np.int64)
    mean, disp, valid = O.kin_moments(sums, counts, min_count=2)
    assert valid.tolist() == [True, False, False]
    assert mean[0].tolist() == [-1.0, 0.0, 0.0]
    assert disp[0, 0] == pytest.approx(math.sqrt(3.0), rel=1e-15) and disp[0, 1] == 0.0
    # delta_kin: a model whose v_phi is the target's shifted by 0.25 in every valid bin
    t = np.zeros((nb, 7))
    t[:, 0] = 2.0
    t[:, 6] = 2.0 * 1.0   # sigma_phi = 1, mean 0
    m = t.copy()
    m[:, 3] = 2.0 * 0.25  # mean v_phi 0.25
    m[:, 6] = 2.0 * (1.0 + 0.0625)  # same dispersion about the new mean
    cnt = np.array([5, 5, 1], np.int64)
    out, used = O.delta_kin(m, cnt, t, cnt, min_count=2)
    assert used == 2
    assert out[2] == pytest.approx(0.25, rel=1e-14)
    assert np.abs(np.delete(out, [2, 6])).max() < 1e-15
    assert out[6] == pytest.approx(0.25 / math.sqrt(6.0), rel=1e-14)
    out, _ = O.delta_kin(t, cnt, t, cnt)
    assert np.all(out == 0.0)


def test_delta_grid_definition():
    wt = np.array([0.5, 0.25, 0.25, 0.0])
    assert O.delta_grid(wt, wt) == 0.0
    # a model proportional to the target gives 0 (each is normalised to unit total)
    assert O.delta_grid(3.0 * wt, wt) == 0.0
    # model (0.25, 0.5, 0.25, x): relative differences (0.5, -1, 0) weighted by the target;
    # the last cell has no target weight and is left out
    wm = np.array([0.25, 0.5, 0.25, 0.0])
    assert O.delta_grid(wm, wt) == pytest.approx(math.sqrt(0.5 * 0.25 + 0.25 * 1.0), rel=1e-15)


def test_grid_weights_and_weight_rms():
    wl = W.make("c1", n=5000)
    m = dict(wl.model)
    rng = np.random.default_rng(3)
    m["w"] = rng.uniform(0.5, 1.5, 5000) / 5000
    ps = O.ParticleSet(m)
    ws, wd, cnt = O.grid_weights(wl.potential, wl.prior, ps)
    assert cnt.sum() == 5000 and ws.sum() == pytest.approx(m["w"].sum(), rel=1e-13)
    cells, _, _ = O.cells(wl.potential, wl.prior, ps)
    assert np.array_equal(np.bincount(cells, minlength=len(cnt)), cnt)
    assert np.all(wd >= 0)
    # equal weights have no spread, up to the rounding of the cell mean
    m["w"] = np.full(5000, 2e-4)
    ws, wd, cnt = O.grid_weights(wl.potential, wl.prior, O.ParticleSet(m))
    assert np.all(np.sqrt(wd / np.maximum(cnt, 1)) < 1e-14 * 2e-4)
    # one cell: n p particles of weight a and n (1-p) of weight b: sum of squared deviations
    # n p (1-p) (a-b)^2
    one = dict(wl.prior, nE=1, nx=1)
    n, a, b = 5000, 3e-4, 1e-4
    m["w"] = np.where(np.arange(n) < 1000, a, b)
    ws, wd, cnt = O.grid_weights(wl.potential, one, O.ParticleSet(m))
    assert cnt[0] == n and wd[0] == pytest.approx(n * 0.2 * 0.8 * (a - b) ** 2, rel=1e-10)
    assert O.weight_rms(wd, cnt, 50) == pytest.approx(math.sqrt(0.16) * (a - b), rel=1e-10)
    # cells with min_count or fewer particles are left out
    wd2 = np.array([4.0, 100.0, 9.0])
    c2 = np.array([100, 50, 300], np.int64)
    assert O.weight_rms(wd2, c2, 50) == pytest.approx(math.sqrt(13.0 / 400.0), rel=1e-15)
    assert O.weight_rms(wd2, c2, 1000) == 0.0
