"""Pins of the oracle's spherical-harmonic density coefficients (eq. alm):
a_lm,k = sum_i w_i gamma_k(r_i) Y_lm(theta_i, phi_i) on a 3-D radial grid with cloud-in-cell
weights gamma, the real Y_lm of unit norm, and the shot-noise errors of the targets.

Expected values come from scipy's complex spherical harmonics, quadrature over the sphere,
the linear reproduction property of cloud-in-cell weights, the closed-form Hernquist mass
profile, and the symmetries of the coefficients under rotations and flattening."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import synth
from paper_1202_2355_gb300 import workloads as W
from paper_1202_2355_gb300.workloads import Group

sp = pytest.importorskip("scipy.special")


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


LM = [(l, m) for l in range(7) for m in range(-l, l + 1)]


def test_real_harmonics_match_scipy():
    """m > 0: sqrt2 (-1)^m Re Y_l^m; m < 0: sqrt2 (-1)^|m| Im Y_l^|m|; m = 0: Y_l^0, with
    scipy's complex harmonics (which carry the Condon-Shortley phase)."""
    rng = np.random.default_rng(1)
    for _ in range(40):
        ct, phi = rng.uniform(-1, 1), rng.uniform(-math.pi, math.pi)
        th = math.acos(ct)
        for l, m in LM:
            z = complex(sp.sph_harm_y(l, abs(m), th, phi))
            want = z.real if m == 0 else math.sqrt(2) * (-1) ** abs(m) * (z.real if m > 0 else z.imag)
            assert O.ylm(l, m, ct, phi) == pytest.approx(want, rel=1e-12, abs=1e-13), (l, m)


def test_real_harmonics_are_orthonormal():
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = 2 * math.pi * (np.arange(nphi) + 0.5) / nphi
    sub = [(l, m) for l, m in LM if l <= 4]
    vals = np.array([[O.ylm(l, m, c, f) for c in xg for f in phis] for l, m in sub])
    w = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    G = vals @ (vals * w).T
    assert np.allclose(G, np.eye(len(sub)), atol=1e-12)


def _shells(radii, kinds, err=1.0):
    return Group("shells", kinds, [err] * len(kinds), edges=np.asarray(radii, float))


def test_cloud_in_cell_weights():
    """The weights of a radius sum to 1 and reproduce r itself (linear interpolation);
    inside r_0 all goes to point 0, beyond the last radius nothing is binned."""
    radii = [0.5, 1.0, 2.0, 3.5, 6.0]
    g = _shells(radii, ["alm_0_0"])
    obs = O.ObsSet([g])
    y00 = 1.0 / math.sqrt(4 * math.pi)
    for r in [0.1, 0.5, 0.7, 1.0, 1.9, 3.0, 5.99]:
        ps = O.ParticleSet(dict(x=[r], y=[0.0], z=[0.0], vx=[0.0], vy=[0.0], vz=[0.0], w=[1.0]))
        y = O.observe(obs, ps) / y00
        assert y.sum() == pytest.approx(1.0, rel=1e-14)
        assert np.count_nonzero(y) <= 2
        if r >= radii[0]:
            assert y @ np.asarray(radii) == pytest.approx(r, rel=1e-14)
        else:
            assert y[0] == 1.0
    ps = O.ParticleSet(dict(x=[6.0], y=[0.0], z=[0.0], vx=[0.0], vy=[0.0], vz=[0.0], w=[1.0]))
    assert np.all(O.observe(obs, ps) == 0.0)


def _hat_mass(radii, k, M):
    """int gamma_k(r) dM(r) for the cloud-in-cell hat of point k (Gauss-Legendre)."""
    xg, wg = np.polynomial.legendre.leggauss(40)
    tot = 0.0
    r = np.asarray(radii)
    if k == 0:
        tot += M(r[0])  # everything inside r_0
    for a, b, up in ((r[k - 1] if k > 0 else None, r[k], True), (r[k], r[k + 1] if k + 1 < len(r) else None, False)):
        if a is None or b is None:
            continue
        t = 0.5 * (b - a) * xg + 0.5 * (a + b)
        dens = 4 * math.pi * t * t * synth.hernquist_density(t)
        hat = (t - a) / (b - a) if up else (b - t) / (b - a)
        tot += 0.5 * (b - a) * np.dot(wg, hat * dens)
    return tot


def test_monopole_of_a_hernquist_realisation():
    """a_00,k of a Hernquist sphere (r < 50) against the cloud-in-cell hat integrated over
    the closed-form profile, within 4.5 of the shot-noise errors the targets are given;
    every higher coefficient is zero within its error."""
    radii = np.exp(np.linspace(math.log(0.05), math.log(20.0), 12))
    kinds = [f"alm_{l}_{m}" for l, m in LM if l <= 3]  # 16 kinds, the most a group holds
    g = _shells(radii, kinds)
    obs = O.ObsSet([g])
    n = 200_000
    p = synth.realise_spherical(9, n, W.hernquist_sigma2)
    ps = O.ParticleSet(p)
    y = O.observe(obs, ps)
    Y, sig, _ = O.build_targets(O.ObsSet([g]), ps, np.ones(obs.J))
    assert np.array_equal(Y, y)
    Mt = synth.hernquist_mass(50.0)  # the realisation is truncated at r = 50
    nk = len(radii)
    for k in range(nk):
        want = _hat_mass(radii, k, synth.hernquist_mass) / Mt / math.sqrt(4 * math.pi)
        assert abs(y[k] - want) < 4.5 * sig[k], (k, y[k], want, sig[k])
    # the errors are the same for every (l, m) of a grid point
    assert np.allclose(sig.reshape(len(kinds), nk), sig[:nk][None, :], rtol=0)
    z = (y / sig).reshape(len(kinds), nk)[1:]
    assert np.abs(z).max() < 5.0
    assert np.mean(z ** 2) == pytest.approx(1.0, abs=0.25)


def test_rotation_about_z_and_flattening():
    radii = [0.3, 0.8, 1.5, 3.0, 6.0]
    kinds = ["alm_0_0", "alm_2_0", "alm_2_2", "alm_2_-2", "alm_3_1", "alm_3_-1", "alm_4_4", "alm_4_-4"]
    g = _shells(radii, kinds)
    obs = O.ObsSet([g])
    p = synth.realise_spherical(10, 20_000, W.hernquist_sigma2)
    rng = np.random.default_rng(4)
    p["w"] = rng.uniform(0.5, 1.5, 20_000) / 20_000
    y = O.observe(obs, O.ParticleSet(p)).reshape(len(kinds), -1)
    a = 0.37
    r = dict(p)
    r["x"] = p["x"] * math.cos(a) - p["y"] * math.sin(a)
    r["y"] = p["x"] * math.sin(a) + p["y"] * math.cos(a)
    yr = O.observe(obs, O.ParticleSet(r)).reshape(len(kinds), -1)
    # rotating the particles by a about z: (a_lm, a_l,-m) turns by the angle m a
    assert np.allclose(yr[0], y[0], rtol=1e-12) and np.allclose(yr[1], y[1], rtol=1e-12)
    for i, m in ((2, 2), (4, 1), (6, 4)):
        c, s = math.cos(m * a), math.sin(m * a)
        assert np.allclose(yr[i], c * y[i] - s * y[i + 1], rtol=1e-9, atol=1e-15)
        assert np.allclose(yr[i + 1], s * y[i] + c * y[i + 1], rtol=1e-9, atol=1e-15)
    # an oblate flattening z -> 0.7 z makes a_20 negative, far beyond its noise
    f = dict(p)
    f["z"] = 0.7 * p["z"]
    yf = O.observe(obs, O.ParticleSet(f)).reshape(len(kinds), -1)
    _, sig, _ = O.build_targets(O.ObsSet([g]), O.ParticleSet(f), np.ones(obs.J))
    sig = sig.reshape(len(kinds), -1)
    assert np.all(yf[1, 1:] < -5 * sig[1, 1:])
