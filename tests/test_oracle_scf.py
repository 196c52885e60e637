"""Pins of the oracle's self-consistent stellar potential (Sec. 6): the multipole expansion
of the particles' luminosity on a radial grid, its force, the mass-to-light ratio and the
derivative of the observables that drives it. Checked against the addition theorem of
spherical harmonics, the Hernquist mass profile, finite differences and a velocity
rescaling of the observables (no GPU)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_1202_2355_gb300 import synth
from paper_1202_2355_gb300.workloads import Group


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _pot(r, lmax, ups=1.0, v0=0.0):
    return dict(kind="scf", G=1.0, v0=v0, r0=1.0, q=0.8, scf_r=np.asarray(r, float), scf_lmax=lmax, ups=ups)


def test_single_particle_matches_the_addition_theorem():
    """One unit mass on grid radius r_k: the truncated expansion is
    -G sum_{l <= L} r_<^l / r_>^(l+1) P_l(cos gamma) (sum over m of Y_lm Y_lm = (2l+1)/(4 pi) P_l)."""
    rng = np.random.default_rng(1)
    d = rng.normal(size=3)
    d *= 2.0 / np.linalg.norm(d)
    rp = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])  # the radius as the oracle computes it
    r = np.array([0.5, 1.0, rp, 3.0])
    L = 5
    pot = _pot(r, L)
    p = dict(x=np.array([d[0]]), y=np.array([d[1]]), z=np.array([d[2]]),
             vx=np.zeros(1), vy=np.zeros(1), vz=np.zeros(1), w=np.ones(1))
    d = d / rp
    a = O.scf_coeffs(pot, p)
    assert np.count_nonzero(np.abs(a).sum(1)) == 1  # all on point k = 2
    for _ in range(6):
        x = rng.normal(size=3) * rng.uniform(0.2, 2.5)
        rx = np.linalg.norm(x)
        cg = float(np.dot(x, d) / rx)
        rl, rg = min(rx, rp), max(rx, rp)
        want = -sum(rl ** l / rg ** (l + 1) * special.eval_legendre(l, cg) for l in range(L + 1))
        phi, _ = O.scf_field(pot, a, *x)
        assert phi == pytest.approx(want, rel=1e-12, abs=1e-14)


def test_gradient_is_the_derivative_of_the_potential():
    rng = np.random.default_rng(2)
    n = 400
    p = dict(x=rng.normal(size=n), y=rng.normal(size=n) * 0.7, z=rng.normal(size=n) * 0.5,
             vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n), w=rng.uniform(0.5, 1.5, n))
    pot = _pot(np.exp(np.linspace(math.log(0.1), math.log(4.0), 12)), 4)
    a = O.scf_coeffs(pot, p)
    h = 1e-6
    for _ in range(20):
        x = rng.normal(size=3) * rng.uniform(0.05, 5.0)
        _, g = O.scf_field(pot, a, *x)
        fd = np.zeros(3)
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd[c] = (O.scf_field(pot, a, *(x + e))[0] - O.scf_field(pot, a, *(x - e))[0]) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_monopole_force_of_a_hernquist_realisation():
    """A Hernquist sphere (eq. her, truncated at r = 50): between grid radii r_j and r_j+1 the
    monopole force is G m(<=j)/r^2, m(<=j) the luminosity the cloud-in-cell weights put on the
    points k <= j, whose expectation is the integral of those weights over the closed-form
    mass profile M(<r) = r^2/(1+r)^2 / (50/51)^2. Within Poisson error; l > 0 terms are noise."""
    N = 200_000
    p = synth.realise_spherical(11, N, synth.hernquist_sigma2_iso)
    r = np.exp(np.linspace(math.log(0.05), math.log(40.0), 25))
    pot = _pot(r, 2)
    a = O.scf_coeffs(pot, p)
    Mt = (50.0 / 51.0) ** 2
    dM = lambda s: 2.0 * s / (1.0 + s) ** 3 / Mt  # noqa: E731

    def below(j):  # expected luminosity on grid points 0..j
        m = integrate.quad(dM, 0.0, r[j], limit=200)[0]
        m += integrate.quad(lambda s: dM(s) * (r[j + 1] - s) / (r[j + 1] - r[j]), r[j], r[j + 1])[0]
        return m

    for j in (3, 8, 12, 16, 20):
        x = math.sqrt(r[j] * r[j + 1])
        _, g = O.scf_field(pot, a, x / math.sqrt(3), x / math.sqrt(3), x / math.sqrt(3))
        gr = float(np.linalg.norm(g))
        m = below(j)
        want = m / x ** 2
        sigma = math.sqrt(m * (1 - m) / N) / x ** 2
        assert abs(gr - want) < 4 * sigma + 2e-3 * want, (j, gr, want, sigma)


def test_total_force_is_upsilon_times_the_expansion_plus_the_log_halo():
    rng = np.random.default_rng(4)
    n = 300
    p = dict(x=rng.normal(size=n), y=rng.normal(size=n), z=rng.normal(size=n) * 0.6,
             vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n), w=np.full(n, 1.0 / n))
    r = np.exp(np.linspace(math.log(0.1), math.log(5.0), 10))
    pot = _pot(r, 2, ups=3.5, v0=0.7)
    a = O.scf_coeffs(pot, p)
    P = O.potential(pot)
    P._keep[1][:] = a.ravel()
    halo = dict(kind="log", v0=0.7, r0=1.0, q=0.8)
    for x in ([0.3, 0.2, 0.1], [1.5, -0.4, 0.9], [-3.0, 2.0, -1.0]):
        phi_s, g = O.scf_field(pot, a, *x)
        acc = np.zeros(3)
        import ctypes as C
        ax, ay, az = C.c_double(), C.c_double(), C.c_double()
        O.lib().or_accel(C.byref(P), *x, C.byref(ax), C.byref(ay), C.byref(az))
        want = -3.5 * g + np.array(O.accel(halo, *x))
        assert np.allclose([ax.value, ay.value, az.value], want, rtol=1e-13, atol=1e-15)
        assert O.lib().or_phi(C.byref(P), *x) == pytest.approx(3.5 * phi_s + O.phi(halo, *x), rel=1e-13)


def test_observable_derivative_matches_a_velocity_rescaling():
    """D_j = d y_j / d ln Upsilon with v scaling as Upsilon^(1/2) is half the derivative of
    the observables with respect to ln lambda for velocities scaled by lambda."""
    groups = [Group("annuli", ["mass"], [0.01], edges=np.exp(np.linspace(math.log(0.1), math.log(5), 7))),
              Group("annuli", ["v2", "gh2", "gh3", "gh4"], [0.01] * 4,
                    edges=np.exp(np.linspace(math.log(0.2), math.log(4), 5)))]
    p = synth.realise_spherical(5, 5000, synth.hernquist_sigma2_iso)
    Vp = np.concatenate([np.zeros(6), np.full(4, 0.05)])
    sp = np.concatenate([np.ones(6), np.array([0.5, 0.45, 0.4, 0.3])])
    obs = O.ObsSet(groups, 30.0, Vp=Vp, sp=sp)
    D = O.observe_dlnups(obs, O.ParticleSet(p))
    h = 1e-5
    ys = []
    for lam in (1 + h, 1 - h):
        q = dict(p, vx=p["vx"] * lam, vy=p["vy"] * lam, vz=p["vz"] * lam)
        ys.append(O.observe(obs, O.ParticleSet(q)))
    fd = 0.5 * (ys[0] - ys[1]) / (math.log(1 + h) - math.log(1 - h))
    assert np.all(D[:6] == 0.0)
    assert np.allclose(D, fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())
    # v^2 scales as Upsilon: D = y for the v^2 observables
    y = O.observe(obs, O.ParticleSet(p))
    assert np.allclose(D[6:10], y[6:10], rtol=1e-12)
