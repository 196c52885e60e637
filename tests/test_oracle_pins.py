"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form,
an invariant, a brute-force evaluation on a tiny input, or a special case that
reduces to a textbook or library routine. The paper (arXiv 1202.2355) prints no
worked numerical example, so every pin follows from the equations it cites.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special

import oracle as O
from paper_1202_2355_gb300 import synth
from paper_1202_2355_gb300.workloads import Group

HERN = dict(kind="hernquist", G=1.0, M=1.0, a=1.0)
MS = synth.nfw_ms_from_m200(20.0, 10.0)
HNFW = dict(kind="hernquist_nfw", G=1.0, M=1.0, a=1.0, Ms=MS, rs=8.0)
LOGQ = dict(kind="log", v0=1.0, r0=1.0, q=0.8)


def _parts(arrs):
    x, y, z, vx, vy, vz, w = [np.atleast_1d(np.asarray(a, np.float64)) for a in arrs]
    return dict(x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, w=w)


# ---------------------------------------------------------------- potentials

def _laplacian(pot, x, y, z, h):
    f0 = O.phi(pot, x, y, z)
    s = 0.0
    for d in np.eye(3):
        s += O.phi(pot, x + h * d[0], y + h * d[1], z + h * d[2]) \
            + O.phi(pot, x - h * d[0], y - h * d[1], z - h * d[2]) - 2 * f0
    return s / (h * h)


@pytest.mark.parametrize("r", [0.3, 1.0, 2.5, 7.0])
def test_hernquist_potential_obeys_poisson_with_eq_her_density(r):
    """Laplacian of phi equals 4 pi G rho, rho(r) = a M / (2 pi r (r+a)^3) (eq. her)."""
    x, y, z = r * np.array([0.48, 0.6, 0.64])
    lap = _laplacian(HERN, x, y, z, 1e-3 * r)
    rho = 1.0 / (2 * math.pi * r * (r + 1) ** 3)
    assert lap == pytest.approx(4 * math.pi * rho, rel=2e-5)


@pytest.mark.parametrize("r", [0.5, 3.0, 20.0])
def test_nfw_part_obeys_poisson(r):
    x, y, z = r * np.array([0.6, 0.0, 0.8])
    lap = _laplacian(HNFW, x, y, z, 1e-3 * r)
    rho_h = 1.0 / (2 * math.pi * r * (r + 1) ** 3)
    rho_nfw = MS / (4 * math.pi * r * (8.0 + r) ** 2)
    assert lap == pytest.approx(4 * math.pi * (rho_h + rho_nfw), rel=2e-5)


@pytest.mark.parametrize("R,z", [(0.5, 0.2), (2.0, -1.0), (0.1, 3.0)])
def test_flattened_log_potential_density(R, z):
    """Poisson density of the flattened logarithmic potential (eq. log_halo):
    rho = v0^2/(4 pi G q^2) [(2q^2+1) r0^2 + R^2 + (2 - q^-2) z^2] / (r0^2 + R^2 + z^2/q^2)^2."""
    q = 0.8
    lap = _laplacian(LOGQ, R, 0.0, z, 1e-3)
    rho = ((2 * q * q + 1) + R * R + (2 - q ** -2) * z * z) / (1 + R * R + z * z / q ** 2) ** 2 \
        / (4 * math.pi * q * q)
    assert lap == pytest.approx(4 * math.pi * rho, rel=1e-5)


@pytest.mark.parametrize("pot", [HERN, HNFW, LOGQ])
def test_acceleration_is_minus_gradient(pot):
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = rng.normal(size=3) * rng.uniform(0.05, 5.0)
        a = O.accel(pot, *p)
        g = np.zeros(3)
        for k in range(3):
            h = 1e-5 * max(1.0, abs(p[k]))
            e = np.zeros(3)
            e[k] = h
            g[k] = (O.phi(pot, *(p + e)) - O.phi(pot, *(p - e))) / (2 * h)
        assert np.allclose(a, -g, rtol=1e-6, atol=1e-9)


def test_nfw_small_radius_series_is_continuous():
    """The series branch of M_nfw(r) joins the closed form at q = 1e-3 (rs = 8 -> r = 8e-3)."""
    pot = dict(HNFW, M=0.0)
    r_lo, r_hi = 8e-3 * (1 - 1e-12), 8e-3 * (1 + 1e-12)
    a_lo = O.accel(pot, r_lo, 0, 0)[0] / r_lo
    a_hi = O.accel(pot, r_hi, 0, 0)[0] / r_hi
    assert a_lo == pytest.approx(a_hi, rel=1e-9)
    # and both equal -G M(<r)/r^3 from the mpmath-free high-precision series value
    q = 1e-3
    mu = sum((-1) ** k * (k - 1) / k * q ** k for k in range(2, 30))
    assert a_hi == pytest.approx(-MS * mu / 8e-3 ** 3, rel=1e-9)


# ---------------------------------------------------------------- leapfrog

def _orbit(pot, p0, dt, nsteps):
    ps = O.ParticleSet(_parts([*p0, 1.0]))
    out = []
    for _ in range(nsteps):
        O.leapfrog(pot, ps, dt)
        out.append([ps[k][0] for k in ("x", "y", "z", "vx", "vy", "vz")])
    return np.array(out)


def _EL(pot, s):
    E = np.array([0.5 * (q[3] ** 2 + q[4] ** 2 + q[5] ** 2) + O.phi(pot, *q[:3]) for q in s])
    L = np.cross(s[:, :3], s[:, 3:])
    return E, L


@pytest.mark.parametrize("pot", [HERN, HNFW])
def test_leapfrog_conserves_angular_momentum_in_spherical_potential(pot):
    p0 = [1.2, -0.3, 0.4, 0.1, 0.35, -0.2]
    s = _orbit(pot, p0, 0.01, 3000)
    _, L = _EL(pot, s)
    L0 = np.cross(p0[:3], p0[3:])
    assert np.max(np.abs(L - L0)) < 1e-13


def test_leapfrog_conserves_lz_in_axisymmetric_potential():
    p0 = [1.0, 0.2, 0.3, -0.1, 0.6, 0.2]
    s = _orbit(LOGQ, p0, 0.01, 3000)
    Lz = s[:, 0] * s[:, 4] - s[:, 1] * s[:, 3]
    assert np.max(np.abs(Lz - (p0[0] * p0[4] - p0[1] * p0[3]))) < 1e-13


def test_leapfrog_energy_error_is_second_order_and_bounded():
    p0 = [1.0, 0.0, 0.0, 0.0, 0.3, 0.1]
    errs = []
    for dt in (0.02, 0.01):
        s = _orbit(HERN, p0, dt, int(round(40.0 / dt)))
        E, _ = _EL(HERN, s)
        E0 = 0.5 * (0.3 ** 2 + 0.1 ** 2) + O.phi(HERN, 1.0, 0, 0)
        errs.append(np.max(np.abs(E - E0)))
        # bounded: no secular drift between the first and last quarter
        q = len(E) // 4
        assert abs(np.max(np.abs(E[-q:] - E0)) - np.max(np.abs(E[:q] - E0))) < 0.5 * errs[-1] + 1e-12
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


def test_leapfrog_is_time_reversible():
    p0 = np.array([0.7, 0.2, -0.4, 0.3, -0.1, 0.5])
    ps = O.ParticleSet(_parts([*p0, 1.0]))
    for _ in range(500):
        O.leapfrog(HNFW, ps, 0.01)
    for k in ("vx", "vy", "vz"):
        ps[k][0] *= -1
    for _ in range(500):
        O.leapfrog(HNFW, ps, 0.01)
    back = np.array([ps[k][0] for k in ("x", "y", "z")] + [-ps[k][0] for k in ("vx", "vy", "vz")])
    assert np.allclose(back, p0, atol=1e-12)


def test_circular_orbit_period():
    """Circular orbit at r = 1 in the Hernquist potential: v_c = sqrt(r)/(r+1) = 0.5,
    period 2 pi r / v_c = 4 pi."""
    dt = 4 * math.pi / 4000
    s = _orbit(HERN, [1.0, 0, 0, 0, 0.5, 0], dt, 4000)
    r = np.sqrt((s[:, :3] ** 2).sum(1))
    assert np.max(np.abs(r - 1.0)) < 1e-5
    assert np.allclose(s[-1, :3], [1.0, 0, 0], atol=1e-5)


# ---------------------------------------------------------------- Gauss-Hermite

def test_hermite_polynomials_match_scipy():
    for n in range(7):
        for x in (-2.3, -0.4, 0.0, 0.9, 3.1):
            assert O.hermite(n, x) == pytest.approx(special.eval_hermite(n, x), rel=1e-13, abs=1e-12)


def test_gh_kernels_are_orthogonal_with_norm_2_sqrt_pi():
    """int u_m u_n dnu = delta_mn / (2 sqrt pi), so int K_m K_n = 2 sqrt(pi) delta_mn."""
    nodes, wts = np.polynomial.hermite.hermgauss(60)  # weight exp(-x^2)
    for m in range(7):
        for n in range(7):
            f = np.array([O.gh_kernel(m, x) * O.gh_kernel(n, x) for x in nodes]) * np.exp(nodes ** 2)
            val = np.dot(wts, f)
            assert val == pytest.approx(2 * math.sqrt(math.pi) * (m == n), abs=1e-11)


def _gauss_expect(n, m, s):
    """E[K_n(nu)] for nu ~ N(m, s^2), by Gauss-Hermite quadrature."""
    nodes, wts = np.polynomial.hermite.hermgauss(80)
    nu = m + math.sqrt(2) * s * nodes
    return np.dot(wts, [O.gh_kernel(n, v) for v in nu]) / math.sqrt(math.pi)


def test_gaussian_losvd_gives_h0_one_and_higher_zero():
    assert _gauss_expect(0, 0.0, 1.0) == pytest.approx(1.0, abs=1e-13)
    for n in range(1, 7):
        assert _gauss_expect(n, 0.0, 1.0) == pytest.approx(0.0, abs=1e-13)


@pytest.mark.parametrize("m,s", [(0.3, 1.0), (-0.1, 1.2), (0.0, 0.8)])
def test_h1_h2_closed_forms_and_first_order_relations(m, s):
    """For nu ~ N(m, s^2): E[K_1] = 2m e^{-m^2/(2(1+s^2))}/(1+s^2)^{3/2}, and for m = 0
    E[K_2] = (s^2-1)/(1+s^2)^{3/2}; near (0, 1) these reduce to eq. h1h2."""
    k1 = 2 * m * math.exp(-m * m / (2 * (1 + s * s))) / (1 + s * s) ** 1.5
    assert _gauss_expect(1, m, s) == pytest.approx(k1, abs=1e-13)
    if m == 0.0:
        assert _gauss_expect(2, 0.0, s) == pytest.approx((s * s - 1) / (1 + s * s) ** 1.5, abs=1e-13)
    # first-order: V_p offset dV (in units of sigma) -> h1 = -dV/(sqrt2 sigma)
    d = 1e-4
    assert _gauss_expect(1, d, 1.0) == pytest.approx(d / math.sqrt(2), rel=1e-6)
    assert _gauss_expect(2, 0.0, 1.0 + d) == pytest.approx(d / math.sqrt(2), rel=1e-3)


# ---------------------------------------------------------------- observables

def _tiny_obs():
    groups = [Group("annuli", ["mass"], [0.01], edges=np.array([0.1, 0.3, 0.7, 1.5, 3.0])),
              Group("annuli", ["v2", "gh3", "gh4"], [0.01, 0.01, 0.01], edges=np.array([0.2, 0.6, 2.0])),
              Group("pixels", ["mass", "gh1"], [0.02, 0.02], nx=3, ny=2, box=(-1.5, 1.5, -1.0, 1.0))]
    Vp = np.array([0] * 4 + [0.05, -0.02] + [0.0] * 6)
    sp = np.array([1] * 4 + [0.4, 0.3] + [0.5] * 6, dtype=float)
    return groups, Vp, sp


@pytest.mark.parametrize("incl", [0.0, 60.0])
def test_kernel_matrix_brute_force(incl):
    """y = K^T w for N = 64, with K built here from the definitions by an independent
    binning (searchsorted / floor) and scipy's Hermite polynomials."""
    groups, Vp, sp = _tiny_obs()
    obs = O.ObsSet(groups, incl, Vp, sp)
    rng = np.random.default_rng(7)
    n = 64
    p = _parts([*rng.normal(size=(3, n)) * 1.2, *rng.normal(size=(3, n)) * 0.4, rng.uniform(0.5, 1.5, n) / n])
    ps = O.ParticleSet(p)
    K = O.kernel_matrix(obs, ps)
    ci, si = math.cos(math.radians(incl)), math.sin(math.radians(incl))
    X, Y = p["x"], p["y"] * ci - p["z"] * si
    v = p["vy"] * si + p["vz"] * ci
    Kref = np.zeros((n, obs.J))
    R = np.hypot(X, Y)
    e0 = groups[0].edges
    p0 = np.searchsorted(e0, R, side="right") - 1
    for i in range(n):
        if 0 <= p0[i] < 4:
            Kref[i, p0[i]] = 1 / (math.pi * (e0[p0[i] + 1] ** 2 - e0[p0[i]] ** 2))
    e1 = groups[1].edges
    p1 = np.searchsorted(e1, R, side="right") - 1
    for i in range(n):
        if 0 <= p1[i] < 2:
            a = p1[i]
            nu = (v[i] - Vp[4 + a]) / sp[4 + a]
            Kref[i, 4 + a] = v[i] ** 2
            for kk, nn in ((1, 3), (2, 4)):
                un = special.eval_hermite(nn, nu) * math.exp(-nu * nu / 2) / math.sqrt(
                    2 ** (nn + 1) * math.pi * math.factorial(nn))
                Kref[i, 4 + kk * 2 + a] = 2 * math.sqrt(math.pi) * un
    px = np.floor((X + 1.5) / 1.0)
    py = np.floor((Y + 1.0) / 1.0)
    for i in range(n):
        if 0 <= px[i] < 3 and 0 <= py[i] < 2:
            a = int(py[i] * 3 + px[i])
            Kref[i, 10 + a] = 1.0
            nu = (v[i] - 0.0) / 0.5
            Kref[i, 16 + a] = 2 * math.sqrt(math.pi) * 2 * nu * math.exp(-nu * nu / 2) / math.sqrt(4 * math.pi)
    assert np.allclose(K, Kref, rtol=1e-13, atol=1e-15)
    assert np.count_nonzero(K) > 40
    y = O.observe(obs, ps)
    assert np.allclose(y, K.T @ p["w"], rtol=1e-14, atol=1e-16)


def _hernquist_sigma_surface(s):
    """Closed-form Hernquist surface density (Hernquist 1990, eqs. 32-33), M = a = 1."""
    if s < 1:
        X = np.arccosh(1 / s) / math.sqrt(1 - s * s)
    else:
        X = np.arccos(1 / s) / math.sqrt(s * s - 1)
    return ((2 + s * s) * X - 3) / (2 * math.pi * (1 - s * s) ** 2)


def test_closed_form_surface_density_is_projection_of_eq_her():
    for R in (0.05, 0.4, 2.0, 7.0):
        proj = 2 * integrate.quad(lambda z: synth.hernquist_density(math.hypot(R, z)), 0, np.inf,
                                  limit=200)[0]
        assert _hernquist_sigma_surface(R) == pytest.approx(proj, rel=1e-7)


@pytest.fixture(scope="module")
def equilibrium():
    return synth.realise_spherical(11, 200_000, synth.hernquist_sigma2_iso, rmax=50.0)


def test_equilibrium_realisation_reproduces_surface_density(equilibrium):
    """Mass per annulus (y_j A_j) of a truncated (r < 50) Hernquist realisation against the
    projected truncated density, within 5 Poisson sigma."""
    edges = np.exp(np.linspace(math.log(0.05), math.log(20), 31))
    obs = O.ObsSet([Group("annuli", ["mass"], [0.01], edges=edges)])
    y = O.observe(obs, O.ParticleSet(equilibrium))
    area = math.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    mt = (50 / 51) ** 2

    def sig_t(R):
        return 2 * integrate.quad(lambda z: synth.hernquist_density(math.hypot(R, z)), 0,
                                  math.sqrt(50 ** 2 - R * R))[0] / mt

    for p in range(30):
        m = integrate.quad(lambda R: 2 * math.pi * R * sig_t(R), edges[p], edges[p + 1])[0]
        err = math.sqrt(m * (1 - m) / 200_000)
        assert abs(y[p] * area[p] - m) < 5 * err + 1e-12, p
    # and the analytic untruncated profile at the centre, where truncation is negligible
    for p in range(3):
        m = integrate.quad(lambda R: 2 * math.pi * R * _hernquist_sigma_surface(R), edges[p],
                           edges[p + 1])[0] / mt
        assert abs(y[p] * area[p] - m) < 5 * math.sqrt(m / 200_000)


def test_equilibrium_realisation_reproduces_projected_dispersion(equilibrium):
    """Sum of w v_los^2 per annulus against the projection of rho sigma_r^2 for the
    isotropic Jeans solution (the velocities are drawn with sigma_r(r))."""
    edges = np.exp(np.linspace(math.log(0.1), math.log(5), 16))
    obs = O.ObsSet([Group("annuli", ["v2"], [0.01], edges=edges)])
    y = O.observe(obs, O.ParticleSet(equilibrium))
    mt = (50 / 51) ** 2
    R = np.hypot(equilibrium["x"], equilibrium["y"])
    for p in range(15):
        def col(Rr):
            return 2 * integrate.quad(
                lambda z: synth.hernquist_density(math.hypot(Rr, z)) *
                synth.hernquist_sigma2_iso(math.hypot(Rr, z)), 0, math.sqrt(2500 - Rr * Rr))[0] / mt
        m = integrate.quad(lambda Rr: 2 * math.pi * Rr * col(Rr), edges[p], edges[p + 1])[0]
        sel = (R >= edges[p]) & (R < edges[p + 1])
        err = np.std(equilibrium["vz"] ** 2 * sel) * math.sqrt(len(R)) / len(R)
        assert abs(y[p] - m) < 5 * err, p


# ---------------------------------------------------------------- priors

@pytest.mark.parametrize("E", [-0.99, -0.7, -0.3, -0.05, -0.001])
def test_circular_L_hernquist_closed_form(E):
    """E_c = -(u+1)/(2u^2), u = r+1 -> u = (-1 - sqrt(1-8E))/(4E); Lc = r^{3/2}/(r+1)."""
    u = (-1 - math.sqrt(1 - 8 * E)) / (4 * E)
    r = u - 1
    assert O.circular_L(HERN, E) == pytest.approx(r ** 1.5 / (r + 1), rel=1e-12)


def test_circular_L_other_potentials_by_root_finding():
    def ec_log(R):  # spherical log, q = 1: phi = 0.5 ln(1+R^2), v_c^2 = R^2/(1+R^2)
        return 0.5 * math.log(1 + R * R) + 0.5 * R * R / (1 + R * R)
    pot = dict(kind="log", v0=1.0, r0=1.0, q=0.8)  # the equatorial plane does not see q
    for E in (0.05, 0.7, 2.0):
        R = optimize.brentq(lambda R: ec_log(R) - E, 1e-9, 1e6, xtol=1e-15, rtol=1e-15)
        assert O.circular_L(pot, E) == pytest.approx(R * R / math.sqrt(1 + R * R), rel=1e-11)

    def menc(r):
        return r * r / (r + 1) ** 2 + MS * (math.log1p(r / 8) - r / (8 + r))

    def phi_n(r):
        return -1 / (r + 1) - MS * math.log1p(r / 8) / r

    for E in (-2.5, -1.5, -0.6):
        R = optimize.brentq(lambda r: phi_n(r) + 0.5 * menc(r) / r - E, 1e-9, 1e6, xtol=1e-15, rtol=1e-15)
        assert O.circular_L(HNFW, E) == pytest.approx(math.sqrt(R * menc(R)), rel=1e-10)


def test_cells_of_special_orbits():
    pri = dict(mode="mpr", nE=30, nx=10, e_spacing="logneg", signed_lz=0, Emin=-1.0, Emax=-1 / 51,
               update_every=25)
    r = 2.0
    vc = math.sqrt(r) / (r + 1)
    E_circ = -1 / (r + 1) + 0.5 * vc * vc
    k = int(math.floor(math.log(-E_circ) / math.log(1 / 51) * 30))
    parts = _parts([[r, 0.0, 0.0], [0.0, r, 0.0], [0.0, 0.0, 0.5], [0.0, 0.0, 0.0], [vc, 0.0, 0.0],
                    [0.0, vc, 0.0], [1.0, 1.0, 1.0]])
    # particle 0: circular (x = 1 -> top bin); particle 1: radial (x = 0)
    parts["vx"][1], parts["vy"][1], parts["vz"][1] = 0.0, vc, 0.0
    c, E, xc = O.cells(HERN, pri, O.ParticleSet(parts))
    assert xc[0] == pytest.approx(1.0, abs=1e-12) and c[0] == k * 10 + 9
    assert xc[1] == 0.0 and c[1] == k * 10
    # particle 2: at rest at r = 0.5 -> E = phi = -2/3, x = 0
    assert E[2] == pytest.approx(-2 / 3, rel=1e-15)
    assert c[2] == int(math.floor(math.log(2 / 3) / math.log(1 / 51) * 30)) * 10
    # signed-Lz variant: counter-rotating circular orbit -> x = -1 -> bin 0
    pri_s = dict(pri, signed_lz=1)
    parts["vy"][0] = -vc
    c2, _, xc2 = O.cells(HERN, pri_s, O.ParticleSet(parts))
    assert xc2[0] == pytest.approx(-1.0, abs=1e-12) and c2[0] == k * 10
    # co-rotating circular orbit -> x = +1 -> top bin; radial orbit -> x = 0 -> middle bin
    parts["vy"][0] = vc
    c3, _, xc3 = O.cells(HERN, pri_s, O.ParticleSet(parts))
    assert xc3[0] == pytest.approx(1.0, abs=1e-12) and c3[0] == k * 10 + 9
    assert xc3[1] == 0.0 and c3[1] == k * 10 + 5
    # an orbit with Lz = 0.3 Lc: x = 0.3 -> signed bin floor(1.3/2*10) = 6, unsigned bin 3
    parts["vx"][0], parts["vy"][0], parts["vz"][0] = 0.0, 0.3 * vc, math.sqrt(1 - 0.09) * vc
    c4, _, xc4 = O.cells(HERN, pri_s, O.ParticleSet(parts))
    assert xc4[0] == pytest.approx(0.3, rel=1e-12) and c4[0] == k * 10 + 6
    c5, _, xc5 = O.cells(HERN, pri, O.ParticleSet(parts))
    assert xc5[0] == pytest.approx(1.0, rel=1e-12) and c5[0] == k * 10 + 9


# ---------------------------------------------------------------- the step

def _small_run(n=400, mode="mpr", **par):
    groups = [Group("annuli", ["mass"], [0.01], edges=np.exp(np.linspace(math.log(0.1), math.log(10), 9))),
              Group("annuli", ["v2", "gh4"], [0.02, 0.02], edges=np.exp(np.linspace(math.log(0.2), math.log(4), 5)))]
    model = synth.realise_spherical(5, n, synth.hernquist_sigma2_iso)
    target = synth.realise_spherical(6, 20_000, synth.hernquist_sigma2_iso)
    obs = O.ObsSet(groups)
    err = np.concatenate([np.full(8, 0.01), np.full(4, 0.02), np.full(4, 0.02)])
    Y, sig, _ = O.build_targets(obs, O.ParticleSet(target), err)
    pri = dict(mode=mode, nE=6, nx=4, e_spacing="logneg", signed_lz=0, Emin=-1.0, Emax=-1 / 51,
               update_every=5)
    p = dict(dt=0.01, eps=1e-4, mu=1e-2, alpha=0.1, renormalize=1, update_rule="exp", n_relax=0)
    p.update(par)
    return obs, Y, sig, pri, p, model


@pytest.mark.parametrize("mode", ["mpr", "gwr"])
def test_fixed_point_when_data_are_the_models_own_observables(mode):
    """At Y = y(0) with frozen orbits (dt = 0) the data term vanishes (Delta = 0), and
    with equal weights of 2^-9 every cell mean equals the weight exactly, so the MPR
    entropy term -ln(w/what) vanishes too: the force of change of eq. modFOC is exactly
    zero for every particle after the first prior update. (With dt = 0 the update itself
    is the identity whatever the force, so the force is checked directly.) GWR keeps its
    -1 of eq. entropy and a flat prior W0/N = w: F = -mu exactly. A positive control
    moves one target value by one sigma: the force is then non-zero."""
    obs, _, sig, pri, p, model = _small_run(mode=mode)
    n = len(model["w"])
    model = dict(model, w=np.full(n, 2.0 ** -9))
    Y0 = O.observe(obs, O.ParticleSet(model))
    p.update(dt=0.0, eps=1.0, mu=5.0)
    run = O.Run(HERN, obs, Y0, sig, pri, p, model)
    w0 = run.w.copy()
    assert run.step(1) == 0  # t = 1: push (frozen), observe, priors
    assert run.chi2 == 0.0 and np.all(run.delta == 0.0)
    if mode == "mpr":
        assert np.all(run.what == 2.0 ** -9)
    F = np.array([run.force(i) for i in range(n)])
    assert np.all(F == (0.0 if mode == "mpr" else -5.0)), F[:5]
    assert run.step(29) == 0
    assert np.array_equal(run.w, w0)
    # positive control: one observable off by one sigma
    Y1 = Y0.copy()
    Y1[3] += sig[3]
    run1 = O.Run(HERN, obs, Y1, sig, pri, p, model)
    assert run1.step(1) == 0
    F1 = np.array([run1.force(i) for i in range(n)])
    assert np.count_nonzero(F1 != F) > 0


def test_renormalisation_preserves_total_weight():
    obs, Y, sig, pri, p, model = _small_run(eps=3e-3)
    run = O.Run(HERN, obs, Y, sig, pri, p, model)
    assert run.step(60) == 0
    assert not np.allclose(run.w, run.w[0])  # weights did move
    assert run.w.sum() == pytest.approx(run.W0, rel=1e-14)


@pytest.mark.parametrize("mode", ["mpr", "gwr"])
def test_force_of_change_is_gradient_of_merit(mode):
    """With alpha = 1 (ytil = y) and priors held fixed, the bracket of eq. modFOC equals
    dF/dw_i for F = -chi^2/2 + mu S, S from eq. S+ (MPR) or eq. entropy (GWR),
    checked by central differences of F computed from observe()."""
    obs, Y, sig, pri, p, model = _small_run(n=120, mode=mode, alpha=1.0, mu=0.7, n_relax=1)
    rng = np.random.default_rng(2)
    model["w"] = model["w"] * rng.uniform(0.5, 1.5, len(model["w"]))
    run = O.Run(HERN, obs, Y, sig, pri, p, model)
    assert run.step(1) == 0  # push, observe, priors; no weight update (relaxation step)
    what = run.what.copy()
    base = {k: run.ps[k].copy() for k in ("x", "y", "z", "vx", "vy", "vz", "w")}

    def merit(w):
        ps = O.ParticleSet(dict(base, w=w))
        y = O.observe(obs, ps)
        chi2 = np.sum(((y - Y) / sig) ** 2)
        if mode == "mpr":
            S = -np.sum(w * (np.log(w / what) - 1))
        else:
            S = -np.sum(w * np.log(w / what))
        return -0.5 * chi2 + p["mu"] * S

    for i in range(0, 120, 7):
        h = 1e-3 * base["w"][i]  # chi^2 is quadratic in w: central differences are exact for it
        wp, wm = base["w"].copy(), base["w"].copy()
        wp[i] += h
        wm[i] -= h
        grad = (merit(wp) - merit(wm)) / (2 * h)
        assert run.force(i) == pytest.approx(grad, rel=1e-6, abs=1e-6 * (abs(grad) + 1))


def _no_data_run(mode, renorm):
    # one aperture far outside the system: K = 0 for every particle, y = Y = 0
    groups = [Group("annuli", ["mass"], [1.0], edges=np.array([1e5, 2e5]))]
    obs = O.ObsSet(groups)
    model = synth.realise_spherical(8, 300, synth.hernquist_sigma2_iso)
    model["w"] = model["w"] * np.random.default_rng(1).uniform(0.2, 3.0, 300)
    pri = dict(mode=mode, nE=5, nx=3, e_spacing="logneg", signed_lz=0, Emin=-1.0, Emax=-1 / 51,
               update_every=10)
    p = dict(dt=0.01, eps=1.0, mu=5.0, alpha=0.1, renormalize=renorm, update_rule="exp", n_relax=0)
    return O.Run(HERN, obs, np.zeros(1), np.ones(1), pri, p, model)


def test_gwr_entropy_drives_weights_to_prior_over_e():
    """Without data, maximising S = -sum w ln(w/what) gives w = what/e (Sec. 2.2)."""
    run = _no_data_run("gwr", 0)
    assert run.step(600) == 0
    assert np.allclose(run.w, run.W0 / 300 / math.e, rtol=1e-9)


def test_mpr_entropy_drives_weights_to_cell_means():
    """Without data, eq. S+ pulls every weight to the moving prior of its cell, so the
    weights become equal within cells while cells keep different values (Sec. 2.3)."""
    run = _no_data_run("mpr", 0)
    assert run.step(1000) == 0
    for c in np.unique(run.cell):
        wc = run.w[run.cell == c]
        assert np.ptp(wc) <= 1e-6 * wc.mean()
    assert np.unique(np.round(run.w, 12)).size > 3
    # weights in a cell are exactly at the current cell prior
    assert np.allclose(run.w, run.what, rtol=1e-6)


def test_smoothing_and_residuals_closed_form():
    """Force-free straight-line motion (M = 0) of one particle across an annulus edge:
    the smoothed mass observable decays as (1-alpha)^k after the crossing (eq. myts),
    and chi^2 follows from eq. delta."""
    edges = np.array([0.5, 1.0, 2.0])
    obs = O.ObsSet([Group("annuli", ["mass"], [0.1], edges=edges)])
    model = _parts([[0.905], [0.0], [0.0], [0.01], [0.0], [0.0], [1.0]])
    alpha = 0.15
    pri = dict(mode="gwr", nE=1, nx=1, e_spacing="linear", signed_lz=0, Emin=-1, Emax=0, update_every=1)
    p = dict(dt=1.0, eps=0.0, mu=0.0, alpha=alpha, renormalize=0, update_rule="exp", n_relax=0)
    Y = np.array([0.2, 0.05])
    sig = np.array([0.1, 0.02])
    run = O.Run(dict(kind="hernquist", G=1.0, M=0.0, a=1.0), obs, Y, sig, pri, p, model)
    a0 = math.pi * (1.0 - 0.25)
    a1 = math.pi * (4.0 - 1.0)
    for t in range(1, 25):
        run.step(1)
        x = 0.905 + 0.01 * t
        if x < 1.0:
            e0, e1 = 1 / a0, 0.0
        else:
            k = t - 9  # first step past the edge is t = 10
            e0 = (1 / a0) * (1 - alpha) ** k
            e1 = (1 / a1) * (1 - (1 - alpha) ** k)
        assert run.ytil == pytest.approx([e0, e1], rel=1e-13, abs=1e-15)
        assert run.chi2 == pytest.approx(((e0 - 0.2) / 0.1) ** 2 + ((e1 - 0.05) / 0.02) ** 2, rel=1e-12)


def test_zero_weight_is_a_fixed_point():
    obs, Y, sig, pri, p, model = _small_run(eps=1e-3)
    model["w"][3] = 0.0
    run = O.Run(HERN, obs, Y, sig, pri, p, model)
    assert run.step(20) == 0
    assert run.w[3] == 0.0 and np.all(np.isfinite(run.w))


def test_euler_rule_reports_negative_weight():
    """Explicit Euler with a large eps dt drives weights negative; the oracle reports it."""
    obs, Y, sig, pri, p, model = _small_run(eps=5.0, update_rule="euler")
    run = O.Run(HERN, obs, Y, sig, pri, p, model)
    assert run.step(5) == 2


# ---------------------------------------------------------------- targets

def test_target_fit_on_gaussian_losvd():
    """Velocities N(0.3, 0.5^2) independent of position: each aperture's LOSVD is Gaussian,
    so the h1 = h2 = 0 iteration (eq. h1h2) recovers V = 0.3, sigma = 0.5 and h3, h4 ~ 0
    within sampling error, and ends with b1 = b2 = 0 to 1e-12."""
    n = 100_000
    rng_pos = synth.realise_spherical(21, n, synth.hernquist_sigma2_iso)
    g = synth.normal(22, 0, n)
    p = dict(rng_pos, vz=0.3 + 0.5 * g)
    groups = [Group("annuli", ["gh1", "gh2", "gh3", "gh4"], [0.01] * 4,
                    edges=np.exp(np.linspace(math.log(0.2), math.log(5), 6)))]
    obs = O.ObsSet(groups)
    Y, sig, iters = O.build_targets(obs, O.ParticleSet(p), np.full(20, 0.01))
    assert 1 <= iters < 100
    npp = Y[:5] / sig[:5] * 0.01  # luminosity per aperture * n ~ count
    lum = sig[:5] / 0.01
    cnt = lum * n
    assert np.all(np.abs(obs.Vp - 0.3) < 5 * 0.5 / np.sqrt(cnt))
    assert np.all(np.abs(obs.sp - 0.5) < 5 * 0.5 / np.sqrt(2 * cnt))
    assert np.allclose(Y[:10], 0.0, atol=1e-12 * lum.max())
    h34 = Y[10:] / np.concatenate([lum, lum])
    assert np.all(np.abs(h34) < 5 / np.sqrt(np.concatenate([cnt, cnt])))
    del npp


def test_jeans_closed_form_matches_quadrature():
    tab = synth.jeans_sigma2_table(synth.hernquist_density, synth.hernquist_mass)
    r = np.array([1e-3, 0.05, 0.5, 2.0, 10.0, 45.0])
    assert np.allclose(synth.sigma2_from_table(tab, r), synth.hernquist_sigma2_iso(r), rtol=2e-5)


def test_target_errors_propagate_from_the_stated_error_variables():
    """sigma(Y) follows from the stated error on each observable's own variable:
    mass: err * Sigma; v2 = l v_rms^2: |dY/dv_rms| err v_rms; GH b_n = l h_n: l err.
    With noise g, the noisy value moves by err*g in that variable."""
    tp = synth.realise_spherical(31, 50_000, synth.hernquist_sigma2_iso)
    edges = np.exp(np.linspace(math.log(0.2), math.log(4), 5))
    groups = [Group("annuli", ["mass", "v2", "gh4"], [0.01, 0.03, 0.02], edges=edges)]
    err = np.concatenate([np.full(4, 0.01), np.full(4, 0.03), np.full(4, 0.02)])
    obs = O.ObsSet(groups)
    Y, sig, _ = O.build_targets(obs, O.ParticleSet(tp), err)
    area = math.pi * (edges[1:] ** 2 - edges[:-1] ** 2)
    lum = Y[:4] * area
    vrms = np.sqrt(Y[4:8] / lum)
    dv = 1e-6 * vrms
    dY = (lum * (vrms + dv) ** 2 - lum * (vrms - dv) ** 2) / (2 * dv)
    assert np.allclose(sig[:4], 0.01 * Y[:4], rtol=1e-14)
    assert np.allclose(sig[4:8], dY * 0.03 * vrms, rtol=1e-8)
    assert np.allclose(sig[8:], lum * 0.02, rtol=1e-12)
    g = np.linspace(-1.5, 1.5, 12)
    obs2 = O.ObsSet(groups)
    Yn, sign, _ = O.build_targets(obs2, O.ParticleSet(tp), err, g)
    assert np.allclose(sign, sig, rtol=1e-14)
    assert np.allclose(Yn[:4], Y[:4] * (1 + 0.01 * g[:4]), rtol=1e-13)
    assert np.allclose(np.sqrt(Yn[4:8] / lum), vrms * (1 + 0.03 * g[4:8]), rtol=1e-12)
    assert np.allclose(Yn[8:] / lum, Y[8:] / lum + 0.02 * g[8:], rtol=1e-12, atol=1e-14)
