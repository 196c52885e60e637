"""CPU FP64 oracle of the chi^2 M2M step with moving priors (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import this
package. It wraps the plain C implementation in m2m_oracle.c through ctypes; the
C file is compiled by `build()` with gcc into oracle/_build/liboracle.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# M2M_ORACLE_SO names a library built elsewhere (the mutation test of the pins loads
# deliberately broken copies of the oracle this way); it is then used as it is.
_SO = os.environ.get("M2M_ORACLE_SO") or os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MAX_GROUPS = 4
MAX_KINDS = 16
POT = {"hernquist": 0, "hernquist_nfw": 1, "log": 2, "scf": 3}
GEOM = {"annuli": 0, "pixels": 1, "shells": 2}
MODE = {"gwr": 0, "mpr": 1}
ESPACING = {"logneg": 0, "exp": 1, "linear": 2}
RULE = {"exp": 0, "euler": 1}


def kind_code(name: str) -> int:
    if name == "mass":
        return 0
    if name == "v2":
        return 1
    if name.startswith("gh"):
        return 10 + int(name[2:])
    if name.startswith("alm_"):  # alm_<l>_<m>: coefficient of the real Y_lm on shells
        l, m = (int(v) for v in name[4:].split("_"))
        return 100 + l * (l + 1) + m
    raise ValueError(name)


def build(force: bool = False) -> str:
    """Compile the oracle C source into a shared library (gcc, -ffp-contract=off)."""
    src = os.path.join(_HERE, "m2m_oracle.c")
    if os.environ.get("M2M_ORACLE_SO"):
        return _SO
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "m2m_oracle.h"))):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                        "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int), ("G", C.c_double), ("M", C.c_double), ("a", C.c_double),
                ("Ms", C.c_double), ("rs", C.c_double), ("v0", C.c_double), ("r0", C.c_double),
                ("q", C.c_double), ("scf_n", C.c_int), ("scf_lmax", C.c_int),
                ("scf_r", C.POINTER(C.c_double)), ("scf_a", C.POINTER(C.c_double)),
                ("scf_ups", C.POINTER(C.c_double))]


class Group(C.Structure):
    _fields_ = [("geometry", C.c_int), ("n_ap", C.c_int), ("edges", C.POINTER(C.c_double)),
                ("nx", C.c_int), ("ny", C.c_int), ("xlo", C.c_double), ("xhi", C.c_double),
                ("ylo", C.c_double), ("yhi", C.c_double), ("n_kinds", C.c_int),
                ("kinds", C.c_int * MAX_KINDS), ("Vp", C.POINTER(C.c_double)),
                ("sp", C.POINTER(C.c_double))]


class Obs(C.Structure):
    _fields_ = [("incl_deg", C.c_double), ("n_groups", C.c_int), ("g", Group * MAX_GROUPS)]


class Prior(C.Structure):
    _fields_ = [("mode", C.c_int), ("nE", C.c_int), ("nx", C.c_int), ("e_spacing", C.c_int),
                ("signed_lz", C.c_int), ("update_every", C.c_int), ("Emin", C.c_double),
                ("Emax", C.c_double), ("smoothing", C.c_int), ("lam", C.c_double),
                ("window_E", C.c_int), ("window_x", C.c_int)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("eps", C.c_double), ("mu", C.c_double),
                ("alpha", C.c_double), ("renormalize", C.c_int), ("update_rule", C.c_int),
                ("n_relax", C.c_long), ("eps_ups", C.c_double)]


_DP = C.POINTER(C.c_double)
_LP = C.POINTER(C.c_long)
_IP = C.POINTER(C.c_int)


class SphGrid(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_phi", C.c_int), ("n_ct", C.c_int), ("r_min", C.c_double),
                ("r_max", C.c_double)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_long)] + [(k, _DP) for k in ("x", "y", "z", "vx", "vy", "vz", "w")]


class State(C.Structure):
    _fields_ = [("cell", C.POINTER(C.c_int)), ("what", _DP), ("grid_mean", _DP),
                ("grid_count", C.POINTER(C.c_long)), ("ytil", _DP), ("yraw", _DP),
                ("delta", _DP), ("chi2", C.c_double), ("W0", C.c_double), ("t", C.c_long),
                ("grid_raw", _DP), ("lam", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        L.or_phi.restype = C.c_double
        L.or_phi.argtypes = [C.POINTER(Potential), C.c_double, C.c_double, C.c_double]
        L.or_accel.argtypes = [C.POINTER(Potential), C.c_double, C.c_double, C.c_double, _DP, _DP, _DP]
        L.or_leapfrog.argtypes = [C.POINTER(Potential), C.POINTER(Particles), C.c_double]
        L.or_hermite.restype = C.c_double
        L.or_hermite.argtypes = [C.c_int, C.c_double]
        L.or_gh_kernel.restype = C.c_double
        L.or_gh_kernel.argtypes = [C.c_int, C.c_double]
        L.or_num_obs.argtypes = [C.POINTER(Obs)]
        L.or_kernel_matrix.argtypes = [C.POINTER(Obs), C.POINTER(Particles), _DP]
        L.or_observe.argtypes = [C.POINTER(Obs), C.POINTER(Particles), _DP]
        L.or_circular_L.restype = C.c_double
        L.or_circular_L.argtypes = [C.POINTER(Potential), C.c_double]
        L.or_cell.argtypes = [C.POINTER(Potential), C.POINTER(Prior)] + [C.c_double] * 6 + [_DP, _DP]
        L.or_force.restype = C.c_double
        L.or_force.argtypes = [C.POINTER(Obs), C.POINTER(Params), C.c_int, C.c_double, C.c_double] + \
            [C.c_double] * 6 + [_DP, _DP]
        L.or_init.argtypes = [C.POINTER(Obs), _DP, _DP, C.POINTER(Prior), C.POINTER(Particles),
                              C.POINTER(State)]
        L.or_run.argtypes = [C.POINTER(Potential), C.POINTER(Obs), _DP, _DP, C.POINTER(Prior),
                             C.POINTER(Params), C.POINTER(Particles), C.POINTER(State), C.c_long]
        L.or_window_means.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _DP, C.POINTER(C.c_long), _DP]
        L.or_smooth_penalty.argtypes = [C.c_int, C.c_int, _DP]
        L.or_smooth_grid.argtypes = [C.c_int, C.c_int, _DP, C.c_double, _DP, _DP]
        L.or_smooth_grid.restype = C.c_int
        L.or_smooth_gcv.argtypes = [C.c_int, C.c_int, _DP, C.c_double, _DP]
        L.or_scf_coeffs.argtypes = [C.POINTER(Potential), C.POINTER(Particles), _DP]
        L.or_scf_phi.argtypes = [C.POINTER(Potential), C.c_double, C.c_double, C.c_double, _DP]
        L.or_scf_phi.restype = C.c_double
        L.or_observe_dlnups.argtypes = [C.POINTER(Obs), C.POINTER(Particles), _DP]
        L.or_smooth_gcv.restype = C.c_int
        L.or_ylm.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_ylm.restype = C.c_double
        L.or_sph_bin.argtypes = [C.POINTER(SphGrid), C.c_double, C.c_double, C.c_double]
        L.or_sph_velocity.argtypes = [C.c_double] * 6 + [_DP, _DP, _DP]
        L.or_kin_sums.argtypes = [C.POINTER(SphGrid), C.POINTER(Particles), _DP, _LP]
        L.or_kin_moments.argtypes = [C.c_long, _DP, _LP, C.c_long, _DP, _DP, _IP]
        L.or_delta_kin.argtypes = [C.c_long, _DP, _LP, _DP, _LP, C.c_long, _DP]
        L.or_delta_kin.restype = C.c_long
        L.or_grid_weights.argtypes = [C.POINTER(Potential), C.POINTER(Prior), C.POINTER(Particles), _DP, _DP, _LP]
        L.or_delta_grid.argtypes = [C.c_int, _DP, _DP]
        L.or_delta_grid.restype = C.c_double
        L.or_weight_rms.argtypes = [C.c_int, _DP, _LP, C.c_long]
        L.or_weight_rms.restype = C.c_double
        L.or_build_targets.argtypes = [C.POINTER(Obs), C.POINTER(Particles), _DP, _DP, _DP, _DP,
                                       _DP, _DP, C.POINTER(C.c_int)]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------------------
# descriptor builders (from plain dicts / workload objects)
# ---------------------------------------------------------------------------

def potential(d: dict) -> Potential:
    """The C descriptor of a potential dict. The self-consistent kind ("scf") carries its
    grid radii scf_r, scf_lmax and the initial ups (mass-to-light ratio); its coefficient
    array and Upsilon are owned by the returned object (attributes a and ups)."""
    P = Potential(POT[d["kind"]], d.get("G", 1.0), d.get("M", 1.0), d.get("a", 1.0),
                  d.get("Ms", 0.0), d.get("rs", 1.0), d.get("v0", 0.0), d.get("r0", 1.0),
                  d.get("q", 1.0))
    if d["kind"] == "scf":
        r = np.ascontiguousarray(d["scf_r"], np.float64)
        L = int(d["scf_lmax"])
        P._keep = (r, np.zeros(len(r) * (L + 1) ** 2), np.array([float(d.get("ups", 1.0))]))
        P.scf_n, P.scf_lmax = len(r), L
        P.scf_r, P.scf_a, P.scf_ups = _dp(P._keep[0]), _dp(P._keep[1]), _dp(P._keep[2])
    return P


def scf_coeffs(pot: dict, particles: dict) -> np.ndarray:
    """a_lm,k of the particles' weights on the grid of a self-consistent potential
    (or_scf_coeffs), shape (n, (lmax+1)^2)."""
    P = potential(pot)
    a = np.zeros((P.scf_n, (P.scf_lmax + 1) ** 2))
    lib().or_scf_coeffs(C.byref(P), C.byref(ParticleSet(particles).s), _dp(a))
    return a


def scf_field(pot: dict, a: np.ndarray, x, y, z):
    """(phi_star, grad phi_star) at a point from coefficients a (or_scf_phi, without Upsilon)."""
    P = potential(pot)
    a = np.ascontiguousarray(a, np.float64)
    P.scf_a = _dp(a)
    g = np.zeros(3)
    phi = lib().or_scf_phi(C.byref(P), x, y, z, _dp(g))
    return phi, g


def observe_dlnups(obs, ps) -> np.ndarray:
    """D_j = d y_j / d ln Upsilon with velocities scaling as Upsilon^(1/2) (or_observe_dlnups)."""
    D = np.zeros(obs.J)
    lib().or_observe_dlnups(C.byref(obs.o), C.byref(ps.s), _dp(D))
    return D


class ObsSet:
    """Observable descriptor; keeps the numpy arrays it points into alive."""

    def __init__(self, groups, incl_deg=0.0, Vp=None, sp=None):
        self.groups = groups
        self.o = Obs()
        self.o.incl_deg = incl_deg
        self.o.n_groups = len(groups)
        self._keep = []
        self.n_ap_total = sum(g.n_ap for g in groups)
        self.Vp = np.zeros(self.n_ap_total) if Vp is None else np.ascontiguousarray(Vp, np.float64)
        self.sp = np.ones(self.n_ap_total) if sp is None else np.ascontiguousarray(sp, np.float64)
        off = 0
        for gi, g in enumerate(groups):
            G = self.o.g[gi]
            G.geometry = GEOM[g.geometry]
            G.n_ap = g.n_ap
            if g.geometry in ("annuli", "shells"):
                e = np.ascontiguousarray(g.edges, np.float64)
                self._keep.append(e)
                G.edges = _dp(e)
            else:
                G.nx, G.ny = g.nx, g.ny
                G.xlo, G.xhi, G.ylo, G.yhi = g.box
            G.n_kinds = len(g.kinds)
            for k, name in enumerate(g.kinds):
                G.kinds[k] = kind_code(name)
            G.Vp = C.cast(self.Vp.ctypes.data + 8 * off, _DP)
            G.sp = C.cast(self.sp.ctypes.data + 8 * off, _DP)
            off += g.n_ap
        self.J = lib().or_num_obs(C.byref(self.o))


def prior(d: dict) -> Prior:
    wE, wx = d.get("window", (0, 0))
    return Prior(MODE[d["mode"]], d["nE"], d["nx"], ESPACING[d["e_spacing"]], d["signed_lz"],
                 d["update_every"], d["Emin"], d["Emax"], int(d.get("smoothing", 0)), float(d.get("lambda", 0.0)),
                 int(wE), int(wx))


def params(d: dict) -> Params:
    return Params(d["dt"], d["eps"], d["mu"], d["alpha"], d["renormalize"], RULE[d["update_rule"]],
                  d["n_relax"], d.get("eps_ups", 0.0))


class ParticleSet:
    """Oracle particle arrays (float64 copies) and their ctypes view."""

    def __init__(self, p: dict):
        self.a = {k: np.array(p[k], dtype=np.float64, copy=True) for k in
                  ("x", "y", "z", "vx", "vy", "vz", "w")}
        self.s = Particles(len(self.a["x"]), *[_dp(self.a[k]) for k in
                                               ("x", "y", "z", "vx", "vy", "vz", "w")])

    def __getitem__(self, k):
        return self.a[k]


# ---------------------------------------------------------------------------
# functions
# ---------------------------------------------------------------------------

def phi(pot: dict, x, y, z) -> float:
    P = potential(pot)
    return lib().or_phi(C.byref(P), x, y, z)


def accel(pot: dict, x, y, z):
    P = potential(pot)
    a = [C.c_double(), C.c_double(), C.c_double()]
    lib().or_accel(C.byref(P), x, y, z, *[C.byref(v) for v in a])
    return np.array([v.value for v in a])


def leapfrog(pot: dict, ps: ParticleSet, dt: float):
    P = potential(pot)
    lib().or_leapfrog(C.byref(P), C.byref(ps.s), dt)


def hermite(n: int, x: float) -> float:
    return lib().or_hermite(n, x)


def gh_kernel(n: int, nu: float) -> float:
    return lib().or_gh_kernel(n, nu)


def kernel_matrix(obs: ObsSet, ps: ParticleSet) -> np.ndarray:
    K = np.zeros((ps.s.n, obs.J))
    lib().or_kernel_matrix(C.byref(obs.o), C.byref(ps.s), _dp(K))
    return K


def observe(obs: ObsSet, ps: ParticleSet) -> np.ndarray:
    y = np.zeros(obs.J)
    lib().or_observe(C.byref(obs.o), C.byref(ps.s), _dp(y))
    return y


def circular_L(pot: dict, E: float) -> float:
    P = potential(pot)
    return lib().or_circular_L(C.byref(P), E)


def cells(pot: dict, pri: dict, ps: ParticleSet):
    P, G = potential(pot), prior(pri)
    n = ps.s.n
    c = np.zeros(n, np.int64)
    E = np.zeros(n)
    xc = np.zeros(n)
    e, xx = C.c_double(), C.c_double()
    a = ps.a
    for i in range(n):
        c[i] = lib().or_cell(C.byref(P), C.byref(G), a["x"][i], a["y"][i], a["z"][i],
                             a["vx"][i], a["vy"][i], a["vz"][i], C.byref(e), C.byref(xx))
        E[i], xc[i] = e.value, xx.value
    return c, E, xc


def build_targets(obs: ObsSet, target: ParticleSet, err: np.ndarray, noise=None):
    """Target Y, sigma, and the fitted per-aperture V_p, sigma_p (written into obs)."""
    J = obs.J
    err = np.ascontiguousarray(err, np.float64)
    Y = np.zeros(J)
    sig = np.zeros(J)
    it = C.c_int()
    nz = None if noise is None else np.ascontiguousarray(noise, np.float64)
    rc = lib().or_build_targets(C.byref(obs.o), C.byref(target.s), _dp(err),
                                None if nz is None else _dp(nz), _dp(obs.Vp), _dp(obs.sp),
                                _dp(Y), _dp(sig), C.byref(it))
    if rc != 0:
        raise RuntimeError(f"oracle target construction failed ({rc})")
    # the C routine re-points the group Vp/sp into the same arrays
    return Y, sig, it.value


class Run:
    """A whole oracle M2M run: particles, targets, priors and smoothed observables."""

    def __init__(self, pot: dict, obs: ObsSet, Y, sig, pri: dict, par: dict, particles: dict):
        self.P = potential(pot)
        self.obs = obs
        self.Y = np.ascontiguousarray(Y, np.float64)
        self.sig = np.ascontiguousarray(sig, np.float64)
        self.G = prior(pri)
        # the rate of the mass-to-light update travels with the self-consistent potential
        self.par = params(dict(par, eps_ups=pot.get("eps_ups", 0.0)))
        self.ps = ParticleSet(particles)
        n = self.ps.s.n
        J = obs.J
        ncell = pri["nE"] * pri["nx"]
        self.cell = np.zeros(n, np.int32)
        self.what = np.zeros(n)
        self.grid_mean = np.zeros(max(ncell, 1))
        self.grid_count = np.zeros(max(ncell, 1), np.int64)
        self.ytil = np.zeros(J)
        self.yraw = np.zeros(J)
        self.delta = np.zeros(J)
        self.grid_raw = np.zeros(max(ncell, 1))
        self.st = State(self.cell.ctypes.data_as(C.POINTER(C.c_int)), _dp(self.what),
                        _dp(self.grid_mean), self.grid_count.ctypes.data_as(C.POINTER(C.c_long)),
                        _dp(self.ytil), _dp(self.yraw), _dp(self.delta), 0.0, 0.0, 0,
                        _dp(self.grid_raw), 0.0)
        lib().or_init(C.byref(obs.o), _dp(self.Y), _dp(self.sig), C.byref(self.G),
                      C.byref(self.ps.s), C.byref(self.st))

    def step(self, n: int) -> int:
        return lib().or_run(C.byref(self.P), C.byref(self.obs.o), _dp(self.Y), _dp(self.sig),
                            C.byref(self.G), C.byref(self.par), C.byref(self.ps.s),
                            C.byref(self.st), n)

    @property
    def chi2(self) -> float:
        return self.st.chi2

    @property
    def t(self) -> int:
        return self.st.t

    @property
    def W0(self) -> float:
        return self.st.W0

    @property
    def ups(self) -> float:
        """Mass-to-light ratio of a self-consistent potential."""
        return float(self.P._keep[2][0])

    @property
    def scf_a(self) -> np.ndarray:
        """Current expansion coefficients of a self-consistent potential, (n, (lmax+1)^2)."""
        return self.P._keep[1].reshape(self.P.scf_n, -1)

    @property
    def lam(self) -> float:
        """Smoothing weight of the last prior update (prior smoothing on)."""
        return self.st.lam

    @property
    def w(self) -> np.ndarray:
        return self.ps.a["w"]

    def force(self, i: int) -> float:
        a = self.ps.a
        return lib().or_force(C.byref(self.obs.o), C.byref(self.par), self.G.mode, a["w"][i],
                              self.what[i], a["x"][i], a["y"][i], a["z"][i], a["vx"][i],
                              a["vy"][i], a["vz"][i], _dp(self.delta), _dp(self.sig))


def window_means(wsum, count, hE: int, hx: int) -> np.ndarray:
    """Moving-window means of a (nE, nx) grid of weight sums and counts (or_window_means)."""
    wsum = np.ascontiguousarray(wsum, np.float64)
    count = np.ascontiguousarray(count, np.int64)
    nE, nx = wsum.shape
    out = np.zeros((nE, nx))
    lib().or_window_means(nE, nx, hE, hx, _dp(wsum), count.ctypes.data_as(C.POINTER(C.c_long)), _dp(out))
    return out


def smooth_penalty(nE: int, nx: int) -> np.ndarray:
    """The finite-difference penalty matrix of the prior grid (or_smooth_penalty)."""
    P = np.zeros((nE * nx, nE * nx))
    lib().or_smooth_penalty(nE, nx, _dp(P))
    return P


def smooth_grid(y, nE: int, nx: int, lam: float = 0.0):
    """(f, lambda): the smoothed grid of eq. smooth_grid; lam <= 0 chooses lambda by GCV."""
    y = np.ascontiguousarray(y, np.float64)
    f = np.zeros_like(y)
    lo = C.c_double()
    rc = lib().or_smooth_grid(nE, nx, _dp(y), lam, _dp(f), C.byref(lo))
    if rc != 0:
        raise RuntimeError(f"or_smooth_grid failed ({rc})")
    return f, lo.value


def smooth_gcv(y, nE: int, nx: int, lam: float) -> float:
    """The GCV score of the smoothed grid at lam > 0 (or_smooth_gcv)."""
    y = np.ascontiguousarray(y, np.float64)
    sc = C.c_double()
    rc = lib().or_smooth_gcv(nE, nx, _dp(y), lam, C.byref(sc))
    if rc != 0:
        raise RuntimeError(f"or_smooth_gcv failed ({rc})")
    return sc.value


def from_workload(wl, target_particles=None):
    """Oracle observable set + targets for a workload (targets built by the oracle)."""
    obs = ObsSet(wl.groups, wl.incl_deg)
    tp = ParticleSet(wl.target if target_particles is None else target_particles)
    Y, sig, _ = build_targets(obs, tp, wl.err_per_obs(), wl.noise)
    return obs, Y, sig


# ---------------------------------------------------------------------------
# diagnostics (Sec. 4.1, Sec. 5)
# ---------------------------------------------------------------------------

KIN_SUMS = 7


def _lp(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(_LP)


def sph_grid(d: dict) -> SphGrid:
    return SphGrid(d["n_r"], d["n_phi"], d["n_ct"], d["r_min"], d["r_max"])


def sph_bin(grid: dict, x, y, z) -> int:
    return lib().or_sph_bin(C.byref(sph_grid(grid)), x, y, z)


def sph_velocity(x, y, z, vx, vy, vz):
    o = [C.c_double(), C.c_double(), C.c_double()]
    lib().or_sph_velocity(x, y, z, vx, vy, vz, *[C.byref(v) for v in o])
    return np.array([v.value for v in o])


def kin_sums(grid: dict, ps: ParticleSet):
    """(sums[nbins, 7], counts[nbins]) of the spherical-bin kinematics."""
    nb = grid["n_r"] * grid["n_phi"] * grid["n_ct"]
    sums = np.zeros(nb * KIN_SUMS)
    cnt = np.zeros(nb, np.int64)
    lib().or_kin_sums(C.byref(sph_grid(grid)), C.byref(ps.s), _dp(sums), _lp(cnt))
    return sums.reshape(nb, KIN_SUMS), cnt


def kin_moments(sums, counts, min_count: int = 1):
    """(mean[nbins, 3], disp[nbins, 3], valid[nbins]) from kin_sums."""
    sums = np.ascontiguousarray(sums, np.float64).ravel()
    counts = np.ascontiguousarray(counts, np.int64)
    nb = len(counts)
    mean, disp = np.zeros(3 * nb), np.zeros(3 * nb)
    valid = np.zeros(nb, np.int32)
    lib().or_kin_moments(nb, _dp(sums), _lp(counts), min_count, _dp(mean), _dp(disp),
                         valid.ctypes.data_as(_IP))
    return mean.reshape(nb, 3), disp.reshape(nb, 3), valid.astype(bool)


def delta_kin(sums_m, counts_m, sums_t, counts_t, min_count: int = 1):
    """(out[7], bins used): rms model-minus-target difference of the six moments, and overall."""
    sm = np.ascontiguousarray(sums_m, np.float64).ravel()
    st = np.ascontiguousarray(sums_t, np.float64).ravel()
    cm = np.ascontiguousarray(counts_m, np.int64)
    ct = np.ascontiguousarray(counts_t, np.int64)
    out = np.zeros(7)
    used = lib().or_delta_kin(len(cm), _dp(sm), _lp(cm), _dp(st), _lp(ct), min_count, _dp(out))
    return out, used


def grid_weights(pot: dict, pri: dict, ps: ParticleSet):
    """(wsum, wdev2, count) per (E, x) cell of the prior grid."""
    nc = pri["nE"] * pri["nx"]
    ws, wd = np.zeros(nc), np.zeros(nc)
    cnt = np.zeros(nc, np.int64)
    P, G = potential(pot), prior(pri)
    lib().or_grid_weights(C.byref(P), C.byref(G), C.byref(ps.s), _dp(ws), _dp(wd), _lp(cnt))
    return ws, wd, cnt


def delta_grid(w_model, w_target) -> float:
    wm = np.ascontiguousarray(w_model, np.float64)
    wt = np.ascontiguousarray(w_target, np.float64)
    return lib().or_delta_grid(len(wm), _dp(wm), _dp(wt))


def weight_rms(wdev2, count, min_count: int = 50) -> float:
    wd = np.ascontiguousarray(wdev2, np.float64)
    cnt = np.ascontiguousarray(count, np.int64)
    return lib().or_weight_rms(len(wd), _dp(wd), _lp(cnt), min_count)


# ---------------------------------------------------------------------------
# spherical-harmonic density coefficients (eq. alm)
# ---------------------------------------------------------------------------

def ylm(l: int, m: int, cos_theta: float, phi: float) -> float:
    """Real spherical harmonic of unit norm, without the Condon-Shortley phase."""
    return lib().or_ylm(l, m, cos_theta, phi)
