"""Python binding of the C ABI in include/m2m.h (ctypes; argument marshalling only).

Every step of the M2M method runs in the CUDA library libm2m.so; this module
only translates Python values into the C descriptors and back. Importing it
does not load the library; the first call does, and raises if the library is
missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_SO = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libm2m.so")
_lib = None

MAX_GROUPS = 4
MAX_KINDS = 16
POT = {"hernquist": 0, "hernquist_nfw": 1, "log": 2, "scf": 3}
GEOM = {"annuli": 0, "pixels": 1, "shells": 2}
MODE = {"gwr": 0, "mpr": 1}
ESPACING = {"logneg": 0, "exp": 1, "linear": 2}
PREC = {"fp64": 0, "mixed": 1}
RULE = {"exp": 0, "euler": 1}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NONFINITE", 5: "ERR_NEG_WEIGHT",
          6: "ERR_OVERFLOW", 7: "ERR_TIMEOUT", 8: "ERR_STATE", 9: "ERR_TARGET"}


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
    raise ValueError(f"unknown observable kind {name!r}")


class M2MError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_DP = C.POINTER(C.c_double)


class Potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("G", C.c_double), ("M", C.c_double), ("a", C.c_double),
                ("Ms", C.c_double), ("rs", C.c_double), ("v0", C.c_double), ("r0", C.c_double),
                ("q", C.c_double), ("scf_n", C.c_int32), ("scf_lmax", C.c_int32), ("scf_r", _DP),
                ("ups", C.c_double), ("eps_ups", C.c_double)]


class ObsGroup(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("n_ap", C.c_int32), ("edges", _DP), ("nx", C.c_int32),
                ("ny", C.c_int32), ("xlo", C.c_double), ("xhi", C.c_double), ("ylo", C.c_double),
                ("yhi", C.c_double), ("n_kinds", C.c_int32), ("kinds", C.c_int32 * MAX_KINDS),
                ("Vp", _DP), ("sp", _DP)]


class Observables(C.Structure):
    _fields_ = [("incl_deg", C.c_double), ("n_groups", C.c_int32), ("groups", ObsGroup * MAX_GROUPS),
                ("Y", _DP), ("sigY", _DP)]


class PriorGrid(C.Structure):
    _fields_ = [("mode", C.c_int32), ("nE", C.c_int32), ("nx", C.c_int32), ("e_spacing", C.c_int32),
                ("signed_lz", C.c_int32), ("update_every", C.c_int32), ("Emin", C.c_double),
                ("Emax", C.c_double), ("smoothing", C.c_int32), ("lam", C.c_double),
                ("window_E", C.c_int32), ("window_x", C.c_int32)]


DEPOSIT = {"auto": 0, "shared": 1, "global": 2}


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("dt", C.c_double), ("renormalize", C.c_int32),
                ("update_rule", C.c_int32), ("n_relax", C.c_int64), ("stream", C.c_void_p),
                ("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("deposit", C.c_int32)]


def library_path() -> str:
    return _SO


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"CUDA library {_SO} is not built; run paper_1202_2355_gb300.build.build()")
        L = C.CDLL(_SO)
        vp = C.c_void_p
        L.m2m_create.argtypes = [C.POINTER(Potential), C.POINTER(Observables), C.POINTER(PriorGrid),
                                 C.c_double, C.c_double, C.c_double, C.POINTER(Options), C.POINTER(vp)]
        L.m2m_load_particles.argtypes = [vp, C.c_int64, _DP, _DP, _DP]
        L.m2m_load_particles_device.argtypes = [vp, C.c_int64, vp, vp, vp]
        L.m2m_step.argtypes = [vp, C.c_int64]
        L.m2m_synchronize.argtypes = [vp]
        L.m2m_get_weights.argtypes = [vp, _DP, C.c_int64]
        L.m2m_get_state.argtypes = [vp, _DP, _DP, C.c_int64]
        L.m2m_get_observables.argtypes = [vp, _DP, _DP, C.c_int32]
        L.m2m_get_chi2.argtypes = [vp, _DP, C.POINTER(C.c_int32), _DP]
        L.m2m_get_priors.argtypes = [vp, _DP, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int64]
        L.m2m_get_step_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.m2m_get_prior_smoothing.argtypes = [vp, _DP, _DP]
        L.m2m_get_particle_count.argtypes = [vp, C.POINTER(C.c_int64)]
        L.m2m_set_timing.argtypes = [vp, C.c_int32]
        L.m2m_get_timing.argtypes = [vp, _DP, C.POINTER(C.c_int64)]
        L.m2m_save_state.argtypes = [vp, C.c_char_p]
        L.m2m_load_state.argtypes = [vp, C.c_char_p]
        L.m2m_build_targets.argtypes = [C.POINTER(Observables), C.c_int64, _DP, _DP, _DP, _DP, _DP,
                                        _DP, _DP, _DP, _DP, C.POINTER(C.c_int32)]
        L.m2m_observe_static.argtypes = [C.POINTER(Observables), C.c_int64, vp, vp, vp, vp, vp]
        L.m2m_observe_static.restype = C.c_int
        L.m2m_last_error.restype = C.c_char_p
        L.m2m_last_error.argtypes = [vp]
        L.m2m_destroy.argtypes = [vp]
        L.m2m_create_batch.argtypes = [C.c_int32, C.POINTER(Potential), C.POINTER(Observables),
                                       C.POINTER(PriorGrid), _DP, _DP, _DP, C.POINTER(Options), C.POINTER(vp)]
        L.m2m_batch_size.argtypes = [vp, C.POINTER(C.c_int32)]
        L.m2m_batch_model.argtypes = [vp, C.c_int32, C.POINTER(vp)]
        L.m2m_batch_autotune.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                         C.POINTER(C.c_int64)]
        _I64P = C.POINTER(C.c_int64)
        L.m2m_diag_kinematics.argtypes = [vp, C.POINTER(SphGrid), C.c_int64, _DP, _DP, _DP, _DP, _I64P, C.c_int64]
        L.m2m_diag_grid.argtypes = [vp, C.POINTER(PriorGrid), C.c_int64, _DP, _DP, _DP, _DP, _DP, _I64P, C.c_int32]
        L.m2m_kin_moments.argtypes = [C.c_int64, _DP, _I64P, C.c_int64, _DP, _DP, C.POINTER(C.c_int32)]
        L.m2m_delta_kin.argtypes = [C.c_int64, _DP, _I64P, _DP, _I64P, C.c_int64, _DP, _I64P]
        L.m2m_delta_grid.argtypes = [C.c_int32, _DP, _DP, _DP]
        L.m2m_weight_rms.argtypes = [C.c_int32, _DP, _I64P, C.c_int64, _DP]
        L.m2m_shard_bounds.argtypes = [vp, C.c_int64, _DP, _DP, _DP, _DP, _DP]
        L.m2m_shard_set.argtypes = [vp, C.c_int64, C.c_double, C.c_double]
        L.m2m_shard_exchange.argtypes = [vp, C.POINTER(C.c_void_p), _I64P]
        L.m2m_step_begin.argtypes = [vp]
        L.m2m_step_end.argtypes = [vp]
        L.m2m_shard_weights_begin.argtypes = [vp]
        L.m2m_batch_get_chi2.argtypes = [vp, _DP, C.c_int32]
        L.m2m_batch_get_chi2.restype = C.c_int
        L.m2m_get_scf.argtypes = [vp, _DP, _DP, C.c_int32]
        L.m2m_get_scf.restype = C.c_int
        for name in ("m2m_diag_kinematics", "m2m_diag_grid", "m2m_kin_moments", "m2m_delta_kin",
                     "m2m_delta_grid", "m2m_weight_rms", "m2m_shard_bounds", "m2m_shard_set",
                     "m2m_shard_exchange", "m2m_step_begin", "m2m_step_end", "m2m_shard_weights_begin"):
            getattr(L, name).restype = C.c_int
        for name in ("m2m_create", "m2m_load_particles", "m2m_load_particles_device", "m2m_step",
                     "m2m_synchronize", "m2m_get_weights", "m2m_get_state", "m2m_get_observables",
                     "m2m_get_chi2", "m2m_get_priors", "m2m_get_step_count", "m2m_get_particle_count",
                     "m2m_save_state", "m2m_set_timing", "m2m_get_timing",
                     "m2m_load_state", "m2m_build_targets", "m2m_create_batch", "m2m_batch_size",
                     "m2m_batch_model", "m2m_batch_autotune", "m2m_get_prior_smoothing"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _check(status: int, ctx=None):
    if status != 0:
        raise M2MError(status, lib().m2m_last_error(ctx).decode())


def potential(d: dict) -> Potential:
    """The C descriptor of a potential dict; the self-consistent kind ("scf") takes scf_r (grid
    radii), scf_lmax, ups (initial mass-to-light ratio) and eps_ups, and the log-halo fields."""
    P = Potential(POT[d["kind"]], d.get("G", 1.0), d.get("M", 1.0), d.get("a", 1.0), d.get("Ms", 0.0),
                  d.get("rs", 1.0), d.get("v0", 0.0), d.get("r0", 1.0), d.get("q", 1.0))
    if d["kind"] == "scf":
        P._r = np.ascontiguousarray(d["scf_r"], np.float64)
        P.scf_n, P.scf_lmax, P.scf_r = len(P._r), int(d["scf_lmax"]), _dp(P._r)
        P.ups, P.eps_ups = float(d.get("ups", 1.0)), float(d.get("eps_ups", 0.0))
    return P


class ObsDesc:
    """C observable descriptor built from workload groups; keeps its arrays alive."""

    def __init__(self, groups, incl_deg=0.0, Y=None, sig=None, Vp=None, sp=None):
        self.o = Observables()
        self.o.incl_deg = incl_deg
        self.o.n_groups = len(groups)
        self._keep = []
        nap = sum(g.n_ap for g in groups)
        self.Vp = np.zeros(nap) if Vp is None else np.ascontiguousarray(Vp, np.float64)
        self.sp = np.ones(nap) if sp is None else np.ascontiguousarray(sp, np.float64)
        off = 0
        for gi, g in enumerate(groups):
            G = self.o.groups[gi]
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
        self.J = sum(len(g.kinds) * g.n_ap for g in groups)
        if Y is not None:
            self.Y = np.ascontiguousarray(Y, np.float64)
            self.sig = np.ascontiguousarray(sig, np.float64)
            self.o.Y = _dp(self.Y)
            self.o.sigY = _dp(self.sig)


class SphGrid(C.Structure):
    _fields_ = [("n_r", C.c_int32), ("n_phi", C.c_int32), ("n_ct", C.c_int32), ("r_min", C.c_double),
                ("r_max", C.c_double)]


KIN_SUMS = 7


def _i64(a):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _particles(particles):
    """(n, pos, vel, w) SoA host arrays of a particle dict, or the fit's own (0, None...)."""
    if particles is None:
        return 0, None, None, None
    pos = _soa(particles, ("x", "y", "z"))
    vel = _soa(particles, ("vx", "vy", "vz"))
    w = np.ascontiguousarray(particles["w"], np.float64)
    return len(w), pos, vel, w


def kin_moments(sums, counts, min_count: int = 1):
    """(mean[nb, 3], disp[nb, 3], valid[nb]) of the spherical-bin sums (m2m_kin_moments)."""
    sums = np.ascontiguousarray(sums, np.float64).ravel()
    counts = np.ascontiguousarray(counts, np.int64)
    nb = len(counts)
    mean, disp = np.zeros(3 * nb), np.zeros(3 * nb)
    valid = np.zeros(nb, np.int32)
    _check(lib().m2m_kin_moments(nb, _dp(sums), _i64(counts), min_count, _dp(mean), _dp(disp),
                                 valid.ctypes.data_as(C.POINTER(C.c_int32))))
    return mean.reshape(nb, 3), disp.reshape(nb, 3), valid.astype(bool)


def delta_kin(sums_m, counts_m, sums_t, counts_t, min_count: int = 1):
    """(out[7], bins used): rms model-minus-target difference of the six moments (m2m_delta_kin)."""
    sm = np.ascontiguousarray(sums_m, np.float64).ravel()
    st = np.ascontiguousarray(sums_t, np.float64).ravel()
    cm = np.ascontiguousarray(counts_m, np.int64)
    ct = np.ascontiguousarray(counts_t, np.int64)
    out = np.zeros(7)
    used = C.c_int64()
    _check(lib().m2m_delta_kin(len(cm), _dp(sm), _i64(cm), _dp(st), _i64(ct), min_count, _dp(out),
                               C.byref(used)))
    return out, used.value


def delta_grid(w_model, w_target) -> float:
    wm = np.ascontiguousarray(w_model, np.float64)
    wt = np.ascontiguousarray(w_target, np.float64)
    d = C.c_double()
    _check(lib().m2m_delta_grid(len(wm), _dp(wm), _dp(wt), C.byref(d)))
    return d.value


def weight_rms(wdev2, counts, min_count: int = 50) -> float:
    wd = np.ascontiguousarray(wdev2, np.float64)
    cnt = np.ascontiguousarray(counts, np.int64)
    r = C.c_double()
    _check(lib().m2m_weight_rms(len(wd), _dp(wd), _i64(cnt), min_count, C.byref(r)))
    return r.value


def prior_grid(d: dict) -> PriorGrid:
    """m2m_prior_grid from a dict: mode ('gwr'/'mpr'), nE, nx, e_spacing, signed_lz,
    update_every, Emin, Emax; optional smoothing (0/1) with lambda, or window (half widths
    in cells, E then x) for the grid-less priors."""
    return PriorGrid(MODE[d["mode"]], d["nE"], d["nx"], ESPACING[d["e_spacing"]], d["signed_lz"],
                     d["update_every"], d["Emin"], d["Emax"], int(d.get("smoothing", 0)),
                     float(d.get("lambda", 0.0)), *(int(v) for v in d.get("window", (0, 0))))


def _soa(p: dict, keys):
    return np.ascontiguousarray(np.concatenate([np.asarray(p[k], np.float64) for k in keys]))


def build_targets(groups, incl_deg, particles: dict, err, noise=None):
    """Target Y, sigma(Y), V_p, sigma_p from a target realisation (m2m_build_targets)."""
    d = ObsDesc(groups, incl_deg)
    n = len(particles["x"])
    pos = _soa(particles, ("x", "y", "z"))
    vel = _soa(particles, ("vx", "vy", "vz"))
    w = np.ascontiguousarray(particles["w"], np.float64)
    err = np.ascontiguousarray(err, np.float64)
    nz = None if noise is None else np.ascontiguousarray(noise, np.float64)
    Y, sig = np.zeros(d.J), np.zeros(d.J)
    Vp, sp = np.zeros(len(d.Vp)), np.zeros(len(d.sp))
    it = C.c_int32()
    _check(lib().m2m_build_targets(C.byref(d.o), n, _dp(pos), _dp(vel), _dp(w), _dp(err), _dp(nz), _dp(Y),
                                   _dp(sig), _dp(Vp), _dp(sp), C.byref(it)))
    return Y, sig, Vp, sp, it.value


def observe_static(groups, incl_deg, n: int, pos_ptr: int, vel_ptr: int, w_ptr: int, y_ptr: int,
                   Vp=None, sp=None, stream=None):
    """Raw observables of device particles into device memory, without allocation
    (m2m_observe_static)."""
    d = ObsDesc(groups, incl_deg, Vp=Vp, sp=sp)
    _check(lib().m2m_observe_static(C.byref(d.o), n, pos_ptr, vel_ptr, w_ptr, y_ptr, stream))
    return d.J


class Fit:
    """One M2M fit held by the CUDA library (m2m_create ... m2m_destroy)."""

    def __init__(self, potential_desc: dict, groups, incl_deg, Y, sig, Vp, sp, prior: dict,
                 params: dict, precision: str = "fp64", stream=None, block: int = 0,
                 blocks_per_sm: int = 0, deposit: str = "auto", handle=None):
        self.desc = ObsDesc(groups, incl_deg, Y, sig, Vp, sp)
        self.J = self.desc.J
        self.ncell = prior["nE"] * prior["nx"] if prior["mode"] == "mpr" else 0
        self.n = 0
        self.owned = handle is None
        if handle is not None:  # a fit of a batch (m2m_batch_model), owned by the batch
            self.h = handle
            return
        P = potential(potential_desc)
        self._pot = P
        G = prior_grid(prior)
        opt = Options(PREC[precision], params["dt"], params["renormalize"], RULE[params["update_rule"]],
                      params["n_relax"], stream, block, blocks_per_sm, DEPOSIT[deposit])
        h = C.c_void_p()
        _check(lib().m2m_create(C.byref(P), C.byref(self.desc.o), C.byref(G), params["eps"], params["mu"],
                                params["alpha"], C.byref(opt), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            if self.owned:
                lib().m2m_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, s):
        _check(s, self.h)

    def load(self, particles: dict):
        n = len(particles["x"])
        pos = _soa(particles, ("x", "y", "z"))
        vel = _soa(particles, ("vx", "vy", "vz"))
        w = np.ascontiguousarray(particles["w"], np.float64)
        self._ck(lib().m2m_load_particles(self.h, n, _dp(pos), _dp(vel), _dp(w)))
        self.n = n

    def load_device(self, n: int, pos_ptr: int, vel_ptr: int, w_ptr: int):
        self._ck(lib().m2m_load_particles_device(self.h, n, pos_ptr, vel_ptr, w_ptr))
        self.n = n

    def step(self, nsteps: int = 1):
        self._ck(lib().m2m_step(self.h, nsteps))

    def synchronize(self):
        self._ck(lib().m2m_synchronize(self.h))

    def weights(self) -> np.ndarray:
        w = np.zeros(self.n)
        self._ck(lib().m2m_get_weights(self.h, _dp(w), self.n))
        return w

    def state(self):
        pos, vel = np.zeros(3 * self.n), np.zeros(3 * self.n)
        self._ck(lib().m2m_get_state(self.h, _dp(pos), _dp(vel), self.n))
        return pos.reshape(3, self.n), vel.reshape(3, self.n)

    def observables(self):
        yt, y = np.zeros(self.J), np.zeros(self.J)
        self._ck(lib().m2m_get_observables(self.h, _dp(yt), _dp(y), self.J))
        return yt, y

    def chi2(self, with_delta: bool = False):
        c2 = C.c_double()
        J = C.c_int32()
        d = np.zeros(self.J) if with_delta else None
        self._ck(lib().m2m_get_chi2(self.h, C.byref(c2), C.byref(J), _dp(d)))
        return (c2.value, d) if with_delta else c2.value

    def priors(self):
        g = np.zeros(max(self.ncell, 1))
        cnt = np.zeros(max(self.ncell, 1), np.int64)
        cells = np.zeros(self.n, np.int32)
        self._ck(lib().m2m_get_priors(self.h, _dp(g), cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                                      cells.ctypes.data_as(C.POINTER(C.c_int32)), self.n))
        return g[:self.ncell], cnt[:self.ncell], cells

    def diag_kinematics(self, grid: dict, particles: dict | None = None):
        """(sums[nbins, 7], counts[nbins]) of the fit's particles (or of `particles`, a dict
        of x..vz, w host arrays) in spherical polar bins (m2m_diag_kinematics)."""
        g = SphGrid(grid["n_r"], grid["n_phi"], grid["n_ct"], grid["r_min"], grid["r_max"])
        nb = grid["n_r"] * grid["n_phi"] * grid["n_ct"]
        sums = np.zeros(nb * KIN_SUMS)
        cnt = np.zeros(nb, np.int64)
        n, pos, vel, w = _particles(particles)
        self._ck(lib().m2m_diag_kinematics(self.h, C.byref(g), n, _dp(pos), _dp(vel), _dp(w), _dp(sums),
                                           _i64(cnt), nb))
        return sums.reshape(nb, KIN_SUMS), cnt

    def diag_grid(self, grid: dict | None = None, particles: dict | None = None):
        """(wsum, wdev2, counts) per (E, x) cell of the fit's grid (or `grid`) for the fit's
        particles (or `particles`) (m2m_diag_grid)."""
        G = None if grid is None else prior_grid(dict(grid, mode=grid.get("mode", "mpr")))
        nc = grid["nE"] * grid["nx"] if grid is not None else self.ncell
        ws, wd = np.zeros(max(nc, 1)), np.zeros(max(nc, 1))
        cnt = np.zeros(max(nc, 1), np.int64)
        n, pos, vel, w = _particles(particles)
        self._ck(lib().m2m_diag_grid(self.h, None if G is None else C.byref(G), n, _dp(pos), _dp(vel), _dp(w),
                                     _dp(ws), _dp(wd), _i64(cnt), nc))
        return ws[:nc], wd[:nc], cnt[:nc]

    def prior_smoothing(self):
        """(raw cell means of the last prior update, smoothing weight used) with smoothing on."""
        raw = np.zeros(max(self.ncell, 1))
        lam = C.c_double()
        self._ck(lib().m2m_get_prior_smoothing(self.h, _dp(raw), C.byref(lam)))
        return raw[:self.ncell], lam.value

    # ---- one shard of a fit split over processes (m2m_shard_*)

    def shard_bounds(self, particles: dict):
        """(sum of weights, largest 2 (E - phi_min)) of these particles (m2m_shard_bounds)."""
        n, pos, vel, w = _particles(particles)
        ws, v2 = C.c_double(), C.c_double()
        self._ck(lib().m2m_shard_bounds(self.h, n, _dp(pos), _dp(vel), _dp(w), C.byref(ws), C.byref(v2)))
        return ws.value, v2.value

    def shard_set(self, n_total: int, w_total: float, v2_bound: float):
        self._ck(lib().m2m_shard_set(self.h, n_total, w_total, v2_bound))

    def shard_exchange(self):
        """(device address, count) of the int64 words to add over the shards."""
        p, k = C.c_void_p(), C.c_int64()
        self._ck(lib().m2m_shard_exchange(self.h, C.byref(p), C.byref(k)))
        return p.value, k.value

    def step_begin(self):
        self._ck(lib().m2m_step_begin(self.h))

    def step_end(self):
        self._ck(lib().m2m_step_end(self.h))

    def shard_weights_begin(self):
        self._ck(lib().m2m_shard_weights_begin(self.h))

    def scf(self):
        """(Upsilon, a_lm,k of the last expansion (n, (lmax+1)^2)) of a self-consistent potential."""
        P = self._pot
        a = np.zeros((P.scf_n, (P.scf_lmax + 1) ** 2))
        u = C.c_double()
        self._ck(lib().m2m_get_scf(self.h, C.byref(u), _dp(a), a.size))
        return u.value, a

    def step_count(self) -> int:
        t = C.c_int64()
        self._ck(lib().m2m_get_step_count(self.h, C.byref(t)))
        return t.value

    def set_timing(self, on: bool):
        self._ck(lib().m2m_set_timing(self.h, 1 if on else 0))

    def timing(self):
        """(summed step-kernel device time in ms, steps timed)."""
        a, k = C.c_double(), C.c_int64()
        self._ck(lib().m2m_get_timing(self.h, C.byref(a), C.byref(k)))
        return a.value, k.value

    def save(self, path: str):
        self._ck(lib().m2m_save_state(self.h, path.encode()))

    def restore(self, path: str):
        self._ck(lib().m2m_load_state(self.h, path.encode()))
        n = C.c_int64()
        self._ck(lib().m2m_get_particle_count(self.h, C.byref(n)))
        self.n = n.value


def fit_from_workload(wl, Y, sig, Vp, sp, precision: str | None = None, params: dict | None = None,
                      prior: dict | None = None, **kw) -> Fit:
    return Fit(wl.potential, wl.groups, wl.incl_deg, Y, sig, Vp, sp, prior or wl.prior,
               params or wl.params, precision or wl.precision, **kw)


class Batch:
    """Many independent fits advanced together (m2m_create_batch). `fits` is a list
    of dicts with the keys of Fit's arguments: potential, groups, incl_deg, Y, sig,
    Vp, sp, prior, params. Per-fit calls go through batch.fit(i), a Fit."""

    def __init__(self, fits, precision: str = "fp64", stream=None, block: int = 0, blocks_per_sm: int = 0):
        M = len(fits)
        self.descs = [ObsDesc(f["groups"], f["incl_deg"], f["Y"], f["sig"], f["Vp"], f["sp"]) for f in fits]
        pots = (Potential * M)(*[potential(f["potential"]) for f in fits])
        obs = (Observables * M)(*[d.o for d in self.descs])
        pri = (PriorGrid * M)(*[prior_grid(f["prior"]) for f in fits])
        eps = np.array([f["params"]["eps"] for f in fits], np.float64)
        mu = np.array([f["params"]["mu"] for f in fits], np.float64)
        alpha = np.array([f["params"]["alpha"] for f in fits], np.float64)
        p0 = fits[0]["params"]
        opt = Options(PREC[precision], p0["dt"], p0["renormalize"], RULE[p0["update_rule"]], p0["n_relax"],
                      stream, block, blocks_per_sm, 0)
        h = C.c_void_p()
        _check(lib().m2m_create_batch(M, pots, obs, pri, _dp(eps), _dp(mu), _dp(alpha), C.byref(opt),
                                      C.byref(h)))
        self.h = h
        self.fits = []
        for i, f in enumerate(fits):
            sub = C.c_void_p()
            self._ck(lib().m2m_batch_model(self.h, i, C.byref(sub)))
            self.fits.append(Fit(f["potential"], f["groups"], f["incl_deg"], f["Y"], f["sig"], f["Vp"], f["sp"],
                                 f["prior"], f["params"], precision, handle=sub))

    def __len__(self):
        return len(self.fits)

    def fit(self, i: int) -> Fit:
        return self.fits[i]

    def _ck(self, s):
        _check(s, self.h)

    def step(self, nsteps: int = 1):
        self._ck(lib().m2m_step(self.h, nsteps))

    def synchronize(self):
        self._ck(lib().m2m_synchronize(self.h))

    def chi2(self) -> np.ndarray:
        """chi^2 of the last step of every fit, in one copy (m2m_batch_get_chi2)."""
        out = np.zeros(len(self.fits))
        self._ck(lib().m2m_batch_get_chi2(self.h, _dp(out), len(self.fits)))
        return out

    def autotune(self, steps: int = 3):
        """(threads per block, blocks per SM, particles per segment) kept by the autotuner."""
        b, k, seg = C.c_int32(), C.c_int32(), C.c_int64()
        self._ck(lib().m2m_batch_autotune(self.h, steps, C.byref(b), C.byref(k), C.byref(seg)))
        return b.value, k.value, seg.value

    def set_timing(self, on: bool):
        self._ck(lib().m2m_set_timing(self.h, 1 if on else 0))

    def timing(self):
        a, k = C.c_double(), C.c_int64()
        self._ck(lib().m2m_get_timing(self.h, C.byref(a), C.byref(k)))
        return a.value, k.value

    def close(self):
        if getattr(self, "h", None):
            for f in self.fits:
                f.h = None
            lib().m2m_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
