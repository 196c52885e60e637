"""Seeded synthetic M2M workloads: particle models, target realisations and settings.

Each workload names the potential, the observable set (apertures, moment kinds
and their errors), the (E, x) prior grid and the step parameters, and draws the
initial particle model and the target realisation from `synth`. Kinds are
symbolic ("mass", "v2", "gh3", ...); the CUDA binding and the oracle wrapper
each translate them into their own codes. Nothing here evaluates the M2M step.

Workloads (G = M = a = 1 units):
  c1  FP64, Hernquist, N = 20,000 isotropic; target 200,000; 30 surface-density
      annuli in [0.05, 20] (1 %), 15 annuli of v2 and h4 in [0.1, 5] (1 %, 0.01);
      dt 0.01, 2,000 steps, eps 1e-3, mu 1e-2, alpha 0.02, MPR grid 30 x 10 every 25.
  c2  FP64, Hernquist, N = 1,000,000 radially biased (sigma_r/sigma_t = 1.5);
      target 2,000,000 isotropic; 60 density annuli + 30 annuli of (v2, h3, h4) to
      R = 8; dt 0.005, 10,000 steps, grid 50 x 20.
  c3  mixed, Hernquist + NFW (rs 8, M200 20, c 10), N = 2,000,000; target with
      5 % noise on v_rms and 0.03 on h4; 40 density annuli to 10, 10 annuli of
      v2, h4 within R < 2; 5,000 steps.
  c4  mixed, flattened log potential (v0 = r0 = 1, q = 0.8) seen at i = 60 deg,
      N = 8,000,000; 64 x 64 pixel maps over [-4, 4]^2 of mass and h1..h4
      (2 %, 0.02); signed-Lz grid 40 x 20, linear in exp(E); eps 1e-6; 5,000 steps.
  c5  mixed batch of 96 independent fits (make_batch): N log-uniform in
      [50,000, 2,000,000]; each a Hernquist + NFW potential with r_s uniform in
      [2, 20] and halo mass M200/M uniform in [1, 30] (c = 10); sigma_r/sigma_t
      uniform in [0.7, 1.5]; target a 200,000-particle isotropic realisation in the
      fit's own potential (seed 1000 + fit); the c2 observable set (J = 150) and
      50 x 20 grid; dt 0.005, 3,000 steps. The per-fit draws come from stream 5 of
      seed 1 (four uniforms per fit: N, r_s, M200/M, anisotropy); models use seed
      2000 + fit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import synth

KIND_NAMES = ("mass", "v2", "gh0", "gh1", "gh2", "gh3", "gh4", "gh5", "gh6")


@dataclass
class Group:
    geometry: str                     # "annuli", "pixels" or "shells"
    kinds: list                       # symbolic kinds
    errs: list                        # error per kind (relative for mass/v2, absolute for gh,
                                      # a multiple of the target's shot noise for alm)
    edges: np.ndarray | None = None   # annuli edges; shells: the 3-D grid radii
    nx: int = 0
    ny: int = 0
    box: tuple = (0.0, 0.0, 0.0, 0.0)  # xlo, xhi, ylo, yhi

    @property
    def n_ap(self) -> int:
        if self.geometry == "shells":
            return len(self.edges)
        return len(self.edges) - 1 if self.geometry == "annuli" else self.nx * self.ny


@dataclass
class Workload:
    name: str
    precision: str
    n: int
    steps: int
    potential: dict
    incl_deg: float
    groups: list
    prior: dict
    params: dict
    model: dict = field(repr=False, default_factory=dict)
    target: dict = field(repr=False, default_factory=dict)
    noise: np.ndarray | None = field(repr=False, default=None)

    @property
    def J(self) -> int:
        return sum(len(g.kinds) * g.n_ap for g in self.groups)

    def err_per_obs(self) -> np.ndarray:
        out = []
        for g in self.groups:
            for e in g.errs:
                out.append(np.full(g.n_ap, float(e)))
        return np.concatenate(out)


def _hernquist_pot():
    return dict(kind="hernquist", G=1.0, M=1.0, a=1.0, Ms=0.0, rs=1.0, v0=0.0, r0=1.0, q=1.0)


def _logspace(lo, hi, n_ap):
    return np.exp(np.linspace(math.log(lo), math.log(hi), n_ap + 1))


def _params(dt, eps=1e-3, mu=1e-2, alpha=0.02):
    return dict(dt=dt, eps=eps, mu=mu, alpha=alpha, renormalize=1, update_rule="exp", n_relax=0)


def hernquist_sigma2(r):
    return synth.hernquist_sigma2_iso(r)


def make(name: str, n: int | None = None, steps: int | None = None,
         n_target: int | None = None, seed: int = 0) -> Workload:
    """Build a workload; n, steps and n_target override the full-size values."""
    name = name.lower()
    if name == "c1":
        wl = Workload(
            name="c1_hernquist_fp64_n20k", precision="fp64", n=20_000, steps=2_000,
            potential=_hernquist_pot(), incl_deg=0.0,
            groups=[Group("annuli", ["mass"], [0.01], edges=_logspace(0.05, 20.0, 30)),
                    Group("annuli", ["v2", "gh4"], [0.01, 0.01], edges=_logspace(0.1, 5.0, 15))],
            prior=dict(mode="mpr", nE=30, nx=10, e_spacing="logneg", signed_lz=0,
                       Emin=-1.0, Emax=-1.0 / 51.0, update_every=25),
            params=_params(0.01))
        nt = n_target or 200_000
        n = n or wl.n
        wl.model = synth.realise_spherical(seed, n, hernquist_sigma2)
        wl.target = synth.realise_spherical(100, nt, hernquist_sigma2)
    elif name == "c2":
        wl = Workload(
            name="c2_hernquist_fp64_n1m", precision="fp64", n=1_000_000, steps=10_000,
            potential=_hernquist_pot(), incl_deg=0.0,
            groups=[Group("annuli", ["mass"], [0.01], edges=_logspace(0.05, 20.0, 60)),
                    Group("annuli", ["v2", "gh3", "gh4"], [0.01, 0.01, 0.01],
                          edges=_logspace(0.1, 8.0, 30))],
            prior=dict(mode="mpr", nE=50, nx=20, e_spacing="logneg", signed_lz=0,
                       Emin=-1.0, Emax=-1.0 / 51.0, update_every=25),
            params=_params(0.005))
        nt = n_target or 2_000_000
        n = n or wl.n
        wl.model = synth.realise_spherical(seed, n, hernquist_sigma2, anisotropy=1.5)
        wl.target = synth.realise_spherical(100, nt, hernquist_sigma2)
    elif name == "c3":
        ms = synth.nfw_ms_from_m200(20.0, 10.0)
        pot = dict(kind="hernquist_nfw", G=1.0, M=1.0, a=1.0, Ms=ms, rs=8.0, v0=0.0, r0=1.0, q=1.0)
        wl = Workload(
            name="c3_hernquist_nfw_mixed_n2m", precision="mixed", n=2_000_000, steps=5_000,
            potential=pot, incl_deg=0.0,
            groups=[Group("annuli", ["mass"], [0.01], edges=_logspace(0.05, 10.0, 40)),
                    Group("annuli", ["v2", "gh4"], [0.05, 0.03], edges=_logspace(0.1, 2.0, 10))],
            prior=dict(mode="mpr", nE=30, nx=10, e_spacing="logneg", signed_lz=0,
                       Emin=-1.0 - ms / 8.0, Emax=-1.0 / 51.0 - ms * math.log1p(50.0 / 8.0) / 50.0,
                       update_every=25),
            params=_params(0.01))
        tab = synth.jeans_sigma2_table(synth.hernquist_density,
                                       lambda r: synth.hernquist_mass(r) + synth.nfw_mass(r, ms, 8.0))
        s2 = lambda r: synth.sigma2_from_table(tab, r)  # noqa: E731
        nt = n_target or 2_000_000
        n = n or wl.n
        wl.model = synth.realise_spherical(seed, n, s2)
        wl.target = synth.realise_spherical(100, nt, s2)
        wl.noise = synth.normal(100, 50, wl.J)
    elif name == "c4":
        pot = dict(kind="log", G=1.0, M=0.0, a=1.0, Ms=0.0, rs=1.0, v0=1.0, r0=1.0, q=0.8)
        wl = Workload(
            name="c4_logflat_maps_mixed_n8m", precision="mixed", n=8_000_000, steps=5_000,
            potential=pot, incl_deg=60.0,
            groups=[Group("pixels", ["mass", "gh1", "gh2", "gh3", "gh4"],
                          [0.02, 0.02, 0.02, 0.02, 0.02], nx=64, ny=64, box=(-4.0, 4.0, -4.0, 4.0))],
            prior=dict(mode="mpr", nE=40, nx=20, e_spacing="exp", signed_lz=1,
                       Emin=0.0, Emax=0.0, update_every=25),
            # eps is not stated for this workload; with 2 % errors on 64 x 64 maps the
            # annulus value 1e-3 gives eps dt F ~ 10^2 (weights overflow), 1e-6 keeps it < 1
            params=_params(0.01, eps=1e-6))
        tab = synth.jeans_sigma2_table(synth.hernquist_density, synth.log_halo_mass_spherical)
        s2 = lambda r: synth.sigma2_from_table(tab, r)  # noqa: E731
        nt = n_target or 2_000_000
        n = n or wl.n
        wl.model = synth.flatten_and_rotate(synth.realise_spherical(seed, n, s2), 0.8)
        vrot = lambda R: 0.3 * R / np.sqrt(1.0 + R * R) * np.tanh(R)  # noqa: E731
        wl.target = synth.flatten_and_rotate(synth.realise_spherical(100, nt, s2), 0.8, vrot)
        m = wl.model
        E = 0.5 * (m["vx"] ** 2 + m["vy"] ** 2 + m["vz"] ** 2) + \
            0.5 * np.log(1.0 + m["x"] ** 2 + m["y"] ** 2 + m["z"] ** 2 / 0.64)
        wl.prior["Emin"] = float(E.min())
        wl.prior["Emax"] = float(E.max())
    else:
        raise ValueError(f"unknown workload {name!r}")
    wl.n = n
    if steps is not None:
        wl.steps = steps
    return wl


def subset(p: dict, n: int) -> dict:
    """First n particles of a realisation, weights rescaled to keep the total."""
    out = {k: np.ascontiguousarray(v[:n]) for k, v in p.items()}
    out["w"] = out["w"] * (p["w"].sum() / out["w"].sum())
    return out


def _c2_groups():
    return [Group("annuli", ["mass"], [0.01], edges=_logspace(0.05, 20.0, 60)),
            Group("annuli", ["v2", "gh3", "gh4"], [0.01, 0.01, 0.01], edges=_logspace(0.1, 8.0, 30))]


def batch_draws(nfits: int = 96, seed: int = 1):
    """Per-fit (N, r_s, M200/M, sigma_r/sigma_t) of the c5 batch."""
    u = synth.uniform(seed, 5, 4 * nfits).reshape(nfits, 4)
    n = np.exp(math.log(5e4) + u[:, 0] * math.log(2e6 / 5e4)).astype(np.int64)
    return n, 2.0 + 18.0 * u[:, 1], 1.0 + 29.0 * u[:, 2], 0.7 + 0.8 * u[:, 3]


def make_batch(name: str = "c5", nfits: int = 96, n_scale: float = 1.0, n_target: int | None = None,
               steps: int | None = None, fits=None) -> list:
    """The fits of a batch workload (only c5), as Workloads. n_scale multiplies
    every particle count (smaller test batches); fits selects a subset by index."""
    if name.lower() != "c5":
        raise ValueError(f"unknown batch workload {name!r}")
    n_all, rs_all, mh_all, ani_all = batch_draws(nfits)
    out = []
    for i in (range(nfits) if fits is None else fits):
        rs, mh = float(rs_all[i]), float(mh_all[i])
        ms = synth.nfw_ms_from_m200(mh, 10.0)
        pot = dict(kind="hernquist_nfw", G=1.0, M=1.0, a=1.0, Ms=ms, rs=rs, v0=0.0, r0=1.0, q=1.0)
        wl = Workload(
            name=f"c5_fit{i:02d}", precision="mixed", n=max(1, int(n_all[i] * n_scale)), steps=steps or 3_000,
            potential=pot, incl_deg=0.0, groups=_c2_groups(),
            prior=dict(mode="mpr", nE=50, nx=20, e_spacing="logneg", signed_lz=0,
                       Emin=-1.0 - ms / rs, Emax=-1.0 / 51.0 - ms * math.log1p(50.0 / rs) / 50.0,
                       update_every=25),
            # the c2 observable set with c2's step: at dt = 0.01 the explicit update with
            # eps = 1e-3 is unstable on these 1 % errors (the oracle's chi^2/J of fit 17
            # grows to ~1e4 within 100 steps); at dt = 0.005 it converges
            params=_params(0.005))
        tab = synth.jeans_sigma2_table(synth.hernquist_density,
                                       lambda r, ms=ms, rs=rs: synth.hernquist_mass(r) + synth.nfw_mass(r, ms, rs))
        s2 = lambda r, tab=tab: synth.sigma2_from_table(tab, r)  # noqa: E731
        wl.model = synth.realise_spherical(2000 + i, wl.n, s2, anisotropy=float(ani_all[i]))
        wl.target = synth.realise_spherical(1000 + i, n_target or 200_000, s2)
        out.append(wl)
    return out
