"""Seeded synthetic inputs for the M2M step: particle realisations and noise draws.

This module is the one place random numbers are drawn. Both the CUDA path and the
CPU oracle take its outputs as plain arrays; it contains none of the M2M step's
arithmetic (no push, no observable kernels, no weight update). What it does hold
is the physics needed to *draw* equilibrium initial conditions:

* Hernquist radii by inverting the cumulative mass M(<r) = M r^2/(r+a)^2
  (Hernquist 1990, the model of Sec. 3.1, eq. `her`), optionally truncated;
* isotropic directions;
* Gaussian velocities with the Jeans dispersion of the tracer in the total
  potential (closed form for a self-consistent Hernquist sphere, quadrature
  otherwise), optionally anisotropic (sigma_r/sigma_t fixed at each r).

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based
generator. Output k of stream (seed, stream) is the SplitMix64 output function
applied to key + (k+1)*0x9E3779B97F4A7C15, where key itself is a SplitMix64
mix of seed and stream. Uniforms are (top 53 bits + 0.5) * 2^-53, in (0, 1).
Normals come from the Box-Muller transform of two independent uniform streams.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n 64-bit outputs of counter-based stream (seed, stream), starting at counter offset."""
    key = _mix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1 + 0x632BE59BD9B4E019)
                           & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + k * _GOLDEN)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    x = stream_u64(seed, stream, n) >> np.uint64(11)
    return (x.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """Standard normal doubles by Box-Muller on streams (stream, stream+1)."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 1, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def unit_vectors(seed: int, stream: int, n: int) -> np.ndarray:
    """Isotropic unit vectors, shape (3, n): cos(theta) uniform in [-1,1], phi uniform."""
    c = 2.0 * uniform(seed, stream, n) - 1.0
    ph = 2.0 * math.pi * uniform(seed, stream + 1, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    return np.stack([s * np.cos(ph), s * np.sin(ph), c])


# --------------------------------------------------------------------------
# Mass models used to draw equilibrium velocities (G = 1 throughout).
# --------------------------------------------------------------------------

def hernquist_mass(r, M=1.0, a=1.0):
    return M * r * r / ((r + a) ** 2)


def hernquist_density(r, M=1.0, a=1.0):
    return a * M / (2.0 * math.pi * r * (r + a) ** 3)


def nfw_mass(r, Ms, rs):
    q = r / rs
    return Ms * (np.log1p(q) - q / (1.0 + q))


def nfw_ms_from_m200(m200: float, c: float) -> float:
    """Characteristic mass M_s with M(<c r_s) = M200 for an NFW halo of concentration c."""
    return m200 / (math.log1p(c) - c / (1.0 + c))


def log_halo_mass_spherical(r, v0=1.0, r0=1.0):
    """Enclosed mass of the spherical (q=1) logarithmic potential 0.5 v0^2 ln(r0^2+r^2)."""
    return v0 * v0 * r ** 3 / (r0 * r0 + r * r)


def hernquist_sigma2_iso(r, M=1.0, a=1.0):
    """Isotropic Jeans sigma_r^2 of a self-consistent Hernquist sphere (Hernquist 1990, eq. 10)."""
    r = np.asarray(r, dtype=np.float64)
    s = r / a
    t = 12.0 * s * (s + 1.0) ** 3 * np.log((s + 1.0) / s) \
        - s / (s + 1.0) * (25.0 + 52.0 * s + 42.0 * s * s + 12.0 * s ** 3)
    return M / (12.0 * a) * t


def jeans_sigma2_table(tracer_density, total_mass, rmin=1e-5, rmax=1e5, n=2000, beta=0.0):
    """Jeans sigma_r^2(r) of a tracer with constant anisotropy beta = 1 - sigma_t^2/sigma_r^2
    in a spherical mass model, on a log grid (beta = 0: isotropic).

    rho sigma_r^2 r^(2 beta) (r) = int_r^inf rho(r') r'^(2 beta) M(r')/r'^2 dr', evaluated by
    16-point Gauss-Legendre quadrature on each log-spaced segment, summed outside-in, with
    the r^(2 beta - 6) power-law tail beyond rmax added analytically.
    Returns (log r grid, sigma_r^2 on the grid).
    """
    lr = np.linspace(math.log(rmin), math.log(rmax), n)
    xg, wg = np.polynomial.legendre.leggauss(16)
    seg = np.zeros(n - 1)
    for k in range(n - 1):
        a_, b_ = lr[k], lr[k + 1]
        t = 0.5 * (b_ - a_) * xg + 0.5 * (b_ + a_)
        rr = np.exp(t)
        f = tracer_density(rr) * rr ** (2.0 * beta) * total_mass(rr) / rr ** 2 * rr  # dr = r dlnr
        seg[k] = 0.5 * (b_ - a_) * np.dot(wg, f)
    # tail: rho ~ C r^-4, M ~ Mtot at large r -> integrand ~ C Mtot r^(2 beta - 6)
    rt = rmax
    c4 = tracer_density(np.array([rt]))[0] * rt ** 4
    mt = total_mass(np.array([rt]))[0]
    tail = c4 * mt * rt ** (2.0 * beta - 5.0) / (5.0 - 2.0 * beta)
    cum = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]]) + tail
    r = np.exp(lr)
    return lr, cum / (tracer_density(r) * r ** (2.0 * beta))


def sigma2_from_table(table, r):
    lr, s2 = table
    return np.interp(np.log(np.clip(r, math.exp(lr[0]), math.exp(lr[-1]))), lr, s2)


# --------------------------------------------------------------------------
# Realisations
# --------------------------------------------------------------------------

def hernquist_radii(seed: int, n: int, a: float = 1.0, rmax: float | None = None) -> np.ndarray:
    """Radii from the Hernquist cumulative mass; truncated at rmax if given."""
    umax = 1.0 if rmax is None else (rmax / (rmax + a)) ** 2
    u = umax * uniform(seed, 0, n)
    su = np.sqrt(u)
    return a * su / (1.0 - su)


def realise_spherical(seed: int, n: int, sigma2_of_r, a: float = 1.0, rmax: float | None = 50.0,
                      anisotropy: float = 1.0, total_weight: float = 1.0) -> dict:
    """Hernquist tracer realisation with Gaussian velocities.

    sigma2_of_r: the isotropic Jeans sigma^2(r) of the tracer in the total potential.
    anisotropy:  sigma_r/sigma_t at every radius, keeping sigma_r^2 + 2 sigma_t^2 = 3 sigma^2.
    Returns a dict of float64 SoA arrays x, y, z, vx, vy, vz, w (weights total_weight/n).
    """
    r = hernquist_radii(seed, n, a, rmax)
    rhat = unit_vectors(seed, 10, n)
    pos = rhat * r
    s2 = sigma2_of_r(r)
    k = anisotropy * anisotropy
    st2 = 3.0 * s2 / (k + 2.0)
    sr2 = k * st2
    g = np.stack([normal(seed, 20, n), normal(seed, 22, n), normal(seed, 24, n)])
    if anisotropy == 1.0:
        vel = g * np.sqrt(s2)
    else:
        # orthonormal tangential basis (e_theta, e_phi) built from rhat
        zc = rhat[2]
        rho_xy = np.sqrt(np.maximum(rhat[0] ** 2 + rhat[1] ** 2, 1e-300))
        ephi = np.stack([-rhat[1] / rho_xy, rhat[0] / rho_xy, np.zeros(n)])
        eth = np.stack([zc * rhat[0] / rho_xy, zc * rhat[1] / rho_xy, -rho_xy])
        vel = rhat * (np.sqrt(sr2) * g[0]) + eth * (np.sqrt(st2) * g[1]) + ephi * (np.sqrt(st2) * g[2])
    w = np.full(n, total_weight / n)
    return {"x": pos[0].copy(), "y": pos[1].copy(), "z": pos[2].copy(),
            "vx": vel[0].copy(), "vy": vel[1].copy(), "vz": vel[2].copy(), "w": w}


def flatten_and_rotate(p: dict, q: float, vrot_of_R=None) -> dict:
    """Squash z by q and optionally add a streaming velocity v_phi(R) about the z axis."""
    out = dict(p)
    out["z"] = p["z"] * q
    if vrot_of_R is not None:
        R = np.sqrt(p["x"] ** 2 + p["y"] ** 2)
        vphi = vrot_of_R(R)
        Rs = np.maximum(R, 1e-300)
        out["vx"] = p["vx"] - vphi * p["y"] / Rs
        out["vy"] = p["vy"] + vphi * p["x"] / Rs
    return out
