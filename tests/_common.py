"""Shared helpers of the GPU parity tests: run the oracle and the CUDA path on the
same seeded workload and compare them element by element."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1202_2355_gb300 import binding as B


def obs_err(y_gpu, y_ora, sig):
    """|y_gpu - y_ora| / max(|y_ora|, sigma_j): the error on the scale that matters to the fit."""
    return np.abs(y_gpu - y_ora) / np.maximum(np.abs(y_ora), sig)


def weight_err(w_gpu, w_ora, W0, n):
    return np.abs(w_gpu - w_ora) / (np.abs(w_ora) + W0 / max(n, 1))


def edge_flip_allowance(groups, p, w, J, incl_deg=0.0):
    """Per observable, the most that particles within FP32 rounding of an annulus edge (R^2
    within 1e-6 relative) can move between the two annuli beside that edge: w |K| for each,
    with K = 1/area for surface mass, v_los^2 for v2 and 1.5 (the bound on 2 sqrt(pi) |u_n|)
    for a Gauss-Hermite kind. FP32 and FP64 may put such a particle in different annuli."""
    allow = np.zeros(J)
    si, ci = np.sin(np.radians(incl_deg)), np.cos(np.radians(incl_deg))
    Y = p["y"] * ci - p["z"] * si
    R2 = p["x"] ** 2 + Y ** 2
    vlos = p["vy"] * si + p["vz"] * ci
    off = 0
    for g in groups:
        if g.geometry != "annuli":
            off += len(g.kinds) * g.n_ap
            continue
        e2 = np.asarray(g.edges, np.float64) ** 2
        k = np.clip(np.searchsorted(e2, R2), 1, len(e2) - 1)
        k = np.where(np.abs(R2 / e2[k - 1] - 1) < np.abs(R2 / e2[k] - 1), k - 1, k)  # nearest edge
        for i in np.nonzero(np.abs(R2 / e2[k] - 1) < 1e-6)[0]:
            for kk, kind in enumerate(g.kinds):
                K = (1.0 / (np.pi * (e2[1:] - e2[:-1])) if kind == "mass" else
                     np.full(g.n_ap, vlos[i] ** 2) if kind == "v2" else np.full(g.n_ap, 1.5))
                for a in (k[i] - 1, k[i]):
                    if 0 <= a < g.n_ap:
                        allow[off + kk * g.n_ap + a] += w[i] * K[a]
        off += len(g.kinds) * g.n_ap
    return allow


class Pair:
    """The same fit run by the oracle and by the CUDA library."""

    def __init__(self, wl, particles=None, prior=None, params=None, precision=None, targets=None, **kw):
        self.wl = wl
        self.p = particles if particles is not None else wl.model
        self.prior = prior or wl.prior
        self.params = params or wl.params
        if targets is None:
            obs, Y, sig = O.from_workload(wl)
        else:
            obs, Y, sig = targets
        self.obs, self.Y, self.sig = obs, Y, sig
        self.ora = O.Run(wl.potential, obs, Y, sig, self.prior, self.params, self.p)
        self.fit = B.Fit(wl.potential, wl.groups, wl.incl_deg, Y, sig, obs.Vp, obs.sp, self.prior,
                         self.params, precision or wl.precision, **kw)
        self.fit.load(self.p)
        self.n = len(self.p["x"])

    def step(self, k):
        rc = self.ora.step(k)
        assert rc == 0, f"oracle status {rc}"
        self.fit.step(k)

    def errors(self):
        yt, yr = self.fit.observables()
        w = self.fit.weights()
        c2 = self.fit.chi2()
        pos, vel = self.fit.state()
        a = self.ora.ps.a
        dpos = max(np.max(np.abs(pos[k] - a[key]) / (1 + np.abs(a[key]))) if self.n else 0.0
                   for k, key in enumerate(("x", "y", "z")))
        dvel = max(np.max(np.abs(vel[k] - a[key]) / (1 + np.abs(a[key]))) if self.n else 0.0
                   for k, key in enumerate(("vx", "vy", "vz")))
        return dict(
            ytil=float(np.max(obs_err(yt, self.ora.ytil, self.sig))),
            yraw=float(np.max(obs_err(yr, self.ora.yraw, self.sig))),
            w=float(np.max(weight_err(w, self.ora.w, self.ora.W0, self.n))) if self.n else 0.0,
            chi2=abs(c2 - self.ora.chi2) / max(self.ora.chi2, 1e-300),
            pos=float(dpos), vel=float(dvel))

    def close(self):
        self.fit.close()
