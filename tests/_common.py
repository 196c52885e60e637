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
