"""Ensembles of full M2M runs for the mixed-precision parity tests.

The M2M feedback between weights and observables makes a run sensitive to discrete
events: a particle that crosses an aperture edge or a prior-cell boundary one step
earlier or later changes an observable by ~1/N_j and, through the force of change, the
whole later trajectory. Two FP64 runs whose initial positions differ by 1e-7 (relative)
end with instantaneous chi^2 differing by ~20 % and chi^2/J averaged over the last 1,000
steps differing by ~3 % (C1, 20,000 particles). FP32 rounding is a perturbation of that
size at every step. The fit quality of a precision is therefore a property of the
distribution of runs: its ensemble mean over initial conditions perturbed at a relative
1e-4 (large enough that the members decorrelate within the run), compared between the
precisions with the same members.

Every perturbation is drawn from the seeded counter-based generator of `synth`."""
from __future__ import annotations

import numpy as np

from paper_1202_2355_gb300 import synth

PERTURB = 1e-4


def perturb(p: dict, seed: int, rel: float = PERTURB) -> dict:
    """x (1 + rel u), u uniform in [-1, 1), for every coordinate and velocity."""
    q = dict(p)
    for k, key in enumerate(("x", "y", "z", "vx", "vy", "vz")):
        u = synth.uniform(seed, 10 + k, len(p[key]))
        q[key] = p[key] * (1.0 + rel * (2.0 * u - 1.0))
    return q


def schedule(steps: int, window: int, every: int):
    """Step counts between samples: straight to the window, then every `every` steps."""
    out, t = [], 0
    while t < steps - window:
        k = min(500, steps - window - t)
        out.append((k, False))
        t += k
    while t < steps:
        out.append((every, True))
        t += every
    return out


def batch_chi2(B, wl, Y, sig, Vp, sp, precision: str, seeds, steps: int, window: int, every: int = 5):
    """chi^2/J sampled every `every` steps over the last `window` steps of `steps`, for one
    batched run per seed (rows), and the smoothed observables of the first member at the end."""
    d = dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=Vp, sp=sp,
             prior=wl.prior, params=wl.params)
    batch = B.Batch([d] * len(seeds), precision=precision)
    try:
        for s, f in zip(seeds, batch.fits):
            f.load(perturb(wl.model, s))
        c = []
        for k, sample in schedule(steps, window, every):
            batch.step(k)
            if sample:
                c.append([f.chi2() / len(Y) for f in batch.fits])
        y0 = batch.fits[0].observables()[0]
    finally:
        batch.close()
    return np.array(c).T, y0


def oracle_chi2(wl, obs, Y, sig, seed: int, steps: int, window: int, every: int = 5):
    """The same samples for one oracle run of the perturbed model (seed), and its final
    smoothed observables. Runs in a worker process."""
    import oracle as O
    run = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, perturb(wl.model, seed))
    c = []
    for k, sample in schedule(steps, window, every):
        assert run.step(k) == 0
        if sample:
            c.append(run.chi2 / len(Y))
    return np.array(c), run.ytil.copy()


# ---- the full-run cases: (workload, steps, averaging window)

def case(name: str):
    """c1: the 20,000-particle Hernquist fit, 2,000 steps. c3r: the Hernquist + NFW fit at
    20,000 particles instead of 2,000,000, its errors scaled by sqrt(2e6 / 2e4) = 10 so that
    Delta_j has the statistics of the full fit, 5,000 steps. c5f4: fit 4 of the batch
    (56,887 particles, its own Hernquist + NFW potential), 3,000 steps."""
    from paper_1202_2355_gb300 import workloads as W
    if name == "c1":
        return W.make("c1"), 2000, 1000
    if name == "c3r":
        wl = W.make("c3", n=20_000, n_target=400_000)
        for g in wl.groups:
            g.errs = [e * 10.0 for e in g.errs]
        return wl, 5000, 2000
    if name == "c5f4":
        return W.make_batch(fits=[4])[0], 3000, 1000
    raise ValueError(name)


def oracle_member(args):
    """(name, seed) -> (name, seed, chi^2/J samples, final smoothed observables), in a worker."""
    import oracle as O
    name, seed = args
    wl, steps, window = case(name)
    obs, Y, sig = O.from_workload(wl)
    c, y = oracle_chi2(wl, obs, Y, sig, seed, steps, window)
    return name, seed, c, y
