"""Global weight entropy (GWR) against moving priors (MPR) on a radially anisotropic target.

The comparison of Sec. 4 (Fig. mu): the same isotropic initial model is fitted to the same
data of a target whose orbits are radially biased, once with the global entropy of eq.
`entropy` (prior W0/N for every particle) and once with the moving priors of eq. `S+`, for
a range of regularisation weights mu. Each final model is assessed by
- chi^2/J, the fit to the data;
- Delta_grid, how well it recovers the target's mass in the (E, x) cells (Sec. 4.1);
- Delta_kin, the rms difference of its intrinsic velocity moments to the target's, here
  per spherical shell (the target is spherical);
- the rms of the weights about their cell means (Sec. 5, Fig. res).
The paper finds that MPR reaches lower Delta_grid and Delta_kin than GWR at a comparable
fit, because its entropy pulls weights towards their cell's mean instead of towards the
initial model. Mode "mprw" is the grid-less variant of Sec. 7: the prior of a particle is
the mean weight in a window of cells of a finer lattice centred on its own cell (by default
a 90 x 30 lattice with half widths 1, 1: a window of one 30 x 10 cell that moves in thirds
of a cell); Delta_grid is still taken on the 30 x 10 grid.

Synthetic stand-in for the paper's truncated target: a Hernquist sphere with constant
anisotropy sigma_r/sigma_t = 1.5 (beta = 5/9) in Jeans equilibrium, Gaussian velocities;
data are the 1M-particle fit's observable set (60 Sigma annuli, 30 annuli of v_rms, h3,
h4) at 1 % errors, with seeded Gaussian noise of those errors added, so that chi^2/J ~ 1
is the noise level; the initial model is an isotropic Hernquist realisation.

Everything runs through the library (targets by m2m_build_targets, fits by m2m_step,
diagnostics by m2m_diag_*). Usage:
    python -m paper_1202_2355_gb300.gwr_vs_mpr --n 1000000 --steps 5000
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import binding as B
from . import synth
from . import workloads as W

# 21 shells to r = 50, no angular bins: the target is spherical (Sec. 4.1 uses 21 shells)
SHELLS = dict(n_r=21, n_phi=1, n_ct=1, r_min=0.01, r_max=50.0)
RATIO = 1.5  # sigma_r / sigma_t of the target


def workload(n: int, n_target: int, alm: bool = False) -> W.Workload:
    """The 1M-particle workload's observables and potential; isotropic initial model
    of n particles (seed 0) and an anisotropic target of n_target particles (seed 100).
    alm: add the 3-D density of eq. alm on 30 quasi-logarithmic radii in [0.05, 20] (a_00 and
    a_20, errors at the target's shot noise), which constrains the mass in energy."""
    wl = W.make("c2", n=1000, n_target=1000)
    if alm:
        radii = np.exp(np.linspace(np.log(0.05), np.log(20.0), 30))
        wl.groups = wl.groups + [W.Group("shells", ["alm_0_0", "alm_2_0"], [1.0, 1.0], edges=radii)]
    beta = 1.0 - 1.0 / RATIO ** 2
    tab = synth.jeans_sigma2_table(synth.hernquist_density, synth.hernquist_mass, beta=beta)
    # realise_spherical splits 3 sigma^2 into sigma_r^2 + 2 sigma_t^2 at the given ratio
    s2 = lambda r: synth.sigma2_from_table(tab, r) * (3.0 - 2.0 * beta) / 3.0  # noqa: E731
    wl.model = synth.realise_spherical(0, n, W.hernquist_sigma2)
    wl.target = synth.realise_spherical(100, n_target, s2, anisotropy=RATIO)
    wl.n = n
    # the (E, x) grid of Sec. 4: 30 x 10 cells, for the priors and for Delta_grid
    wl.prior = dict(wl.prior, nE=30, nx=10)
    # data scattered by their errors (seeded), so that chi^2/J ~ 1 is the noise level
    wl.noise = synth.normal(100, 50, wl.J)
    return wl


def assess(fit: B.Fit, wl: W.Workload, target_grid, target_kin, min_count: int = 100) -> dict:
    wm, wd, cm = fit.diag_grid(wl.prior)
    sm, km = fit.diag_kinematics(SHELLS)
    dk, used = B.delta_kin(sm, km, *target_kin, min_count)
    return dict(delta_grid=B.delta_grid(wm, target_grid), delta_kin=float(dk[6]),
                delta_sigma_r=float(dk[3]), delta_sigma_t=float(0.5 * (dk[4] + dk[5])), shells=used,
                weight_rms_rel=B.weight_rms(wd, cm, 50) * fit.n / max(wm.sum(), 1e-300))


def scan(n: int, n_target: int, steps: int, mus, precision: str = "mixed", modes=("gwr", "mpr"),
         lattice=(90, 30), window=(1, 1), alm: bool = False):
    wl = workload(n, n_target, alm)
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    for mode in ("initial",) + tuple(modes):
        for mu in ([0.0] if mode == "initial" else mus):
            if mode == "mprw":
                prior = dict(wl.prior, mode="mpr", nE=lattice[0], nx=lattice[1], window=window)
            else:
                prior = dict(wl.prior, mode="gwr" if mode == "initial" else mode)
            fit = B.fit_from_workload(wl, Y, sig, Vp, sp, precision=precision, prior=prior,
                                      params=dict(wl.params, mu=mu))
            fit.load(wl.model)
            if mode == "initial":
                tg, _, _ = fit.diag_grid(wl.prior, particles=wl.target)
                tk = fit.diag_kinematics(SHELLS, particles=wl.target)
                marks = assess(fit, wl, tg, tk)
                fit.step(1)  # chi^2 of the initial model: the first step updates no weights
            else:
                fit.step(steps)
                marks = assess(fit, wl, tg, tk)
            row = dict(mode=mode, mu=mu, steps=0 if mode == "initial" else steps,
                       chi2_per_J=fit.chi2() / fit.J, **marks)
            fit.close()
            yield row


# initial particle models of the experiment of Sec. 4.3 (Table trunc_ics): Hernquist spheres,
# isotropic, radially or tangentially biased (constant sigma_r/sigma_t standing in for the
# paper's Osipkov-Merritt and quasi-separable models). The paper also gives them a larger
# scale length (a = 1.5); here a = 1: at a = 1.5 the initial chi^2/J is ~500 and the explicit
# update at this workload's eps dt overflows the weights within the first steps.
INITIAL = {"iso": 1.0, "rad": 2.0, "tan": 0.7}


def initial_model(n: int, kind: str, a: float = 1.0) -> dict:
    ratio = INITIAL[kind]
    beta = 1.0 - 1.0 / ratio ** 2
    tab = synth.jeans_sigma2_table(lambda r: synth.hernquist_density(r, a=a), synth.hernquist_mass, beta=beta)
    s2 = lambda r: synth.sigma2_from_table(tab, r) * (3.0 - 2.0 * beta) / 3.0  # noqa: E731
    return synth.realise_spherical(0, n, s2, a=a, anisotropy=ratio)


def vary_initial(n: int, n_target: int, steps: int, mu_of: dict, precision: str = "mixed", lattice=(90, 30),
                 window=(1, 1)):
    """Sec. 4.3: the same target and data fitted from each initial model of INITIAL, with each
    regularisation at its own mu (mu_of: mode -> mu); yields the initial model's marks
    (mode 'initial') and each final model's."""
    wl = workload(n, n_target)
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    tg = tk = None
    for ic in INITIAL:
        wl.model = initial_model(n, ic)
        for mode in ("initial",) + tuple(mu_of):
            mu = mu_of.get(mode, 0.0)
            if mode == "mprw":
                prior = dict(wl.prior, mode="mpr", nE=lattice[0], nx=lattice[1], window=window)
            else:
                prior = dict(wl.prior, mode="gwr" if mode == "initial" else mode)
            fit = B.fit_from_workload(wl, Y, sig, Vp, sp, precision=precision, prior=prior,
                                      params=dict(wl.params, mu=mu))
            fit.load(wl.model)
            if tg is None:
                tg, _, _ = fit.diag_grid(wl.prior, particles=wl.target)
                tk = fit.diag_kinematics(SHELLS, particles=wl.target)
            if mode == "initial":
                marks = assess(fit, wl, tg, tk)
                fit.step(1)
            else:
                fit.step(steps)
                marks = assess(fit, wl, tg, tk)
            yield dict(initial=ic, mode=mode, mu=mu, steps=0 if mode == "initial" else steps,
                       chi2_per_J=fit.chi2() / fit.J, **marks)
            fit.close()


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--n-target", type=int, default=2_000_000)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--mu", default="0.01,0.1,1,10,100,1000")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--modes", default="gwr,mpr", help="any of gwr, mpr, mprw (grid-less window priors)")
    ap.add_argument("--lattice", default="90,30", help="mprw: nE,nx of the prior lattice")
    ap.add_argument("--window", default="1,1", help="mprw: half widths of the window, in lattice cells")
    ap.add_argument("--alm", action="store_true", help="add the 3-D density data a_00, a_20 on 30 radii")
    ap.add_argument("--initial-models", action="store_true",
                    help="Sec. 4.3: fit from isotropic, radial and tangential initial models, each mode at "
                         "the mu given as --ic-mu gwr=...,mpr=...,mprw=...")
    ap.add_argument("--ic-mu", default="gwr=1e4,mpr=1e5,mprw=1e5")
    a = ap.parse_args()
    mus = [float(x) for x in a.mu.split(",")]
    if a.initial_models:
        mu_of = {k: float(v) for k, v in (kv.split("=") for kv in a.ic_mu.split(","))}
        print(f"{'initial':8s} {'mode':8s} {'mu':>8s} {'chi2/J':>8s} {'D_grid':>8s} {'D_kin':>8s}")
        for r in vary_initial(a.n, a.n_target, a.steps, mu_of, a.precision):
            print(f"{r['initial']:8s} {r['mode']:8s} {r['mu']:8.3g} {r['chi2_per_J']:8.3f} {r['delta_grid']:8.4f} "
                  f"{r['delta_kin']:8.4f}  " + json.dumps(r), flush=True)
        return
    lattice = tuple(int(v) for v in a.lattice.split(","))
    window = tuple(int(v) for v in a.window.split(","))
    print(f"{'mode':8s} {'mu':>8s} {'chi2/J':>8s} {'D_grid':>8s} {'D_kin':>8s} {'rms w/w0':>9s}")
    for r in scan(a.n, a.n_target, a.steps, mus, a.precision, tuple(a.modes.split(",")), lattice, window, a.alm):
        print(f"{r['mode']:8s} {r['mu']:8.3g} {r['chi2_per_J']:8.3f} {r['delta_grid']:8.4f} "
              f"{r['delta_kin']:8.4f} {r['weight_rms_rel']:9.4f}  " + json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
