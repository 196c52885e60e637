"""Spherical-harmonic density observables (eq. alm) on the GPU against the oracle.

A shell group of a_lm coefficients on a 3-D radial grid (cloud-in-cell weights) fitted
alongside the annuli of the 20,000-particle workload: targets, observables, weights and
chi^2 within 1e-10 of the oracle in FP64 after 100 steps, 1e-4 in mixed precision over
the first steps; the batched kernel gives the same fit bit for bit; invalid descriptors
are rejected."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W
from paper_1202_2355_gb300.workloads import Group

from _common import Pair, obs_err

pytestmark = pytest.mark.gpu

KINDS = [f"alm_{l}_{m}" for l in range(3) for m in range(-l, l + 1)] + ["alm_3_1", "alm_4_0", "alm_4_-4"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


def _workload(n=20_000, n_target=200_000):
    wl = W.make("c1", n=n, n_target=n_target)
    radii = np.exp(np.linspace(math.log(0.05), math.log(20.0), 12))
    # errors: the target's shot noise scaled to the model's particle number
    err = math.sqrt(n_target / n)
    wl.groups = wl.groups + [Group("shells", KINDS, [err] * len(KINDS), edges=radii)]
    return wl


@pytest.fixture(scope="module")
def alm_targets():
    return O.from_workload(_workload())


def test_targets_match_oracle():
    wl = _workload(n=1000)
    obs = O.ObsSet(wl.groups, wl.incl_deg)
    Yo, so, _ = O.build_targets(obs, O.ParticleSet(wl.target), wl.err_per_obs(), wl.noise)
    Yg, sg, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    assert np.max(obs_err(Yg, Yo, so)) < 1e-10
    assert np.allclose(sg, so, rtol=1e-10)
    nl = sum(g.n_ap for g in wl.groups[:2])
    assert np.all(Vp[nl:] == 0.0) and np.all(sp[nl:] == 1.0)


def test_fp64_100_steps_match_oracle(alm_targets):
    wl = _workload()
    prior = dict(wl.prior, update_every=25)
    pr = Pair(wl, prior=prior, targets=alm_targets, precision="fp64")
    for k in (1, 24, 75):
        pr.step(k)
        e = pr.errors()
        assert e["ytil"] < 1e-10 and e["yraw"] < 1e-10, e
        assert e["w"] < 1e-10 and e["chi2"] < 1e-10, e
    # the a_lm part of the fit: l = 0 carries the profile, the rest is noise-level
    yt, _ = pr.fit.observables()
    nl = 60
    a = yt[nl:].reshape(len(KINDS), -1)
    assert np.all(a[0] > 0)
    pr.close()


def test_mixed_first_steps_match_oracle(alm_targets):
    wl = _workload()
    pr = Pair(wl, targets=alm_targets, precision="mixed")
    for k in (1, 4):
        pr.step(k)
        e = pr.errors()
        assert e["ytil"] < 1e-4 and e["yraw"] < 1e-4, e
        assert e["chi2"] < 1e-4, e
    pr.close()


def test_batched_fit_is_bit_identical(alm_targets):
    wl = _workload()
    obs, Y, sig = alm_targets
    d = dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=obs.Vp,
             sp=obs.sp, prior=wl.prior, params=wl.params)
    solo = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="fp64")
    solo.load(wl.model)
    solo.step(30)
    bt = B.Batch([d, d], precision="fp64")
    for i in range(2):
        bt.fit(i).load(wl.model)
    bt.step(30)
    for i in range(2):
        assert np.array_equal(bt.fit(i).weights(), solo.weights())
        assert np.array_equal(bt.fit(i).observables()[0], solo.observables()[0])
    bt.close()
    solo.close()


def test_invalid_shell_descriptors_are_rejected(alm_targets):
    wl = _workload(n=2000)
    obs, Y, sig = alm_targets

    def make(groups, **kw):
        return B.Fit(wl.potential, groups, wl.incl_deg, Y[:sum(len(g.kinds) * g.n_ap for g in groups)],
                     sig[:sum(len(g.kinds) * g.n_ap for g in groups)], obs.Vp, obs.sp, wl.prior, wl.params, **kw)

    radii = np.array([0.5, 1.0, 2.0])
    with pytest.raises(B.M2MError, match="l <= 6"):
        make([Group("shells", ["alm_7_0"], [1.0], edges=radii)])
    with pytest.raises(B.M2MError, match="increasing"):
        make([Group("shells", ["alm_0_0"], [1.0], edges=np.array([1.0, 0.5, 2.0]))])
    with pytest.raises(B.M2MError, match="unknown observable kind"):
        make([Group("annuli", ["alm_0_0"], [1.0], edges=radii)])
    with pytest.raises(B.M2MError, match="shared deposit"):
        make([Group("shells", ["alm_0_0"], [1.0], edges=radii)], deposit="global")
    f = make([Group("shells", ["alm_0_0", "alm_2_0"], [1.0, 1.0], edges=radii)])
    f.close()
