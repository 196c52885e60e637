"""The self-consistent stellar potential (Sec. 6) on the GPU against the oracle: particles
moving in Upsilon phi_star + the log halo, phi_star the multipole expansion of their own
light rebuilt on the prior schedule, with Upsilon fixed or fitted during the run. FP64 within
1e-10 of the oracle: observables, weights, chi^2, the expansion coefficients and Upsilon; the
prior cells exactly. Mixed precision within 1e-4 over the first steps."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import synth
from paper_1202_2355_gb300 import workloads as W

from _common import obs_err, weight_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


def _setup(eps_ups, n=1200, lmax=2):
    wl = W.make("c1", n=n, n_target=40_000)
    pot = dict(kind="scf", G=1.0, v0=0.45, r0=1.0, q=0.9, scf_r=np.exp(np.linspace(math.log(0.05), math.log(30.0), 10)),
               scf_lmax=lmax, ups=1.2, eps_ups=eps_ups)
    wl.potential = pot
    wl.prior = dict(mode="mpr", nE=12, nx=6, e_spacing="linear", signed_lz=0, Emin=-3.0, Emax=2.0, update_every=10)
    wl.params = dict(wl.params, eps=3e-4)
    # a model with some flattening, so that l = 2 terms matter
    wl.model["z"] = wl.model["z"] * 0.8
    return wl


def _run(wl, precision, steps):
    obs, Y, sig = O.from_workload(wl)
    ora = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, wl.model)
    fit = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision=precision)
    fit.load(wl.model)
    out = []
    done = 0
    for k in steps:
        assert ora.step(k - done) == 0
        fit.step(k - done)
        done = k
        ups, a = fit.scf()
        out.append((k, ups, a, ora.ups, ora.scf_a.copy(), fit.observables()[0], ora.ytil.copy(), fit.weights(),
                    ora.w.copy(), fit.chi2(), ora.chi2, fit.priors(), (ora.W0, ora.grid_count.copy(), ora.cell.copy())))
    fit.close()
    return out, sig


@pytest.mark.parametrize("eps_ups", [0.0, 2e-4])
def test_scf_fp64_matches_oracle(eps_ups):
    wl = _setup(eps_ups)
    out, sig = _run(wl, "fp64", [1, 5, 11, 25])
    for k, ups, a, ups_o, a_o, y, y_o, w, w_o, c2, c2_o, pri, (W0, cnt_o, cell_o) in out:
        scale = np.abs(a_o).max()
        assert np.max(np.abs(a - a_o)) < 1e-10 * scale, k
        assert abs(ups - ups_o) < 1e-10 * ups_o, k
        assert np.max(obs_err(y, y_o, sig)) < 1e-10, k
        assert np.max(weight_err(w, w_o, W0, wl.n)) < 1e-10, k
        assert abs(c2 - c2_o) < 1e-10 * c2_o, k
        g, cnt, cells = pri
        assert np.array_equal(cnt, cnt_o) and np.array_equal(cells, cell_o), k
    if eps_ups > 0:
        assert out[-1][1] != 1.2  # Upsilon moved
    else:
        assert out[-1][1] == 1.2


def test_scf_mixed_first_steps():
    wl = _setup(2e-3)
    out, sig = _run(wl, "mixed", [1, 3])
    for k, ups, a, ups_o, a_o, y, y_o, w, w_o, c2, c2_o, pri, _ in out:
        assert np.max(np.abs(a - a_o)) < 1e-4 * np.abs(a_o).max(), k
        assert abs(ups - ups_o) < 1e-4 * ups_o, k
        assert np.max(obs_err(y, y_o, sig)) < 1e-4, k


def test_scf_descriptor_errors():
    wl = _setup(0.0, n=200)
    obs, Y, sig = O.from_workload(wl)
    for bad in (dict(scf_lmax=7), dict(scf_r=np.array([1.0, 0.5])), dict(ups=0.0), dict(eps_ups=-1.0)):
        with pytest.raises(B.M2MError):
            B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, params=wl.params)._pot if False else \
                B.Fit(dict(wl.potential, **bad), wl.groups, wl.incl_deg, Y, sig, obs.Vp, obs.sp, wl.prior, wl.params)
    d = dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=obs.Vp, sp=obs.sp,
             prior=wl.prior, params=wl.params)
    with pytest.raises(B.M2MError, match="not available in batches"):
        B.Batch([d])
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp)
    f.load(wl.model)
    with pytest.raises(B.M2MError, match="checkpoints"):
        f.save("/tmp/m2m_scf_checkpoint.bin")
    f.close()
