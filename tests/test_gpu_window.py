"""Grid-less moving priors on the GPU (the window of cells centred on each particle's cell,
the reading of the cumulative grid-less variant of Sec. 7) against the oracle, through the
C ABI. FP64 within 1e-10 of the oracle on observables, weights, chi^2 and priors; prior
cells and counts exact. The window sums are exact integer sums, so a fit in a batch is
bit-identical to the same fit alone."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W

from _common import Pair

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


@pytest.fixture(scope="module")
def c1_targets():
    return O.from_workload(W.make("c1"))


def _check(pr, nc, tol=TOL):
    e = pr.errors()
    assert e["ytil"] < tol and e["yraw"] < tol, e
    assert e["w"] < tol and e["chi2"] < tol, e
    g, cnt, cells = pr.fit.priors()
    assert np.array_equal(cnt, pr.ora.grid_count[:nc])
    assert np.array_equal(cells, pr.ora.cell)
    assert np.allclose(g, pr.ora.grid_mean[:nc], rtol=tol, atol=1e-26 * pr.ora.W0)
    return g, cnt, cells


@pytest.mark.parametrize("window", [(2, 1), (1, 0), (0, 3)])
def test_window_priors_match_oracle_fp64(c1_targets, window):
    """C1 (Hernquist, N = 20,000) on a 12 x 8 grid, priors every 10 steps, 4 updates."""
    wl = W.make("c1")
    prior = dict(wl.prior, nE=12, nx=8, update_every=10, window=window)
    pr = Pair(wl, prior=prior, targets=c1_targets, precision="fp64")
    for _ in range(4):
        pr.step(10)
        _check(pr, 96)
    pr.close()


def test_ragged_sizes_and_full_width(c1_targets):
    """N not a multiple of the block, priors every 7 steps; and a window covering the whole
    grid, where every prior is the mean weight W/N."""
    wl = W.make("c1", n=1013)
    pr = Pair(wl, prior=dict(wl.prior, nE=9, nx=5, update_every=7, window=(1, 2)), targets=c1_targets)
    pr.step(43)
    _check(pr, 45)
    pr.close()
    prior = dict(wl.prior, nE=9, nx=5, update_every=7, window=(9, 5))
    pr = Pair(wl, prior=prior, targets=c1_targets)
    pr.step(8)  # updates at t = 1 and t = 8
    g, _, _ = _check(pr, 45)
    # the update at t = 8 binned the weights after seven weight updates and renormalised to W0
    assert np.allclose(g, pr.ora.W0 / pr.n, rtol=1e-12)
    pr.close()


def test_window_in_mixed_precision(c1_targets):
    """Mixed mode: exact integer window sums of the FP32 weights; within 1e-4 of the FP64
    oracle over the first steps."""
    wl = W.make("c1")
    prior = dict(wl.prior, nE=12, nx=8, update_every=5, window=(2, 1))
    pr = Pair(wl, prior=prior, targets=c1_targets, precision="mixed")
    for _ in range(3):
        pr.step(5)
        e = pr.errors()
        assert e["ytil"] < 1e-4 and e["yraw"] < 1e-4 and e["chi2"] < 1e-4, e
    g, cnt, cells = pr.fit.priors()
    ok = pr.ora.grid_mean[:96] > 0
    assert np.max(np.abs(g[ok] / pr.ora.grid_mean[:96][ok] - 1)) < 1e-4
    pr.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_with_windows_is_bit_identical(precision):
    wls = W.make_batch(fits=[0, 1, 2], n_scale=0.02, n_target=50_000)
    for i, wl in enumerate(wls):
        wl.prior = dict(wl.prior, update_every=10, window=(i, 1))
        wl.params = dict(wl.params, eps=1e-4)
    targets = [O.from_workload(wl) for wl in wls]
    descs = [dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=t[1], sig=t[2], Vp=t[0].Vp,
                  sp=t[0].sp, prior=wl.prior, params=wl.params) for wl, t in zip(wls, targets)]
    batch = B.Batch(descs, precision=precision)
    for wl, f in zip(wls, batch.fits):
        f.load(wl.model)
    batch.step(25)
    batch.synchronize()
    got = [(f.weights(), f.priors()) for f in batch.fits]
    batch.close()
    for wl, t, (w, pri) in zip(wls, targets, got):
        f = B.fit_from_workload(wl, t[1], t[2], t[0].Vp, t[0].sp, precision=precision)
        f.load(wl.model)
        f.step(25)
        assert np.array_equal(w, f.weights())
        for u, v in zip(pri, f.priors()):
            assert np.array_equal(u, v)
        f.close()


def test_window_option_errors(c1_targets):
    wl = W.make("c1", n=2000)
    obs, Y, sig = c1_targets
    with pytest.raises(B.M2MError, match="half widths"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, prior=dict(wl.prior, window=(-1, 0)))
    with pytest.raises(B.M2MError, match="exclude each other"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, prior=dict(wl.prior, window=(1, 1), smoothing=1))
