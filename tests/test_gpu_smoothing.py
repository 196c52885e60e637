"""Prior smoothing on the GPU (Sec. 2.3.2, eq. smooth_grid) against the oracle: the
penalised spline fit of the grid of cell means with lambda fixed or chosen by GCV, used as
the moving priors. FP64 within 1e-10 of the oracle; the chosen lambda must agree."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W

from _common import Pair, obs_err, weight_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


@pytest.fixture(scope="module")
def c1_targets():
    return O.from_workload(W.make("c1"))


@pytest.mark.parametrize("lam", [0.0, 2.5])
def test_smoothed_priors_match_oracle_fp64(c1_targets, lam):
    wl = W.make("c1")
    prior = dict(wl.prior, nE=12, nx=8, update_every=10, smoothing=1, **{"lambda": lam})
    pr = Pair(wl, prior=prior, targets=c1_targets, precision="fp64")
    for it in range(3):
        pr.step(10)
        e = pr.errors()
        assert e["ytil"] < 1e-10 and e["yraw"] < 1e-10, e
        assert e["w"] < 1e-10 and e["chi2"] < 1e-10, e
        g, cnt, cells = pr.fit.priors()
        assert np.array_equal(cnt, pr.ora.grid_count[:96]) and np.array_equal(cells, pr.ora.cell)
        raw, used = pr.fit.prior_smoothing()
        scale = pr.ora.W0 / pr.n
        assert np.max(np.abs(raw - pr.ora.grid_raw[:96])) < 1e-10 * scale
        assert np.max(np.abs(g - pr.ora.grid_mean[:96])) < 1e-10 * scale
        if lam > 0:
            assert used == lam == pr.ora.lam
        elif it > 0:
            # at the first update (t = 1) every weight is still 1/N: the cell means are
            # constant, the GCV score is 0 for every lambda and the fit does not depend on
            # it; from the next update on the data fix lambda
            assert used == pr.ora.lam or abs(used / pr.ora.lam - 1) < 1e-12
    # the fit is smoother than the raw means: smaller second differences
    raw2 = raw.reshape(12, 8)
    g2 = g.reshape(12, 8)
    assert np.abs(np.diff(g2, n=2, axis=0)).sum() < np.abs(np.diff(raw2, n=2, axis=0)).sum()
    pr.close()


def test_smoothing_in_mixed_precision(c1_targets):
    """Mixed mode smooths its FP64 cell sums the same way: priors within 1e-4 of the FP64
    run after the second update (at the first one the means are constant and lambda is
    not determined)."""
    wl = W.make("c1")
    obs, Y, sig = c1_targets
    prior = dict(wl.prior, nE=12, nx=8, update_every=10, smoothing=1, **{"lambda": 0.0})
    out = {}
    for prec in ("fp64", "mixed"):
        f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision=prec, prior=prior)
        f.load(wl.model)
        f.step(12)
        out[prec] = (f.priors()[0], f.prior_smoothing())
        f.close()
    g64, (raw64, l64) = out["fp64"]
    g32, (raw32, l32) = out["mixed"]
    scale = np.abs(g64).max()
    assert np.max(np.abs(g32 - g64)) < 1e-4 * scale
    assert abs(np.log10(l32) - np.log10(l64)) < 0.05


def test_smoothing_option_errors(c1_targets):
    wl = W.make("c1", n=2000)
    obs, Y, sig = c1_targets
    with pytest.raises(B.M2MError, match="nE, nx >= 3"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, prior=dict(wl.prior, nE=2, smoothing=1))
    with pytest.raises(B.M2MError, match="lambda"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, prior=dict(wl.prior, smoothing=1, **{"lambda": -1.0}))
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp)
    f.load(wl.model)
    with pytest.raises(B.M2MError, match="smoothing is off"):
        f.prior_smoothing()
    f.close()
    d = dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=obs.Vp, sp=obs.sp,
             prior=dict(wl.prior, smoothing=1), params=wl.params)
    with pytest.raises(B.M2MError, match="not available in batches"):
        B.Batch([d, d])
