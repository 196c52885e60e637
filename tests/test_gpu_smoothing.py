"""Prior smoothing on the GPU (Sec. 2.3.2, eq. smooth_grid) against the oracle: the
penalised spline fit of the grid of cell means with lambda fixed or chosen by GCV, used as
the moving priors. FP64 within 1e-10 of the oracle; a lambda chosen by GCV must score
within 1e-10 of the oracle's choice."""
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
    """Three prior updates (t = 1, 11, 21). With lambda fixed both sides smooth with it.
    With lambda chosen by GCV a flat minimum has many correct answers, so the GPU's choice
    is judged by its GCV score: within 1e-10 (relative) of the score at the oracle's own
    choice. The oracle then smooths with the GPU's lambda at that update, so that the two
    runs stay in step and the fit at that lambda is compared to 1e-10."""
    wl = W.make("c1")
    prior = dict(wl.prior, nE=12, nx=8, update_every=10, smoothing=1, **{"lambda": lam})
    pr = Pair(wl, prior=prior, targets=c1_targets, precision="fp64")
    scale = pr.ora.W0 / pr.n
    # step 1 bins the priors; steps 2..10 do not
    pr.fit.step(1)
    for it in range(3):
        raw, used = pr.fit.prior_smoothing()
        if lam > 0:
            assert used == lam
        else:
            # the oracle's raw means at this update: run it through the update with the
            # GPU's lambda, then judge the GPU's lambda against the oracle's own GCV choice
            pr.ora.G.lam = used
        assert pr.ora.step(1) == 0
        pr.ora.G.lam = lam
        raw_o = pr.ora.grid_raw[:96].copy()
        assert np.max(np.abs(raw - raw_o)) < 1e-10 * scale
        if lam == 0 and it > 0:
            # at the first update (t = 1) every weight is still 1/N: the cell means are
            # constant, the GCV score is 0 for every lambda and the fit does not depend on
            # it; from the next update on the data fix lambda
            _, lam_o = O.smooth_grid(raw_o, 12, 8, 0.0)
            g_gpu = O.smooth_gcv(raw_o, 12, 8, used)
            g_ora = O.smooth_gcv(raw_o, 12, 8, lam_o)
            assert abs(g_gpu - g_ora) <= 1e-10 * g_ora, (used, lam_o, g_gpu, g_ora)
        e = pr.errors()
        assert e["ytil"] < 1e-10 and e["yraw"] < 1e-10, e
        assert e["w"] < 1e-10 and e["chi2"] < 1e-10, e
        g, cnt, cells = pr.fit.priors()
        assert np.array_equal(cnt, pr.ora.grid_count[:96]) and np.array_equal(cells, pr.ora.cell)
        assert np.max(np.abs(g - pr.ora.grid_mean[:96])) < 1e-10 * scale
        if it < 2:
            pr.step(9)
            pr.fit.step(1)
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
