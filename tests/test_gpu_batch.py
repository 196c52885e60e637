"""Batches of independent fits (m2m_create_batch): one launch per step over all fits.

A fit advanced in a batch must give bit-identical results to the same fit advanced
alone (the sums are exact integers, whatever the launch shape), fits of uneven and
zero size included, and each fit must match the oracle like a single fit.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W

from _common import obs_err, weight_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


def _fits(n_fits=5, n_scale=0.02, with_tiny=True, eps=1e-4):
    """The first fits of the c5 batch scaled down. With a few thousand particles the
    chi^2 of the 1 % data is ~10^6, and eps = 1e-3 grows weights by ~e per step, past
    the mixed-precision fixed-point range (2^12 W0) within a few steps (in either
    execution); eps = 1e-4 keeps the test fits in range."""
    wls = W.make_batch(fits=list(range(n_fits)), n_scale=n_scale, n_target=50_000)
    for wl in wls:
        wl.prior = dict(wl.prior, update_every=10)
        wl.params = dict(wl.params, eps=eps)
    if with_tiny:
        wls[1].model = W.subset(wls[1].model, 37)
        wls[1].n = 37
        wls[3].model = {k: v[:0].copy() for k, v in wls[3].model.items()}  # a fit with no particles
        wls[3].n = 0
    return wls


def _desc(wl, targets):
    obs, Y, sig = targets
    return dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=obs.Vp,
                sp=obs.sp, prior=wl.prior, params=wl.params)


def _snapshot(f):
    return dict(w=f.weights(), y=f.observables(), chi2=f.chi2(), pri=f.priors(), t=f.step_count())


def _same(a, b):
    assert a["t"] == b["t"]
    assert np.array_equal(a["w"], b["w"])
    assert np.array_equal(a["y"][0], b["y"][0]) and np.array_equal(a["y"][1], b["y"][1])
    assert a["chi2"] == b["chi2"] or (np.isnan(a["chi2"]) and np.isnan(b["chi2"]))
    for u, v in zip(a["pri"], b["pri"]):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_is_bit_identical_to_separate_fits(precision):
    wls = _fits()
    targets = [O.from_workload(wl) for wl in wls]
    batch = B.Batch([_desc(wl, t) for wl, t in zip(wls, targets)], precision=precision)
    for wl, f in zip(wls, batch.fits):
        f.load(wl.model)
    batch.step(30)
    batch.synchronize()
    got = [_snapshot(f) for f in batch.fits]
    chi2_all = batch.chi2()
    batch.close()
    for wl, t, g in zip(wls, targets, got):
        f = B.fit_from_workload(wl, t[1], t[2], t[0].Vp, t[0].sp, precision=precision)
        f.load(wl.model)
        f.step(30)
        _same(g, _snapshot(f))
        f.close()
    # the batched chi^2 read gives every fit's own value
    assert np.array_equal(np.array([g["chi2"] for g in got]), chi2_all, equal_nan=True)


def test_batch_fits_match_the_oracle_fp64():
    wls = _fits(n_fits=3, n_scale=0.01, with_tiny=False, eps=1e-3)
    targets = [O.from_workload(wl) for wl in wls]
    batch = B.Batch([_desc(wl, t) for wl, t in zip(wls, targets)], precision="fp64")
    oras = []
    for wl, t, f in zip(wls, targets, batch.fits):
        f.load(wl.model)
        oras.append(O.Run(wl.potential, t[0], t[1], t[2], wl.prior, wl.params, wl.model))
    for _ in range(2):
        batch.step(12)
        for o in oras:
            assert o.step(12) == 0
        for wl, t, f, o in zip(wls, targets, batch.fits, oras):
            yt, yr = f.observables()
            assert np.max(obs_err(yt, o.ytil, t[2])) < 1e-10
            assert np.max(obs_err(yr, o.yraw, t[2])) < 1e-10
            assert np.max(weight_err(f.weights(), o.w, o.W0, wl.n)) < 1e-10
            assert abs(f.chi2() - o.chi2) < 1e-10 * o.chi2
            _, cnt, cells = f.priors()
            assert np.array_equal(cells, o.cell) and np.array_equal(cnt, o.grid_count)
    batch.close()


def test_autotune_does_not_change_results():
    wls = _fits(n_fits=4, n_scale=0.02)
    targets = [O.from_workload(wl) for wl in wls]
    descs = [_desc(wl, t) for wl, t in zip(wls, targets)]
    a = B.Batch(descs, precision="mixed")
    b = B.Batch(descs, precision="mixed")
    for wl, fa, fb in zip(wls, a.fits, b.fits):
        fa.load(wl.model)
        fb.load(wl.model)
    shape = a.autotune(steps=1)
    assert shape[0] in (128, 256) and shape[1] >= 1 and 0 < shape[2] <= 32768
    t = a.fit(0).step_count()
    assert t >= 2
    a.step(20)
    b.step(t + 20)
    for fa, fb in zip(a.fits, b.fits):
        _same(_snapshot(fa), _snapshot(fb))
    a.close()
    b.close()


def test_reloading_and_stepping_one_fit_of_a_batch():
    wls = _fits(n_fits=3, n_scale=0.01, with_tiny=False)
    targets = [O.from_workload(wl) for wl in wls]
    batch = B.Batch([_desc(wl, t) for wl, t in zip(wls, targets)], precision="fp64")
    for wl, f in zip(wls, batch.fits):
        f.load(wl.model)
    batch.step(5)
    # a different particle count for fit 1 rebuilds the batch's segments
    small = W.subset(wls[1].model, 1234)
    batch.fit(1).load(small)
    batch.fit(2).step(3)  # one fit stepped alone
    batch.step(10)
    solo = []
    for i, (wl, t) in enumerate(zip(wls, targets)):
        f = B.fit_from_workload(wl, t[1], t[2], t[0].Vp, t[0].sp, precision="fp64")
        f.load(small if i == 1 else wl.model)
        f.step({0: 15, 1: 10, 2: 18}[i])
        solo.append(_snapshot(f))
        f.close()
    for f, s in zip(batch.fits, solo):
        _same(_snapshot(f), s)
    batch.close()


def test_batch_handle_rejects_per_fit_calls():
    wls = _fits(n_fits=2, n_scale=0.005, with_tiny=False)
    targets = [O.from_workload(wl) for wl in wls]
    batch = B.Batch([_desc(wl, t) for wl, t in zip(wls, targets)], precision="mixed")
    c2, J = C.c_double(), C.c_int32()
    assert B.lib().m2m_get_chi2(batch.h, C.byref(c2), C.byref(J), None) == 8  # M2M_ERR_STATE
    with pytest.raises(B.M2MError, match="fit 0 has no particles"):
        batch.step(1)
    n = C.c_int32()
    assert B.lib().m2m_batch_size(batch.h, C.byref(n)) == 0 and n.value == 2
    h = C.c_void_p()
    assert B.lib().m2m_batch_model(batch.h, 2, C.byref(h)) == 1  # out of range
    B.lib().m2m_destroy(batch.fit(0).h)  # owned by the batch: no effect
    batch.fit(0).load(wls[0].model)
    batch.fit(1).load(wls[1].model)
    batch.step(2)
    batch.synchronize()
    assert batch.fit(0).step_count() == 2
    batch.close()
