"""Pins of the oracle's grid-less moving priors (the cumulative grid-less variant named in
the outlook of Sec. 7, read as a window of cells centred on each particle's own cell).

The oracle sums the cells of each window (or_window_means). The pins check it against things
fixed without that code: the mean over particle pairs on tiny inputs, constant and linear
weight fields, the cell means of Sec. 2.3.1 at zero width, and a whole oracle run whose priors
at the first update are the pair means of the initial weights."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import workloads as W


def _pair_means(kE, kx, w, hE, hx):
    """Per particle: the mean weight over all particles j with |kE_j - kE_i| <= hE and
    |kx_j - kx_i| <= hx (pairs of particles, no cells)."""
    near = (np.abs(kE[:, None] - kE[None, :]) <= hE) & (np.abs(kx[:, None] - kx[None, :]) <= hx)
    return (near * w[None, :]).sum(1) / near.sum(1)


def _cell_sums(kE, kx, w, nE, nx):
    s = np.zeros((nE, nx))
    n = np.zeros((nE, nx), np.int64)
    np.add.at(s, (kE, kx), w)
    np.add.at(n, (kE, kx), 1)
    return s, n


@pytest.mark.parametrize("hE,hx", [(0, 0), (1, 0), (0, 2), (1, 1), (2, 3), (9, 9)])
def test_window_means_equal_pair_means(hE, hx):
    O.build()
    rng = np.random.default_rng(7 + 10 * hE + hx)
    nE, nx, n = 9, 6, 400
    # clustered cells, some empty, so that windows are uneven and cut at the edges
    kE = np.minimum(rng.geometric(0.25, n) - 1, nE - 1)
    kx = rng.integers(0, nx, n)
    w = rng.lognormal(0.0, 1.0, n)
    s, c = _cell_sums(kE, kx, w, nE, nx)
    m = O.window_means(s, c, hE, hx)
    assert np.allclose(m[kE, kx], _pair_means(kE, kx, w, hE, hx), rtol=1e-13, atol=0)
    # a window without particles has prior 0
    for k in range(nE):
        for l in range(nx):
            if c[max(0, k - hE):k + hE + 1, max(0, l - hx):l + hx + 1].sum() == 0:
                assert m[k, l] == 0.0


def test_zero_width_is_the_cell_mean():
    O.build()
    rng = np.random.default_rng(3)
    s = rng.random((7, 5))
    c = rng.integers(0, 4, (7, 5))
    m = O.window_means(s, c, 0, 0)
    want = np.where(c > 0, s / np.maximum(c, 1), 0.0)
    assert np.array_equal(m, want)


def test_constant_weights_give_the_constant():
    O.build()
    c = np.random.default_rng(4).integers(1, 30, (12, 8))
    m = O.window_means(2.5 * c, c, 2, 1)
    assert np.allclose(m, 2.5, rtol=1e-15, atol=0)


def test_linear_field_is_kept_inside_and_pulled_inwards_at_the_edges():
    """Equal counts and cell means a + b k + d l: a symmetric window returns the centre's
    value; at the edges the cut window averages only the cells that exist."""
    O.build()
    nE, nx, hE, hx = 10, 7, 2, 1
    k, l = np.meshgrid(np.arange(nE), np.arange(nx), indexing="ij")
    mean = 1.0 + 0.3 * k - 0.05 * l
    cnt = np.full((nE, nx), 4, np.int64)
    m = O.window_means(mean * cnt, cnt, hE, hx)
    inner = (k >= hE) & (k < nE - hE) & (l >= hx) & (l < nx - hx)
    assert np.allclose(m[inner], mean[inner], rtol=0, atol=1e-14)
    # k = 0: cells 0..hE; l = 0: cells 0..hx
    kc = np.array([np.arange(max(0, i - hE), min(nE, i + hE + 1)).mean() for i in range(nE)])
    lc = np.array([np.arange(max(0, j - hx), min(nx, j + hx + 1)).mean() for j in range(nx)])
    assert np.allclose(m, 1.0 + 0.3 * kc[:, None] - 0.05 * lc[None, :], rtol=0, atol=1e-14)


def test_run_priors_are_pair_means_of_the_weights_at_the_update():
    """A whole oracle run with the window: the priors set at the first update (t = 1, before
    that step's weight update) are the pair means of the initial weights over the particles'
    cells at that time."""
    O.build()
    wl = W.make("c1", n=3000, n_target=20_000)
    obs, Y, sig = O.from_workload(wl)
    model = dict(wl.model)
    w0 = np.random.default_rng(11).lognormal(0.0, 0.5, len(model["w"])) * model["w"]
    model["w"] = w0.copy()
    nE, nx, hE, hx = 12, 6, 2, 1
    prior = dict(wl.prior, nE=nE, nx=nx, update_every=5, window=(hE, hx))
    run = O.Run(wl.potential, obs, Y, sig, prior, wl.params, model)
    assert run.step(1) == 0
    kE, kx = run.cell // nx, run.cell % nx
    assert np.allclose(run.what, _pair_means(kE, kx, w0, hE, hx), rtol=1e-13, atol=0)
    # and the weights moved from w0, so the next update sees other weights
    assert not np.array_equal(run.w, w0)


def test_window_with_smoothing_is_refused():
    O.build()
    wl = W.make("c1", n=500, n_target=5_000)
    obs, Y, sig = O.from_workload(wl)
    prior = dict(wl.prior, nE=8, nx=5, update_every=5, smoothing=1, window=(1, 1), **{"lambda": 1.0})
    run = O.Run(wl.potential, obs, Y, sig, prior, wl.params, wl.model)
    assert run.step(1) != 0
