"""Pins of the oracle's smoothing of the prior grid (Sec. 2.3.2, eq. smooth_grid):
a penalised least-squares fit |y - f|^2 + lambda sum (f_EE^2 + 2 f_Ex^2 + f_xx^2), with
finite-difference derivatives and lambda chosen by generalized cross validation. Checked
against what the definition fixes, with numpy written independently of the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _penalty_numpy(f):
    """sum over the grid of (f_EE)^2 + 2 (f_Ex)^2 + (f_xx)^2 by numpy differences."""
    ee = np.diff(f, n=2, axis=0)
    xx = np.diff(f, n=2, axis=1)
    ex = np.diff(np.diff(f, axis=0), axis=1)
    return float((ee ** 2).sum() + 2 * (ex ** 2).sum() + (xx ** 2).sum())


def test_penalty_is_the_finite_difference_sum():
    rng = np.random.default_rng(1)
    nE, nx = 7, 5
    P = O.smooth_penalty(nE, nx)
    assert np.allclose(P, P.T)
    for _ in range(5):
        f = rng.standard_normal((nE, nx))
        assert f.ravel() @ P @ f.ravel() == pytest.approx(_penalty_numpy(f), rel=1e-12)


def test_penalty_null_space_is_the_planes():
    nE, nx = 6, 4
    P = O.smooth_penalty(nE, nx)
    k, l = np.meshgrid(np.arange(nE), np.arange(nx), indexing="ij")
    for plane in (np.ones_like(k), k, l, 2 + 3 * k - 0.5 * l):
        assert np.abs(P @ plane.ravel().astype(float)).max() < 1e-12
    ev = np.linalg.eigvalsh(P)
    assert np.sum(ev < 1e-10) == 3 and ev[3] > 1e-3
    # a bilinear or quadratic surface is penalised
    assert (k * l).ravel() @ P @ (k * l).ravel() > 0.1
    assert (k * k).ravel() @ P @ (k * k).ravel() > 0.1


def test_limits_plane_and_interpolation():
    """lambda -> infinity: the least-squares plane; lambda -> 0: the data (Sec. 2.3.2)."""
    rng = np.random.default_rng(2)
    nE, nx = 8, 6
    y = rng.standard_normal(nE * nx)
    k, l = np.meshgrid(np.arange(nE), np.arange(nx), indexing="ij")
    A = np.c_[np.ones(nE * nx), k.ravel(), l.ravel()]
    plane = A @ np.linalg.lstsq(A, y, rcond=None)[0]
    # the distance to the plane falls like 1/lambda (the non-plane modes are damped by
    # 1/(1 + lambda d_k), d_k > 0)
    err = [np.abs(O.smooth_grid(y, nE, nx, lam)[0] - plane).max() for lam in (1e3, 1e5, 1e7)]
    assert err[0] > 50 * err[1] > 50 * 50 * err[2] * 0.5
    assert err[2] < 1e-5
    f_0, _ = O.smooth_grid(y, nE, nx, 1e-12)
    assert np.abs(f_0 - y).max() < 1e-9


def test_fixed_lambda_solution_minimises_the_objective():
    rng = np.random.default_rng(3)
    nE, nx, lam = 6, 5, 0.7
    y = rng.standard_normal(nE * nx)
    f, used = O.smooth_grid(y, nE, nx, lam)
    assert used == lam

    def obj(g):
        return float(((y - g) ** 2).sum() + lam * _penalty_numpy(g.reshape(nE, nx)))

    base = obj(f)
    for _ in range(20):
        d = 1e-4 * rng.standard_normal(nE * nx)
        assert obj(f + d) >= base
    # stationarity: (f - y) + lambda P f = 0, with the numpy penalty's gradient
    eps = 1e-6
    grad = np.array([(obj(f + eps * e) - obj(f - eps * e)) / (2 * eps) for e in np.eye(nE * nx)])
    assert np.abs(grad).max() < 1e-6


def _gcv_numpy(y, P, lam):
    n = len(y)
    A = np.linalg.inv(np.eye(n) + lam * P)
    r = y - A @ y
    return n * (r @ r) / (n - np.trace(A)) ** 2


def test_gcv_picks_the_minimum_of_the_gcv_score():
    """The weight the oracle picks minimises the GCV score (computed here with a dense
    inverse) over a fine grid of log10 lambda, to within the grid spacing."""
    rng = np.random.default_rng(4)
    nE, nx = 10, 6
    k, l = np.meshgrid(np.arange(nE) / nE, np.arange(nx) / nx, indexing="ij")
    truth = np.exp(-3 * k) * (1 + 0.5 * np.cos(3 * l))
    y = (truth + 0.05 * rng.standard_normal(truth.shape)).ravel()
    P = O.smooth_penalty(nE, nx)
    f, lam = O.smooth_grid(y, nE, nx, 0.0)
    grid = np.linspace(-4, 6, 401)
    scores = np.array([_gcv_numpy(y, P, 10 ** t) for t in grid])
    best = grid[np.argmin(scores)]
    assert abs(np.log10(lam) - best) <= 0.05
    assert _gcv_numpy(y, P, lam) <= scores.min() * (1 + 1e-9)
    # the fit is closer to the smooth truth than the noisy data
    assert np.abs(f - truth.ravel()).mean() < np.abs(y - truth.ravel()).mean()
    # and it equals the dense solve at that weight
    assert np.allclose(f, np.linalg.solve(np.eye(nE * nx) + lam * P, y), rtol=0, atol=1e-12)


def test_run_uses_the_smoothed_grid_as_priors():
    """With smoothing on, an oracle run's priors are the smoothed cell means of the
    update, and particles' priors are their cells' smoothed values."""
    wl = W.make("c1", n=3000, n_target=20_000)
    obs, Y, sig = O.from_workload(wl)
    prior = dict(wl.prior, nE=8, nx=5, update_every=5, smoothing=1, **{"lambda": 0.0})
    run = O.Run(wl.potential, obs, Y, sig, prior, wl.params, wl.model)
    assert run.step(6) == 0
    f, lam = O.smooth_grid(run.grid_raw[:40], 8, 5, 0.0)
    assert lam == run.lam
    assert np.array_equal(f, run.grid_mean[:40])
    assert np.array_equal(run.what, run.grid_mean[run.cell])
    raw = run.grid_raw[:40]
    cnt = run.grid_count[:40]
    assert np.all(raw[cnt == 0] == 0)
