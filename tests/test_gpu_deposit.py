"""Deposit strategies and the large observable sets that need the global one.

The step kernel accumulates the observables either in per-block shared-memory
fixed-point sums or directly in the global fixed-point sums (observable sets too
large for shared memory, like 64 x 64 maps of five moments). Both add the same
integers, so the results must be bit-identical; the global path must also match
the oracle like the shared one, including at the full size of the map workload.
"""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import workloads as W
from paper_1202_2355_gb300.workloads import Group

from _common import Pair, obs_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()


def _run(wl, targets, precision, deposit, steps, prior, **kw):
    obs, Y, sig = targets
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision=precision, prior=prior, deposit=deposit, **kw)
    f.load(wl.model)
    f.step(steps)
    out = dict(w=f.weights(), y=f.observables(), chi2=f.chi2(), pri=f.priors())
    f.close()
    return out


def _assert_identical(a, b, chi2_rel=0.0):
    assert np.array_equal(a["w"], b["w"])
    assert np.array_equal(a["y"][0], b["y"][0]) and np.array_equal(a["y"][1], b["y"][1])
    assert abs(a["chi2"] - b["chi2"]) <= chi2_rel * abs(a["chi2"])
    for u, v in zip(a["pri"], b["pri"]):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_and_global_deposits_are_bit_identical_annuli(precision):
    wl = W.make("c1", n=20_000)
    targets = O.from_workload(wl)
    prior = dict(wl.prior, update_every=10)
    a = _run(wl, targets, precision, "shared", 30, prior)
    b = _run(wl, targets, precision, "global", 30, prior)
    _assert_identical(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_and_global_deposits_are_bit_identical_maps(precision):
    wl = W.make("c4", n=30_000, n_target=100_000)
    wl.groups = [Group("pixels", ["mass", "gh1", "gh2", "gh3", "gh4"], [0.02] * 5, nx=12, ny=12,
                       box=(-4.0, 4.0, -4.0, 4.0))]
    wl.params = dict(wl.params, eps=1e-6)
    targets = O.from_workload(wl)
    prior = dict(wl.prior, update_every=10)
    a = _run(wl, targets, precision, "shared", 25, prior)
    b = _run(wl, targets, precision, "global", 25, prior)
    _assert_identical(a, b)


@pytest.mark.parametrize("precision,deposit,blocks", [
    ("mixed", "global", [(1024, 0), (512, 0), (256, 0), (160, 3)]),
    ("fp64", "global", [(256, 0), (96, 0)]),
    ("mixed", "shared", [(256, 0), (96, 0), (224, 4)]),
])
def test_launch_shapes_give_identical_fits(precision, deposit, blocks):
    """Threads per block and blocks per SM change only the order of integer additions
    (and, with global deposits, the size of the aperture window). The chi^2 sum over the
    observables is the one floating-point sum whose order follows the block size, also
    for block sizes that are not powers of two."""
    wl = W.make("c4", n=30_000, n_target=100_000)
    wl.groups = [Group("pixels", ["mass", "gh1", "gh2", "gh3", "gh4"], [0.02] * 5, nx=12, ny=12,
                       box=(-4.0, 4.0, -4.0, 4.0))]
    wl.params = dict(wl.params, eps=1e-6)
    targets = O.from_workload(wl)
    prior = dict(wl.prior, update_every=10)
    runs = [_run(wl, targets, precision, deposit, 25, prior, block=b, blocks_per_sm=s) for b, s in blocks]
    for r in runs[1:]:
        _assert_identical(runs[0], r, chi2_rel=1e-13)


def test_block_size_limits():
    wl = W.make("c1", n=2000)
    obs, Y, sig = O.from_workload(wl)
    with pytest.raises(B.M2MError, match="multiple of 32, <= 256"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="mixed", deposit="shared", block=512)
    with pytest.raises(B.M2MError, match="multiple of 32, <= 256"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="fp64", deposit="global", block=512)
    with pytest.raises(B.M2MError, match="multiple of 32, <= 1024"):
        B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="mixed", deposit="global", block=100)
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision="mixed", deposit="global", block=1024)
    f.close()


def test_full_map_fp64_global_deposit_matches_oracle():
    """64 x 64 maps of mass and h1..h4 (J = 20,480; the FP64 sums need 320 KiB, so the
    library picks the global deposit) against the oracle within 1e-10 after 20 steps.

    In sparsely populated outer pixels a Gauss-Hermite sum b_n = sum_i w_i K_n(nu_i)
    can cancel to far below its terms, and the rounding of any FP64 evaluation of it
    scales with sum_i w_i |K_n| <= max|K_n| l_p (l_p the pixel's sum of weights), not
    with |b_n|. The error is therefore taken relative to max(|y|, sigma, max|K_n| l_p)."""
    wl = W.make("c4", n=200_000, n_target=500_000)
    g = wl.groups[0]
    xlo, xhi, ylo, yhi = g.box
    area = (xhi - xlo) / g.nx * (yhi - ylo) / g.ny
    kmax = [_gh_kmax(n) for n in (1, 2, 3, 4)]
    pr = Pair(wl, precision="fp64", prior=dict(wl.prior, update_every=10))
    pr.step(20)
    e = pr.errors()
    assert e["w"] < 1e-10 and e["chi2"] < 1e-10, e
    assert e["pos"] < 1e-12 and e["vel"] < 1e-12, e
    yt, yr = pr.fit.observables()
    nap = g.n_ap
    for yg, yo in ((yr, pr.ora.yraw), (yt, pr.ora.ytil)):
        l = np.abs(yo[:nap]) * area
        scale = np.concatenate([np.abs(yo[:nap])] + [km * l for km in kmax])
        err = np.abs(yg - yo) / np.maximum(np.maximum(np.abs(yo), pr.sig), scale)
        assert err.max() < 1e-10, (int(np.argmax(err)), float(err.max()))
        # and plainly relative to max(|y|, sigma) on all but a few cancelling sums
        assert np.mean(obs_err(yg, yo, pr.sig) < 1e-10) > 0.999
    _, cnt, cells = pr.fit.priors()
    assert np.array_equal(cells, pr.ora.cell) and np.array_equal(cnt, pr.ora.grid_count)
    pr.close()


def _gh_kmax(n):
    """max over nu of |K_n| = |c_n H_n(nu) exp(-nu^2/2)| (physicists' H_n), on a fine grid."""
    from math import factorial, sqrt
    from numpy.polynomial import hermite as H
    nu = np.linspace(-12, 12, 240001)
    c = np.zeros(n + 1)
    c[n] = 1.0
    return float(np.max(np.abs(sqrt(2.0 ** (1 - n) / factorial(n)) * H.hermval(nu, c) * np.exp(-0.5 * nu * nu))))


def test_full_size_map_workload_mixed_against_oracle():
    """The 8,000,000-particle map workload (mixed precision, global deposit) against the
    FP64 oracle: the deposits at load and after the first push, then the weights after
    the first force of change.

    A particle within rounding of a pixel edge may fall on the other side in FP32:
    such decisions are not unique. Each observable is allowed 1e-4 of max(|y|, sigma)
    plus the most the ambiguous particles next to its pixel could move it (their
    weight times the kernel's bound); the others must agree to 1e-4. With 2 % errors
    on 64 x 64 maps the coefficients c_j = Delta_j/sigma_j reach 1e8, so one flipped
    particle changes the force on a whole pixel; the weights after the update are
    compared for particles away from edges in pixels no flip can reach."""
    wl = W.make("c4")
    g = wl.groups[0]
    pr = Pair(wl)
    assert wl.precision == "mixed" and wl.J == 20_480
    nx, ny = g.nx, g.ny
    xlo, xhi, ylo, yhi = g.box
    area = (xhi - xlo) / nx * (yhi - ylo) / ny
    kmax = np.array([1.0 / area] + [_gh_kmax(n) for n in (1, 2, 3, 4)])
    ci, si = np.cos(np.radians(wl.incl_deg)), np.sin(np.radians(wl.incl_deg))
    alpha = wl.params["alpha"]
    w_dep = pr.ora.w.copy()  # the weights the next deposit uses
    B_til = None
    for steps in (0, 1):
        if steps:
            w_dep = pr.ora.w.copy()
            pr.step(steps)
        a = pr.ora.ps.a
        fx = (a["x"] - xlo) * (nx / (xhi - xlo))
        fy = (a["y"] * ci - a["z"] * si - ylo) * (ny / (yhi - ylo))
        # pixels a particle may fall in: both sides of an edge closer than 4e-5 pixel
        # widths (FP32 rounding of the projected position is ~1e-6 of a pixel)
        dxe = np.abs(fx - np.round(fx)) < 4e-5
        dye = np.abs(fy - np.round(fy)) < 4e-5
        amb = dxe | dye
        bound = np.zeros((ny + 2, nx + 2))
        fxa, fya, wa = fx[amb], fy[amb], w_dep[amb]
        for sx in (0, 1):
            for sy in (0, 1):
                ix = np.where(dxe[amb], np.round(fxa) - sx, np.floor(fxa)).astype(np.int64) + 1
                iy = np.where(dye[amb], np.round(fya) - sy, np.floor(fya)).astype(np.int64) + 1
                # count each distinct candidate pixel once
                dup = ((sx == 1) & ~dxe[amb]) | ((sy == 1) & ~dye[amb])
                keep = ~dup & (ix >= 0) & (ix <= nx + 1) & (iy >= 0) & (iy <= ny + 1)
                np.add.at(bound, (iy[keep], ix[keep]), wa[keep])
        bpix = bound[1:-1, 1:-1].ravel()
        B_j = np.concatenate([kmax[k] * bpix for k in range(5)])
        # the smoothed observables carry the bounds of earlier steps (eq. myts)
        B_til = B_j if B_til is None else (1 - alpha) * B_til + alpha * B_j
        yt, yr = pr.fit.observables()
        for yg, yo, Bb in ((yr, pr.ora.yraw, B_j), (yt, pr.ora.ytil, B_til)):
            err = np.abs(yg - yo)
            allowed = 1e-4 * np.maximum(np.abs(yo), pr.sig) + Bb
            assert np.all(err <= allowed), (steps, int(np.argmax(err / allowed)), float(np.max(err / allowed)))
            clean = Bb == 0
            assert clean.mean() > 0.5
            assert np.max(obs_err(yg[clean], yo[clean], pr.sig[clean])) < 1e-4
        print(f"map workload, step {pr.ora.t}: {int(amb.sum())} ambiguous particles, "
              f"{int((B_j > 0).sum())} observables bounded, chi2 {pr.fit.chi2():.6e} vs {pr.ora.chi2:.6e}")
        assert abs(pr.fit.chi2() / pr.ora.chi2 - 1) < 1e-2
    # weights after the first force of change: particles inside the map, away from
    # edges, in pixels whose five smoothed observables (which set c_j) no flip reached
    ipx = np.floor(fx).astype(np.int64)
    ipy = np.floor(fy).astype(np.int64)
    inside = (ipx >= 0) & (ipx < nx) & (ipy >= 0) & (ipy < ny) & ~amb
    pix = np.where(inside, ipy * nx + ipx, 0)
    clean_pix = B_til.reshape(5, -1).max(axis=0) == 0
    sel = inside & clean_pix[pix]
    assert sel.mean() > 0.1
    w = pr.fit.weights()
    rel = np.abs(w[sel] - pr.ora.w[sel]) / pr.ora.w[sel]
    print(f"weights after the first update: {int(sel.sum())} compared, max rel err {rel.max():.2e}")
    assert rel.max() < 1e-4
    pr.close()
