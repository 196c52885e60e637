"""The library's host arithmetic of the diagnostics (moments, Delta_kin, Delta_grid, weight
rms; Sec. 4.1 and Sec. 5) against the oracle's on the same inputs. These calls touch no
device, so they run without a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import build as BUILD


@pytest.fixture(scope="module", autouse=True)
def _built():
    BUILD.build()
    O.build()


def _sums(rng, nb, empty_every=7):
    """Per-bin sums of random particles (weights and velocities), some bins empty."""
    sums = np.zeros((nb, 7))
    counts = np.zeros(nb, np.int64)
    for b in range(nb):
        n = 0 if b % empty_every == 0 else int(rng.integers(1, 60))
        w = rng.uniform(0.1, 1.0, n)
        v = rng.normal(rng.normal(0, 0.3, 3), rng.uniform(0.2, 1.0, 3), (n, 3))
        sums[b, 0] = w.sum()
        sums[b, 1:4] = w @ v
        sums[b, 4:7] = w @ (v * v)
        counts[b] = n
    return sums, counts


def test_moments_and_delta_kin_match_oracle():
    rng = np.random.default_rng(11)
    nb = 300
    sm, cm = _sums(rng, nb)
    st, ct = _sums(rng, nb, empty_every=5)
    for min_count in (1, 10, 30):
        mean, disp, valid = B.kin_moments(sm, cm, min_count)
        mo, do, vo = O.kin_moments(sm, cm, min_count)
        assert np.array_equal(valid, vo)
        assert np.allclose(mean, mo, rtol=1e-14, atol=0) and np.allclose(disp, do, rtol=1e-12, atol=1e-15)
        out, used = B.delta_kin(sm, cm, st, ct, min_count)
        oo, uo = O.delta_kin(sm, cm, st, ct, min_count)
        assert used == uo
        assert np.allclose(out, oo, rtol=1e-12, atol=0)


def test_delta_grid_and_weight_rms_match_oracle():
    rng = np.random.default_rng(12)
    nc = 300
    wt = rng.uniform(0, 1, nc) * (rng.uniform(0, 1, nc) > 0.2)
    wm = wt * rng.uniform(0.5, 1.5, nc) * 7.0
    assert B.delta_grid(wm, wt) == pytest.approx(O.delta_grid(wm, wt), rel=1e-13)
    assert B.delta_grid(wt, wt) == 0.0
    assert B.delta_grid(np.zeros(nc), wt) == 0.0
    wd = rng.uniform(0, 1e-8, nc)
    cnt = rng.integers(0, 200, nc).astype(np.int64)
    for mc in (0, 50, 150):
        assert B.weight_rms(wd, cnt, mc) == pytest.approx(O.weight_rms(wd, cnt, mc), rel=1e-13)
    assert B.weight_rms(wd, cnt, 10**6) == 0.0


def test_host_arithmetic_rejects_bad_arguments():
    lib = B.lib()
    assert lib.m2m_delta_grid(-1, None, None, None) != 0
    assert "m2m_delta_grid" in lib.m2m_last_error(None).decode()
    assert lib.m2m_weight_rms(3, None, None, 0, None) != 0
    assert lib.m2m_delta_kin(2, None, None, None, None, 1, None, None) != 0
