"""One fit split into shards (contiguous particle ranges) whose integer sums are added
between the per-particle pass and the finalize of every step: bit-identical to the
unsplit fit. The ranks are emulated in one process on one GPU: every shard makes its pass,
then the test adds the shards' exchange words and writes the sum back to each (what an
all-reduce over the ranks does), then every shard finalizes. No kernel waits on another."""
import numpy as np
import pytest

import oracle as O
from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import dist as D
from paper_1202_2355_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    from paper_1202_2355_gb300 import build
    build.build()
    O.build()
    return t


def _exchange(torch, shards):
    words = []
    for f in shards:
        ptr, count = f.shard_exchange()
        f.synchronize()
        words.append(torch.as_tensor(D._DeviceWords(ptr, count), device="cuda"))
    total = torch.stack(words).sum(0)
    for w in words:
        w.copy_(total)
    torch.cuda.synchronize()


def _split_run(torch, wl, Y, sig, Vp, sp, precision, world, steps, prior=None):
    shards = [B.fit_from_workload(wl, Y, sig, Vp, sp, precision=precision, prior=prior) for _ in range(world)]
    parts = [D.take_range(wl.model, *D.shard_range(wl.n, r, world)) for r in range(world)]
    bounds = [f.shard_bounds(p) for f, p in zip(shards, parts)]
    w_total = sum(b[0] for b in bounds)
    v2 = max(b[1] for b in bounds)
    for f, p in zip(shards, parts):
        f.shard_set(wl.n, w_total, v2)
        f.load(p)
    _exchange(torch, shards)
    for f in shards:
        f.step_end()
    yield shards
    for t in steps:
        for _ in range(t):
            for f in shards:
                f.step_begin()
            _exchange(torch, shards)
            for f in shards:
                f.step_end()
        yield shards
    for f in shards:
        f.shard_weights_begin()
    _exchange(torch, shards)
    yield [f.weights() for f in shards]


def _whole(f):
    yt, yr = f.observables()
    c2, d = f.chi2(with_delta=True)
    g, cnt, _ = f.priors()
    return yt, yr, c2, d, g, cnt


@pytest.mark.parametrize("precision,world,smooth", [("fp64", 2, 0), ("mixed", 3, 0), ("mixed", 2, 1)])
def test_split_fit_is_bit_identical_to_the_whole_fit(torch, precision, world, smooth):
    wl = W.make("c1", n=20_003)
    obs, Y, sig = O.from_workload(wl)
    prior = dict(wl.prior, nE=12, nx=8, update_every=10, smoothing=1, **{"lambda": 0.0}) if smooth else None
    ref = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp, precision=precision, prior=prior)
    ref.load(wl.model)
    steps = [1, 25, 34]  # through the prior updates at t = 1, 26, 51 (or every 10 with smoothing)
    run = _split_run(torch, wl, Y, sig, obs.Vp, obs.sp, precision, world, steps, prior=prior)
    for k, t in enumerate([0] + steps):
        shards = next(run)
        if t:
            ref.step(t)
        want = _whole(ref)
        for f in shards:
            got = _whole(f)
            for a, b in zip(got, want):
                assert np.array_equal(a, b), (k, t)
    ws = next(run)
    assert np.array_equal(np.concatenate(ws), ref.weights())
    pos, _ = ref.state()
    lo, hi = D.shard_range(wl.n, world - 1, world)
    assert np.array_equal(shards[-1].state()[0], pos[:, lo:hi])
    assert ref.chi2() > 0
    for f in shards:
        f.close()
    ref.close()


def test_shard_protocol_errors(torch):
    wl = W.make("c1", n=2000)
    obs, Y, sig = O.from_workload(wl)
    f = B.fit_from_workload(wl, Y, sig, obs.Vp, obs.sp)
    with pytest.raises(B.M2MError, match="not a shard"):
        f.step_begin()
    w, v2 = f.shard_bounds(wl.model)
    assert w == pytest.approx(wl.model["w"].sum()) and v2 > 0
    with pytest.raises(B.M2MError, match="v2_bound"):
        f.shard_set(2000, w, -1.0)
    f.shard_set(2000, w, 0.5 * v2)
    with pytest.raises(B.M2MError, match="above the shard bound"):
        f.load(wl.model)
    f.shard_set(2000, w, v2)
    f.load(wl.model)
    with pytest.raises(B.M2MError, match="m2m_step_begin"):
        f.step(1)
    with pytest.raises(B.M2MError, match="needs a loaded shard"):
        f.step_begin()  # the load's exchange and m2m_step_end are still due
    f.step_end()
    with pytest.raises(B.M2MError, match="follows a load"):
        f.step_end()
    with pytest.raises(B.M2MError, match="m2m_shard_weights_begin"):
        f.weights()
    f.close()
