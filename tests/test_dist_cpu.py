"""The N > 1 host path on CPU: two gloo ranks (world size 2, 127.0.0.1), each running
its own fit on the oracle, the split of a batch's fits over the ranks, and the
max-over-ranks timing reduction. No GPU and no data-path collective."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1202_2355_gb300 import dist as D
from paper_1202_2355_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank its own fit: the small c1 workload with the rank's seed
        wl = W.make("c1", n=500, n_target=20_000, seed=D.rank_seed(rank))
        obs, Y, sig = O.from_workload(wl)
        run = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, wl.model)
        assert run.step(5) == 0
        # the batch split every rank computes on its own must agree across ranks
        n = W.batch_draws()[0]
        parts = D.split_fits(n, world)
        got = [None] * world
        dist.all_gather_object(got, parts)
        t_max = D.max_over_ranks(1.0 + rank)
        q.put((rank, run.chi2, run.w.copy(), parts, got, t_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_fits_and_agree_on_the_split():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, chi2, w, parts, got, t_max = q.get(timeout=300)
        out[r] = (chi2, w, parts, got, t_max)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle as O
    for r in range(world):
        chi2, w, parts, got, t_max = out[r]
        # the rank's fit equals the same fit run serially: no cross-talk between ranks
        wl = W.make("c1", n=500, n_target=20_000, seed=D.rank_seed(r))
        obs, Y, sig = O.from_workload(wl)
        run = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, wl.model)
        assert run.step(5) == 0
        assert chi2 == run.chi2 and np.array_equal(w, run.w)
        assert got == [parts] * world
        assert t_max == 2.0
    assert not np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_split_fits_is_a_balanced_partition(world):
    n = W.batch_draws()[0]
    parts = D.split_fits(n, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(n)))
    loads = [int(sum(n[i] for i in p)) for p in parts]
    # longest-processing-time bound: no rank above the mean by more than the largest fit
    assert max(loads) - sum(loads) / world <= int(n.max())
    assert D.split_fits(n, world) == parts


def test_max_over_ranks_without_a_process_group():
    assert D.max_over_ranks(3.5) == 3.5


# ---- one fit split over ranks: the shard protocol on CPU ranks

class _FakeShard:
    """A stand-in for a library shard on the CPU: the same protocol calls, with the pass
    depositing each particle's w K_ij (the oracle's dense kernel matrix) as two-word
    fixed-point integers (floor(v 2^s) and the next 32 fraction bits), and a finalize that
    turns the summed words into y and moves every weight by a function of y. Only the words
    cross ranks."""

    def __init__(self, obs, sig):
        self.obs, self.sig = obs, sig
        self.log = []

    def shard_bounds(self, p):
        self.log.append("bounds")
        return float(np.sum(p["w"])), float(np.max(p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2))

    def shard_set(self, n_total, w_total, v2):
        self.log.append("set")
        self.scale = 2.0 ** (50 - int(np.ceil(np.log2(w_total * 4.0))))

    def load(self, p):
        import oracle as O
        self.log.append("load")
        self.p = p
        self.K = O.kernel_matrix(self.obs, O.ParticleSet(p)).T  # J x n
        self._deposit()

    def _deposit(self):
        v = self.K * self.p["w"][None, :] * self.scale  # exact: power-of-two scale
        hi = np.floor(v)
        lo = np.floor((v - hi) * 2.0 ** 32)
        self.words = np.concatenate([hi.astype(np.int64).sum(1),
                                     lo.astype(np.int64).sum(1)])

    def shard_exchange(self):
        return self.words

    def step_end(self):
        self.log.append("end")
        J = len(self.words) // 2
        self.y = (self.words[:J].astype(np.float64) + self.words[J:].astype(np.float64) * 2.0 ** -32) / self.scale

    def step_begin(self):
        self.log.append("begin")
        F = (self.K * (self.y / self.sig ** 2)[:, None]).sum(0)
        self.p = dict(self.p, w=self.p["w"] * np.exp(-1e-9 * F))
        self._deposit()

    def shard_weights_begin(self):
        self.log.append("wbegin")

    def weights(self):
        return self.p["w"].copy()


def _shard_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = W.make("c1", n=3001, n_target=20_000)
        obs, Y, sig = O.from_workload(wl)
        fake = _FakeShard(obs, sig)

        def exchange(f):
            t = torch.from_numpy(f.shard_exchange())
            dist.all_reduce(t, op=dist.ReduceOp.SUM)

        drv = D.ShardDriver(fake, exchange, D.torch_reduce)
        lo, hi = D.shard_range(wl.n, rank, world)
        drv.load(D.take_range(wl.model, lo, hi), wl.n)
        drv.step(4)
        w = drv.weights()
        q.put((rank, fake.y.copy(), w, lo, hi, fake.log))
    except Exception as e:  # report instead of leaving the parent waiting
        q.put((rank, repr(e), None, None, None, None))
        raise
    finally:
        dist.destroy_process_group()


def _run_world(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, y, w, lo, hi, log = q.get(timeout=300)
        assert w is not None, y
        out[r] = (y, w, lo, hi, log)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def test_split_fit_on_two_gloo_ranks_is_bit_identical_to_one_rank():
    one = _run_world(1)[0]
    two = _run_world(2)
    for r in range(2):
        y, w, lo, hi, log = two[r]
        assert np.array_equal(y, one[0])
        assert np.array_equal(w, one[1][lo:hi])
        assert log == ["bounds", "set", "load", "end"] + ["begin", "end"] * 4 + ["wbegin"]
    assert two[0][3] == two[1][2] and two[0][2] == 0 and two[1][3] == 3001


@pytest.mark.parametrize("n,world", [(0, 1), (7, 3), (3001, 2), (10, 10), (5, 8)])
def test_shard_ranges_tile_the_particles(n, world):
    r = [D.shard_range(n, k, world) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
    assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
