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
