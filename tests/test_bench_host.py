"""Host logic of bench.py that decides what is timed: the timed window starts at a
prior-update step (priors are binned at steps t = 1, 1 + P, 1 + 2P, ...), so the
amortised binning is inside it for any --steps, and the host description the CPU
baseline carries. No GPU."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _is_prior_step(t, every):
    return (t - 1) % every == 0


@pytest.mark.parametrize("t0", [0, 1, 5, 24, 25, 26, 49, 50, 77])
def test_alignment_makes_the_next_step_a_prior_step(bench, t0):
    every = 25
    taken = []
    t = t0 + bench.align_to_prior_step(None, t0, every, lambda: taken.append(1))
    assert len(taken) == t - t0 < every
    assert _is_prior_step(t + 1, every)


@pytest.mark.parametrize("K,expect", [(1, 1), (20, 1), (25, 1), (26, 2), (500, 20), (1000, 40)])
def test_prior_steps_in_an_aligned_window(bench, K, expect):
    assert bench.prior_steps_in(50, K, 25) == expect
    assert bench.prior_steps_in(50, K, 25) == sum(_is_prior_step(t, 25) for t in range(51, 51 + K))


def test_host_description(bench):
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["nproc"] >= 1


def test_roofline_headline_is_the_method_byte_fraction(bench):
    for prec, b in (("mixed", 58), ("fp64", 114)):
        r = bench.roofline("c2", prec, 1_000_000, 1.0)
        assert r["bound"] == "hbm" and r["unit"] == "GB/s"
        assert r["achieved"] == pytest.approx(b * 1e6 / 1e-3 / 1e9)
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert "alu" in bench.roofline("c2", "fp64", 1_000_000, 1.0)


def test_reference_arm_runs_on_the_host_and_prints_one_line():
    """bench.py --impl reference times the oracle on the host cores: one JSON line with the
    reference fields, on a machine without a GPU as well."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_on_another_rank_exits_without_work():
    """Under torchrun the reference arm runs on rank 0 only; the other ranks exit 0 and print
    nothing."""
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1", MASTER_PORT="29533")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
