#!/usr/bin/env python
"""M2M particle-steps/s on one GB300 (or N GPUs, one process each).

A "step" is one full M2M step over all particles: the pending force of change,
the leap-frog push, the observable deposit, the prior binning on update steps,
and the finalize (smoothing, residuals, chi^2, priors). The default workload is
the batch of 96 independent mixed-precision fits (Hernquist + NFW potentials,
5.2e7 particles in all, 150 observables and a 50 x 20 prior grid each, dt 0.005)
advanced by one launch per step. `--workload c1..c4` selects a single fit
(c2: the 1,000,000-particle FP64 Hernquist fit).

Timing: at least W untimed warm-up steps, continued until the next step is a
prior-update step, then exactly K steps, each bracketed by CUDA events recorded
by the library on its stream, so the timed window holds ceil(K / P) of the
binning steps that come every P = 25 steps. L2 is flushed (256 MiB write) between
timed steps, outside the timed events. Max over ranks. `e2e` repeats the run
through the public API from pinned host buffers: load, K x (step, read chi^2),
read the weights, wall clock. `--impl reference` times the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M2M particle-steps/s (push+observe+MPR weight update) at stated chi2 error, 1 GB300"
UNIT = "particle-steps/s"
WORKLOADS = {"c1": 0, "c2": 1, "c3": 2, "c4": 3, "c5": 4}


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 peak of a GB300 from its unit counts and clock: 152 SMs x 4 FP64 flop per
# clock per SM (2 DFMA lanes) x 2.07 GHz = 1.2586 TFLOP/s (nominal 1.25). An FMA
# loop reaches 1.162 TFLOP/s on this part.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12

# Per particle-step figures of the step kernel, by precision:
#   bytes         algorithmic state traffic of the method (read + write): the 6
#                 coordinates and the weight read and written, and the 2-byte prior
#                 cell read; the roofline's achieved bandwidth uses these;
#   design_bytes  what this kernel streams by design, with the caches that trade
#                 traffic for arithmetic (acceleration, apertures, exp(-nu^2/2));
#   flops         FP64 flops the FP64 kernel executes (DFMA = 2, DADD/DMUL = 1: ncu
#                 sm__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on.sum over
#                 one step launch / N), including the iterative sqrt, division, log
#                 and exp;
#   method_flops  operations the method itself asks for per particle-step on the
#                 1M-particle FP64 workload (an FMA counts 2; a square root, a division,
#                 an exp or a log counts 1): push 31, projection 6, aperture radius 3,
#                 kernel values 21, force of change 23, weight 2, total weight 1, and the
#                 prior binning of one step in 25 (40 / 25 = 1.6), rounded to 88.
KERNEL_FIGURES = {
    # method: 7 x 8 B read and written, cell 2 B = 114 B; design: read x..vz, ln w and the
    # force factor (64 B), prior cell, cached apertures and cached exp(-nu^2/2) (2 + 2 + 8 B);
    # write 64 + 2 + 8 B
    "fp64": {"bytes": 114, "design_bytes": 150, "flops": 151.37, "method_flops": 88},
    # method: 7 x 4 B read and written, cell 2 B = 58 B; design: read 6 coordinates + w
    # (28 B), prior cell and cached apertures (2 + 2 B); write 28 B + 2 B of apertures
    "mixed": {"bytes": 58, "design_bytes": 62, "flops": None},
}
# Mixed-precision workloads in the Hernquist + NFW potential keep the force factor of the
# acceleration between steps as FP64 mode does: 4 B read and 4 B written.
MIXED_CACHED_ACCEL = {"c3", "c5"}
ACCEL_BYTES_MIXED = 8

# dram__bytes_read.sum + dram__bytes_write.sum of one step launch / N, from an ncu
# capture of the kernel as it stands, by (workload, precision): (bytes per unit, N of
# the capture); absent: not captured since the kernel last changed. c5: the 12-fit
# subset of the batch (fits 0, 8, ..., 88), traffic scaled to a full launch by the
# particle count; c2: the whole 1M-particle fit.
DRAM_PER_UNIT = {("c5", "mixed"): (63.82, 8_384_798), ("c2", "fp64"): (89.77, 1_000_000)}


class ClockSampler:
    """nvidia-smi sampled every 100 ms while running (SM clock and throttle reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_cpu() -> dict:
    """Logical cores and CPU model of this host (the oracle's timings run here)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def align_to_prior_step(fit_or_batch, t: int, every: int, step) -> int:
    """Untimed steps so that the next step is a prior-update step: priors are binned at
    steps t = 1, 1 + P, 1 + 2P, ..., so after t completed steps the next one bins when
    t is a multiple of P. Returns the number of steps taken."""
    extra = (-t) % every
    for _ in range(extra):
        step()
    return extra


def prior_steps_in(t0: int, K: int, every: int) -> int:
    """Prior-update steps among steps t0 + 1 .. t0 + K."""
    return sum(1 for t in range(t0 + 1, t0 + K + 1) if (t - 1) % every == 0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def roofline(workload: str, precision: str, n: int, ms_per_launch: float, kernel: str = "k_step") -> dict:
    """Roofline of the step kernel (the only kernel of the timed region).

    The headline is the HBM fraction at the method's state traffic: 58 B (FP32) or
    114 B (FP64) per particle-step, the coordinates and the weight read and written
    and the 2-byte prior cell read. design_gbs counts what the kernel streams with its
    caches (62 B, 70 B where it keeps the force factor, 150 B in FP64). The FP64 kernel
    is bound by the FP64 pipe rather than HBM; its ALU fraction is given beside the
    headline, from the method's own operation count per particle-step."""
    f = dict(KERNEL_FIGURES[precision])
    if precision == "mixed" and workload in MIXED_CACHED_ACCEL:
        f["design_bytes"] += ACCEL_BYTES_MIXED
    sec = ms_per_launch / 1e3
    gbs = f["bytes"] * n / sec / 1e9
    design_gbs = f["design_bytes"] * n / sec / 1e9
    hbm, hbm_src = _hbm_peak()
    dram = DRAM_PER_UNIT.get((workload, precision))
    traffic = None if dram is None else dram[0] * n
    out = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "traffic": traffic, "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured"
           else hbm_src,
           "kernel": kernel, "units_per_launch": n, "unit_of_work": "particle-step",
           "ms_per_launch": ms_per_launch, "algorithmic_bytes_per_unit": f["bytes"],
           "design_bytes_per_unit": f["design_bytes"], "design_gbs": design_gbs,
           "design_frac": design_gbs / hbm,
           "traffic_per_unit_measured_at_n": None if dram is None else dram[1]}
    if precision == "fp64":
        method = f["method_flops"]
        out["alu"] = {"bound_in_practice": "fp64 pipe", "method_flops_per_unit": method,
                      "achieved_tflops": method * n / sec / 1e12, "peak_tflops": FP64_PEAK_TFLOPS,
                      "frac": method * n / sec / 1e12 / FP64_PEAK_TFLOPS,
                      "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
                      "executed_flops_per_unit": f["flops"]}
    return out


def _sample_workload(wl_name: str, n_sample: int):
    """The first n_sample particles of a workload (of the first fit for the c5 batch)."""
    from paper_1202_2355_gb300 import workloads as W
    if wl_name == "c5":
        wl = W.make_batch(fits=[0])[0]
        wl.model = W.subset(wl.model, min(n_sample, wl.n))
        wl.n = len(wl.model["x"])
        return wl
    return W.make(wl_name, n=n_sample)


def cpu_baseline(wl_name: str, n_sample: int, steps: int):
    """The oracle as it stands, single-threaded, on the first n_sample particles of the workload."""
    import oracle as O
    wl = _sample_workload(wl_name, n_sample)
    n_sample = wl.n
    obs, Y, sig = O.from_workload(wl)
    run = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, wl.model)
    t0 = time.perf_counter()
    rc = run.step(steps)
    dt = time.perf_counter() - t0
    assert rc == 0
    return n_sample * steps / dt, dt, n_sample


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O
    from paper_1202_2355_gb300 import workloads as W
    O.build()
    wl = _sample_workload(args.workload, args.ref_sample)
    n_sample = wl.n
    obs, Y, sig = O.from_workload(wl)
    run = O.Run(wl.potential, obs, Y, sig, wl.prior, wl.params, wl.model)
    assert run.step(args.warmup) == 0
    t0 = time.perf_counter()
    assert run.step(args.steps) == 0
    dt = time.perf_counter() - t0
    v = n_sample * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "sample_particles": n_sample,
                       "note": "CPU FP64 oracle, single thread, on the first particles of the workload"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{n_sample} particles of {wl.name}, {args.steps} steps",
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _e2e(B, wl, Y, sig, Vp, sp, stream, n, K, ws):
    """Wall-clock seconds of a whole job through the public API: load from pinned host
    buffers, K x (one step, read chi^2), read the weights back."""
    import ctypes as C

    import torch
    import torch.distributed as dist

    pos = torch.from_numpy(np.concatenate([wl.model[k] for k in ("x", "y", "z")])).pin_memory()
    vel = torch.from_numpy(np.concatenate([wl.model[k] for k in ("vx", "vy", "vz")])).pin_memory()
    wts = torch.from_numpy(np.ascontiguousarray(wl.model["w"])).pin_memory()
    wout = torch.empty(n, dtype=torch.float64).pin_memory()
    fit = B.fit_from_workload(wl, Y, sig, Vp, sp, stream=stream.cuda_stream)
    lib = B.lib()
    c2 = C.c_double()
    J = C.c_int32()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    B._check(lib.m2m_load_particles(fit.h, n, C.cast(pos.data_ptr(), B._DP), C.cast(vel.data_ptr(), B._DP),
                                    C.cast(wts.data_ptr(), B._DP)), fit.h)
    for _ in range(K):
        B._check(lib.m2m_step(fit.h, 1), fit.h)
        B._check(lib.m2m_get_chi2(fit.h, C.byref(c2), C.byref(J), None), fit.h)
    B._check(lib.m2m_get_weights(fit.h, C.cast(wout.data_ptr(), B._DP), n), fit.h)
    dt = time.perf_counter() - t0
    fit.close()
    if ws > 1:
        t = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t[0])
    return dt


def run_batch(args):
    """The c5 batch: 96 independent mixed-precision fits of uneven size advanced by one
    launch per step (m2m_create_batch), launch shape from the library's autotuner."""
    import ctypes as C

    import torch
    import torch.distributed as dist

    from paper_1202_2355_gb300 import binding as B
    from paper_1202_2355_gb300 import build as BUILD
    from paper_1202_2355_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    BUILD.build()
    K, Wm = args.steps, args.warmup
    n_all = W.batch_draws()[0]
    scale = 1.0 if args.n is None else args.n / float(n_all.sum())
    # the 96 fits are split over the ranks by particle count (strong scaling: the job is
    # fixed); each rank advances its share as one batch, with no collective on the data path
    from paper_1202_2355_gb300 import dist as D
    pool = list(range(len(n_all))) if args.fits is None else [int(v) for v in args.fits.split(",")]
    counts = np.maximum(1, (n_all[pool] * scale).astype(np.int64))
    mine = [pool[i] for i in D.split_fits(counts, ws)[rank]]
    wls = W.make_batch(n_scale=scale, fits=mine)
    descs = []
    for wl in wls:
        Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
        descs.append(dict(potential=wl.potential, groups=wl.groups, incl_deg=wl.incl_deg, Y=Y, sig=sig, Vp=Vp,
                          sp=sp, prior=wl.prior, params=wl.params))
        wl.target = None
    ntot = sum(wl.n for wl in wls)
    stream = torch.cuda.Stream()
    fixed = None if args.shape is None else [int(v) for v in args.shape.split(",")]
    batch = B.Batch(descs, precision="mixed", stream=stream.cuda_stream,
                    block=fixed[0] if fixed else 0, blocks_per_sm=fixed[1] if fixed else 0)
    for wl, f in zip(wls, batch.fits):
        f.load(wl.model)
    if fixed and len(fixed) != 2:
        raise SystemExit("--shape takes block,blocks_per_sm")
    shape = (fixed[0], fixed[1], "library default") if fixed else batch.autotune(steps=2)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    every = wls[0].prior["update_every"]

    def one_step():
        batch.step(1)
        flush.fill_(1)

    with torch.cuda.stream(stream):
        for _ in range(Wm):
            one_step()
        batch.synchronize()
        t_start = batch.fits[0].step_count()
        t_start += align_to_prior_step(batch, t_start, every, one_step)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    batch.set_timing(True)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for _ in range(K):
                batch.step(1)
                flush.fill_(1)
        batch.synchronize()
        torch.cuda.synchronize()
    step_ms, nt = batch.timing()
    batch.set_timing(False)
    assert nt == K
    chi2_per_J = float(np.mean([f.chi2() / f.J for f in batch.fits]))
    n_job = int(counts.sum())
    if ws > 1:
        t = torch.tensor([step_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t[0])
        dist.barrier()
    # every rank's share of the job is done within the slowest rank's time
    value = n_job * K / (step_ms / 1e3)

    e2e = None
    if not args.no_e2e:
        # end to end through the public API: load every fit from pinned host buffers,
        # K x (one batched step, read every fit's chi^2), read every fit's weights
        pinned = []
        for wl in wls:
            pinned.append((torch.from_numpy(np.concatenate([wl.model[k] for k in ("x", "y", "z")])).pin_memory(),
                           torch.from_numpy(np.concatenate([wl.model[k] for k in ("vx", "vy", "vz")])).pin_memory(),
                           torch.from_numpy(np.ascontiguousarray(wl.model["w"])).pin_memory(),
                           torch.empty(wl.n, dtype=torch.float64).pin_memory()))
        lib = B.lib()
        c2 = np.zeros(len(wls))
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for wl, f, (pos, vel, wts, _) in zip(wls, batch.fits, pinned):
            B._check(lib.m2m_load_particles(f.h, wl.n, C.cast(pos.data_ptr(), B._DP), C.cast(vel.data_ptr(), B._DP),
                                            C.cast(wts.data_ptr(), B._DP)), f.h)
        for _ in range(K):
            B._check(lib.m2m_step(batch.h, 1), batch.h)
            B._check(lib.m2m_batch_get_chi2(batch.h, B._dp(c2), len(wls)), batch.h)
        for wl, f, (_, _, _, wout) in zip(wls, batch.fits, pinned):
            B._check(lib.m2m_get_weights(f.h, C.cast(wout.data_ptr(), B._DP), wl.n), f.h)
        dt = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([dt], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t[0])
        e2e = {"value": n_job * K / dt, "unit": UNIT, "h2d_bytes_per_step": 7 * 8 * ntot / K,
               "d2h_bytes_per_step": 16 * len(wls) + 8 * ntot / K,
               "note": "every fit loaded from pinned host memory once, K x (batched step + every fit's chi^2 "
                       "read in one copy), every fit's weights read"}
    batch.close()
    roof = roofline("c5", "mixed", ntot, step_ms / K)
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            import oracle as O
            O.build()
            v, dt, ns = cpu_baseline("c5", args.cpu_sample, args.cpu_steps)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"first {ns} particles of fit 0 of the c5 batch, {args.cpu_steps} steps, "
                             f"{dt:.1f} s single-threaded FP64",
                   "host": host_cpu()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
            "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
            "config": {"workload": "c5_batch96_hernquist_nfw_mixed" if args.fits is None else
                       f"c5 fits {args.fits}", "fits": len(pool), "n_particles": n_job,
                       "fits_rank0": len(wls), "n_particles_rank0": ntot,
                       "timed_window": f"starts at a prior-update step; {prior_steps_in(t_start, K, every)} of the "
                                       f"{K} timed steps bin the priors (every {every})",
                       "observables_per_fit": wls[0].J, "prior_grid": "50x20 every 25", "dt": wls[0].params["dt"],
                       "precision": "mixed", "launch_shape": {"block": shape[0], "blocks_per_sm": shape[1],
                                                              "segment": shape[2]},
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "parallelism": f"the {len(pool)} fits split over {ws} GPU(s) by particle count, "
                                      f"one batch per GPU, no data-path collective",
                       "chi2_per_J_end_mean": chi2_per_J},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": K,  # one batched step kernel per step for all fits
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_sharded(args):
    """N > 1 GPUs on one single-fit workload: the fit split over the ranks by particles
    (contiguous ranges), one NCCL all-reduce of the int64 exchange words per step between
    each rank's pass and the finalize every rank runs on the same sums; bit-identical to
    the whole fit on one GPU. Strong scaling: the job is the one fit."""
    import torch
    import torch.distributed as dist

    from paper_1202_2355_gb300 import binding as B
    from paper_1202_2355_gb300 import build as BUILD
    from paper_1202_2355_gb300 import dist as D
    from paper_1202_2355_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    BUILD.build()
    K, Wm = args.steps, args.warmup
    wl = W.make(args.workload, n=args.n)
    if args.precision:
        wl.precision = args.precision
    n = wl.n
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    lo, hi = D.shard_range(n, rank, ws)
    part = D.take_range(wl.model, lo, hi)
    stream = torch.cuda.Stream()
    fit = B.fit_from_workload(wl, Y, sig, Vp, sp, stream=stream.cuda_stream)
    drv = D.ShardDriver(fit, D.nccl_exchange, D.torch_reduce)
    drv.load(part, n)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    every = wl.prior["update_every"] if wl.prior["mode"] == "mpr" else 1

    def one_step():
        drv.step(1)
        flush.fill_(1)

    with torch.cuda.stream(stream):
        for _ in range(Wm):
            one_step()
        t_start = fit.step_count()
        t_start += align_to_prior_step(fit, t_start, every, one_step)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    # each step bracketed on the shard's stream: pass, exchange and finalize
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for k in range(K):
                ev[k][0].record(stream)
                drv.step(1)
                ev[k][1].record(stream)
                flush.fill_(1)
        torch.cuda.synchronize()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    chi2 = fit.chi2()
    t = torch.tensor([step_ms], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    step_ms = float(t[0])
    dist.barrier()
    fit.close()
    value = n * K / (step_ms / 1e3)
    roof = roofline(args.workload, wl.precision, hi - lo, step_ms / K, kernel="k_step (shard) + all-reduce")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64" if wl.precision == "fp64" else "f32+i64", "data": "synthetic",
            "config": {"workload": wl.name, "n_particles": n, "observables": wl.J,
                       "prior_grid": f"{wl.prior['nE']}x{wl.prior['nx']} every {wl.prior['update_every']}",
                       "dt": wl.params["dt"], "precision": wl.precision,
                       "timed_window": f"starts at a prior-update step; {prior_steps_in(t_start, K, every)} of the "
                                       f"{K} timed steps bin the priors (every {every})",
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "parallelism": f"one fit split over {ws} GPUs by particles, one NCCL all-reduce of "
                                      f"the int64 sums per step", "chi2_per_J_end": chi2 / wl.J},
            "roofline": roof, "cpu_baseline": None, "e2e": None,
            "gpu_launches": 2 * K,  # per step: the shard's pass and its finalize
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1202_2355_gb300 import binding as B
    from paper_1202_2355_gb300 import build as BUILD
    from paper_1202_2355_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    BUILD.build()
    K, Wm = args.steps, args.warmup

    # one independent fit per rank (its own seed): weak scaling, no collective on the data path
    wl = W.make(args.workload, seed=rank, n=args.n)
    if args.precision:
        wl.precision = args.precision
    n = wl.n
    Y, sig, Vp, sp, _ = B.build_targets(wl.groups, wl.incl_deg, wl.target, wl.err_per_obs(), wl.noise)
    stream = torch.cuda.Stream()
    fit = B.fit_from_workload(wl, Y, sig, Vp, sp, stream=stream.cuda_stream)
    fit.load(wl.model)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    every = wl.prior["update_every"] if wl.prior["mode"] == "mpr" else 1

    def one_step():
        fit.step(1)
        flush.fill_(1)

    with torch.cuda.stream(stream):
        for _ in range(Wm):
            one_step()
        fit.synchronize()
        t_start = fit.step_count()
        t_start += align_to_prior_step(fit, t_start, every, one_step)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    fit.set_timing(True)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for _ in range(K):
                fit.step(1)
                flush.fill_(1)
        fit.synchronize()
        torch.cuda.synchronize()
    step_ms, nt = fit.timing()
    fit.set_timing(False)
    assert nt == K
    chi2 = fit.chi2()
    if ws > 1:
        t = torch.tensor([step_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        step_ms = float(t[0])
        dist.barrier()
    fit.close()
    value = ws * n * K / (step_ms / 1e3)

    # end to end through the public API from pinned host buffers
    e2e_s = None if args.no_e2e else _e2e(B, wl, Y, sig, Vp, sp, stream, n, K, ws)

    roof = roofline(args.workload, wl.precision, n, step_ms / K)
    line = None
    if rank == 0:
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            import oracle as O
            O.build()
            v, dt, _ = cpu_baseline(args.workload, args.cpu_sample, args.cpu_steps)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"first {args.cpu_sample} particles of {wl.name}, {args.cpu_steps} steps, "
                             f"{dt:.1f} s single-threaded FP64",
                   "host": host_cpu()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": step_ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if wl.precision == "fp64" else "f32+i64",
            "data": "synthetic",
            "config": {"workload": wl.name, "n_particles": n, "observables": wl.J,
                       "prior_grid": f"{wl.prior['nE']}x{wl.prior['nx']} every {wl.prior['update_every']}",
                       "dt": wl.params["dt"], "precision": wl.precision,
                       "timed_window": f"starts at a prior-update step; {prior_steps_in(t_start, K, every)} of the "
                                       f"{K} timed steps bin the priors (every {every})",
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "parallelism": f"{ws} independent fit(s), one per GPU", "chi2_per_J_end": chi2 / wl.J},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": None if e2e_s is None else {
                "value": ws * n * K / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 7 * 8 * n / K, "d2h_bytes_per_step": 8 + 8 * n / K,
                "note": "load from pinned host memory once, K x (step + chi^2 read), weights read"},
            "gpu_launches": K,  # one step kernel per step (the finalize runs in its last block)
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c5")
    ap.add_argument("--cpu-sample", type=int, default=200_000)
    ap.add_argument("--cpu-steps", type=int, default=60)
    ap.add_argument("--ref-sample", type=int, default=10_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="override the particle count (profiling)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None, help="override (profiling)")
    ap.add_argument("--fits", default=None, help="c5: comma-separated fit indices instead of all 96 (profiling)")
    ap.add_argument("--shape", default=None, help="c5: block,blocks_per_sm instead of the autotuner "
                                                  "(profiling; the segment is the library default)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_batch(args)
    if _dist()[0] > 1:
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
