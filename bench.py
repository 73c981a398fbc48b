#!/usr/bin/env python3
"""Benchmark of the fused log-likelihood + gradient + Hessian-diagonal evaluation.

One step = one hawkes_hess_diag call (FP32C) on the 100,000-event synthetic
workload (2,000 x 2,000 km, 1,500 days, 556 hotspots, log-rates N(0, 0.25)):
pack, row pass, row finish with the integral term, reduction, column pass.
It prints one JSON line:

  value     N(N-1) pair-interactions per second, summed over ranks (inputs resident)
  e2e       the same metric through the C-ABI with host buffers: every step copies
            x, y, t, r from pinned host memory and reads loglik, gradient and Hessian back
  roofline  the row pass (dominant kernel) against the FP32 pipe (ALU bound)
  cpu_baseline  the FP64 oracle on this host's cores, on a bounded sample of rows
  hmc       ESS/s of a short preconditioned HMC chain on the 23,422-event workload
  hmc_tree_mass  the same chain with the tree-structured mass on the log-rates
  predictive  posterior-predictive simulation 30 days ahead of that workload
            for 4,096 parameter settings (draws/s)
  surrogate the learned gradient surrogate at 500,000 events: 20,000 exact
            warm-up pairs, surrogate HMC against exact HMC from the same state
            (acceptance, surrogate gradient error, ESS/s, gains)
  parity    per-output errors of the timed results against the stored FP64
            oracle evaluation of the workload
  roofline_st  the space-time passes (the sampler's path) over the pairs they evaluate

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--shards]

With --impl reference the FP64 CPU oracle runs instead (on rank 0 only), each
step a bounded sample of the same workload.  N > 1 under torchrun runs N
independent replicas (the evaluation needs no exchange between GPUs); with
--shards the N ranks instead split one evaluation (row shards, an all-gather
of per-tile records, column shards, an all-gather of the entries) and the
line reports strong scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2103_03348_b300 import synth  # noqa: E402

METRIC = "loglik+grad+Hdiag pair-interactions/s and % FP32 roofline at N=1e5; HMC ESS/s"
UNIT = "pair-interactions/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 126 MB L2

# FP32 pipe: the device's SM count (148 on B300) x 128 lanes, one
# FADD/FMUL/FFMA per lane per clock, at the maximum SM clock (2,032 MHz on
# B300, read from nvidia-smi during the timed region): 38.49e12 lane-slots/s.
LANES, SM_MAX_MHZ_DEFAULT = 128, 2032.0

# Algorithmic FP32 lane-slots per pair (see the design notes): background terms
# for every ordered pair, excitation and column terms for causal pairs inside
# the exact FP32 underflow band.  A column pair costs 7: two differences, one
# add (g^ + r^) and two FMAs for the exponent d'^2 - g^ - r^ in the
# excitation's scaled coordinates, and the two accumulations.
ROW_BG_SLOTS, ROW_EXC_SLOTS, COL_SLOTS = 14, 7, 7
# A coarser count, also reported: every ordered pair charged the full
# excitation and mask work (26 slots), and 10 per column pair.
COARSE_ROW_SLOTS, COARSE_COL_SLOTS = 26, 10


def workload_config(w):
    return {"workload": f"{w.name}: 2000x2000 km, 1500 d, 556 hotspots (sigma 20 km), offspring 0.5, "
                        f"omega 0.1/d, h 5 km, log-rates N(0,0.25)",
            "n_events": w.n, "params": [float(v) for v in w.params], "precision": "fp32c",
            "outputs": "loglik + gradient[6+N] + Hessian diagonal[6+N]",
            "l2": "flushed between timed steps (256 MB write); inputs 3.2 MB would otherwise stay in L2"}


def band_pairs(w) -> int:
    """Causal pairs whose FP32 excitation term can exceed 2^-128 (the exact underflow band)."""
    log2e = 1.4426950408889634
    cut = (128.0 + float(np.max(w.r)) * log2e) / (w.params[4] * log2e)
    hi = np.searchsorted(w.t, w.t, side="left")           # first index with t == t_n (sources strictly before)
    lo = np.searchsorted(w.t, w.t - cut, side="left")     # first index inside the band
    return int(np.sum(hi - lo))


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), float(f[3]), f[5], f[6], f[7], f[8]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        load = [r for r in rows if r[2] > 150.0] or rows
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# FP64 oracle on the host (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample_rate(w, target_s: float = 12.0, rng_seed: int = 0, threads=None):
    """Pairs/s of the FP64 oracle on a bounded row/column sample of the workload
    (on `threads` host threads; all of them by default).

    A full evaluation visits every (row, source) pair in the row loop and every
    source's later targets in the column loop.  The sample evaluates k whole
    rows (all N sources, with the derivative sums) and k whole columns (all
    later targets); the rate is k(N-1) definition pairs per (row + column) time.
    """
    import oracle
    rng = np.random.default_rng(rng_seed)
    threads = oracle.max_threads() if threads is None else int(threads)
    lam_stub = np.ones(w.n)  # column sums are timed with unit intensities: same work, values unused

    def run(k):
        idx = np.sort(rng.choice(w.n, k, replace=False))
        t0 = time.perf_counter()
        oracle.rows(w.x, w.y, w.t, w.r, w.params, idx, threads=threads)
        oracle.rate_terms(w.x, w.y, w.t, w.r, w.params, lam_stub, idx, threads=threads)
        return time.perf_counter() - t0

    oracle.build()  # compile/load outside the timed sample
    k = max(threads, 8)
    dt = run(k)
    while dt < 0.05 * target_s and k < w.n:  # grow the pilot until its time is measurable
        k = min(w.n, 4 * k)
        dt = run(k)
    k2 = int(min(w.n, max(k, k * target_s / max(dt, 1e-3))))
    dt2 = run(k2)
    return k2 * (w.n - 1) / dt2, threads, k2, dt2


def small_config_table(dev, stream, all_threads):
    """The FP64 oracle in full at the two small configurations (2,000 and 23,422
    events; one thread and all threads, the 23,422-event single-thread figure
    on a row/column sample), beside the GPU's FP64 and FP32C evaluations of the
    same workloads (CUDA events, inputs resident, median of 5 after 2 warm-ups)."""
    import oracle
    import torch
    from paper_2103_03348_b300 import hawkes
    out = {}
    for name in ("unit_square", "ebola_like"):
        wc = synth.make(name)
        pairs_c = wc.n * (wc.n - 1)
        row = {"n_events": wc.n}
        t0 = time.perf_counter()
        oracle.evaluate(wc.x, wc.y, wc.t, wc.r, np.array(wc.params), want=2, threads=all_threads)
        row["oracle_all_threads_s"] = time.perf_counter() - t0
        row["oracle_threads"] = all_threads
        if wc.n <= 5000:
            t0 = time.perf_counter()
            oracle.evaluate(wc.x, wc.y, wc.t, wc.r, np.array(wc.params), want=2, threads=1)
            row["oracle_one_thread_s"] = time.perf_counter() - t0
        else:
            rate1, _, k1, dt1 = oracle_sample_rate(wc, target_s=4.0, rng_seed=2, threads=1)
            row["oracle_one_thread_s"] = pairs_c / rate1
            row["oracle_one_thread_note"] = f"extrapolated from {k1} whole rows + columns in {dt1:.1f} s"
        to_dev = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
        x, y, t, r = to_dev(wc.x), to_dev(wc.y), to_dev(wc.t), to_dev(wc.r)
        for prec in ("fp64", "fp32c"):
            ms_ = []
            for i in range(7):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hawkes._call("hess", x, y, t, r, wc.params, prec, stream=stream, check=False)
                e1.record(stream)
                e1.synchronize()
                if i >= 2:
                    ms_.append(e0.elapsed_time(e1))
            row[f"gpu_{prec}_ms"] = float(np.median(ms_))
        row["pairs_per_s"] = {"oracle_all_threads": pairs_c / row["oracle_all_threads_s"],
                              "oracle_one_thread": pairs_c / row["oracle_one_thread_s"],
                              "gpu_fp64": pairs_c / (row["gpu_fp64_ms"] * 1e-3),
                              "gpu_fp32c": pairs_c / (row["gpu_fp32c_ms"] * 1e-3)}
        out[wc.name] = row
    return out


def cpu_info():
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return model


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = synth.make("large")
    steps, warmup = args.steps, args.warmup
    per_step_s = max(0.2, min(2.0, 150.0 / max(steps + warmup, 1)))
    rates = []
    threads = k = 0
    for i in range(warmup + steps):
        rate, threads, k, dt = oracle_sample_rate(w, target_s=per_step_s, rng_seed=i)
        if i >= warmup:
            rates.append(rate)
    value = float(statistics.median(rates))
    ms = w.n * (w.n - 1) / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{k} whole rows + {k} whole columns of the N={w.n} workload per step "
                                       f"(FP64 C oracle, OpenMP over rows; CPU: {cpu_info()})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def profile_traffic():
    """DRAM traffic per row-pass launch from the committed ncu summary, if none of
    the row kernel's sources has changed since it was captured (the summary lists
    a digest per source file)."""
    path = os.path.join(ROOT, "profiles", "row32_large_N100000.txt")
    csrc = os.path.join(ROOT, "paper_2103_03348_b300", "csrc")
    try:
        digests, traffic = {}, None
        for line in open(path).read().splitlines():
            if line.startswith("source_sha256_16 (") and ":" in line:
                name = line[len("source_sha256_16 ("):line.index(")")]
                digests[name] = line.split(":", 1)[1].strip()
            elif line.startswith("dram_bytes_per_launch:"):
                traffic = float(line.split(":", 1)[1])
        if traffic is None or "k_row32.cu" not in digests:
            return None
        for name, want in digests.items():
            if hashlib.sha256(open(os.path.join(csrc, name), "rb").read()).hexdigest()[:16] != want:
                return None
        return traffic
    except (OSError, ValueError):
        return None


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2103_03348_b300 import build, hawkes

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.make("large")
    n = w.n
    pairs = n * (n - 1)
    to_dev = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    x, y, t, r = to_dev(w.x), to_dev(w.y), to_dev(w.t), to_dev(w.r)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    out = {"loglik": torch.empty((), dtype=torch.float64, device=dev),
           "grad": torch.empty(6 + n, dtype=torch.float64, device=dev),
           "hdiag": torch.empty(6 + n, dtype=torch.float64, device=dev),
           "status": torch.empty((), dtype=torch.int32, device=dev)}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]  # step start/end, row start/end, col start/end

    prec = args.kernel_precision  # fp32c unless a --kernel-only profiling run asks for another

    def step(timed=True):
        hawkes._call("hess", x, y, t, r, w.params, prec, stream=stream, check=False, out=out,
                     phase_events=ev[2:6] if timed else None)

    from paper_2103_03348_b300 import replicas

    barrier = replicas.barrier

    # correctness gate before timing
    step(False)
    torch.cuda.synchronize()
    if int(out["status"].item()) != 0:
        raise RuntimeError(f"status {int(out['status'].item())}: {hawkes.strerror(int(out['status'].item()))}")

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    def timed_steps(k, call, phases=False):
        """k steps enqueued back to back, each bracketed by its own events with an
        untimed L2 flush before it; one synchronize at the end, so that the host's
        launch work overlaps the device's and only device time is measured.
        Returns the per-step milliseconds (and the row / column phase times)."""
        marks = []
        for _ in range(k):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(6 if phases else 2)]
            flush.zero_()  # untimed: evicts the L2 between steps
            e[0].record(stream)
            call(e[2:6] if phases else None)
            e[1].record(stream)
            marks.append(e)
        torch.cuda.synchronize()
        ms_ = [e[0].elapsed_time(e[1]) for e in marks]
        if not phases:
            return ms_
        return ms_, [e[2].elapsed_time(e[3]) for e in marks], [e[4].elapsed_time(e[5]) for e in marks]

    def fused(phase):
        hawkes._call("hess", x, y, t, r, w.params, prec, stream=stream, check=False, out=out, phase_events=phase)

    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local_rank) as clk:
        step_ms, row_ms, col_ms = timed_steps(args.steps, fused, phases=True)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    value, ms = replicas.aggregate_throughput(pairs, float(np.mean(step_ms)), dev)

    if args.kernel_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms, "precision": prec,
                              "row_ms": float(np.mean(row_ms)), "col_ms": float(np.mean(col_ms)),
                              "steps": args.steps, "warmup": args.warmup, "kernel_only": True}), flush=True)
        return 0

    # end to end through the public API with host buffers: every step uploads x, y, t, r from pinned
    # host memory and reads loglik, gradient and Hessian diagonal back.  Two device sets of inputs and
    # outputs and a copy stream let step i+1's upload and step i's read-back run during step i's
    # evaluation (a set is refilled only once the evaluation that used it has finished); the L2 flush
    # before each evaluation is inside the timed region here.  Time = first upload to last read-back.
    pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory()  # noqa: E731
    host_in = (pin(w.x), pin(w.y), pin(w.t), pin(w.r))
    e2e_steps = max(3, min(args.steps, 30))
    sets = [((x, y, t, r), out), (tuple(torch.empty_like(a) for a in (x, y, t, r)),
                                  {k: torch.empty_like(v) for k, v in out.items()})]
    host_out = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items() if k != "status"}
                for _ in range(e2e_steps)]
    copy_s = torch.cuda.Stream(device=dev)
    uploaded = [torch.cuda.Event() for _ in range(2)]
    evaluated = [torch.cuda.Event() for _ in range(2)]
    t_first, t_last = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(i):
        dins, _ = sets[i % 2]
        with torch.cuda.stream(copy_s):
            if i >= 2:
                copy_s.wait_event(evaluated[i % 2])  # the set's previous evaluation has read its inputs
            for hsrc, dsrc in zip(host_in, dins):
                dsrc.copy_(hsrc, non_blocking=True)
            uploaded[i % 2].record(copy_s)

    def e2e_pass():
        torch.cuda.synchronize()
        t_first.record(copy_s)
        upload(0)
        for i in range(e2e_steps):
            if i + 1 < e2e_steps:
                upload(i + 1)
            (dx, dy, dt, dr), dout = sets[i % 2]
            stream.wait_event(uploaded[i % 2])
            with torch.cuda.stream(stream):
                flush.zero_()
            hawkes._call("hess", dx, dy, dt, dr, w.params, prec, stream=stream, check=False, out=dout)
            evaluated[i % 2].record(stream)
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(evaluated[i % 2])
                for k, hdst in host_out[i].items():
                    hdst.copy_(dout[k], non_blocking=True)
        t_last.record(copy_s)
        t_last.synchronize()
        return t_first.elapsed_time(t_last) / e2e_steps

    e2e_pass()  # warm-up: first use of the second set and of the copy stream
    e2e_ms = [e2e_pass()]
    if not all(np.array_equal(host_out[-1][k].numpy(), out[k].cpu().numpy()) for k in host_out[-1]):
        raise RuntimeError("the end-to-end pass read back other results than the resident evaluation")
    e2e_value = world * pairs / (float(np.mean(e2e_ms)) * 1e-3)

    # the same evaluation with exact background band skipping (bit-identical results)
    k_alt = max(3, min(args.steps, 50))
    band_out = {k: torch.empty_like(v) for k, v in out.items()}
    ws_band = torch.empty(hawkes.workspace_size(n, "fp32c_band"), dtype=torch.uint8, device=dev)
    band = lambda _: hawkes._call("hess", x, y, t, r, w.params, "fp32c_band", stream=stream, check=False,  # noqa: E731
                                  out=band_out, workspace=ws_band)
    timed_steps(3, band)  # warm-up
    band_ms = timed_steps(k_alt, band)

    # the same evaluation on space-time tiles (events regrouped by location inside
    # time slabs; group pairs whose FP32 terms all underflow are skipped; results
    # equal FP32C's up to summation order), event preparation included
    ws_st = torch.empty(hawkes.workspace_size(n, "fp32c_st"), dtype=torch.uint8, device=dev)
    st = lambda ph: hawkes._call("hess", x, y, t, r, w.params, "fp32c_st", stream=stream, check=False,  # noqa: E731
                                 out=band_out, workspace=ws_st, phase_events=ph)
    timed_steps(3, st)  # warm-up
    st_ms, st_row_ms, st_col_ms = timed_steps(k_alt, st, phases=True)
    st_pairs = hawkes.st_live_pairs(n, ws_st, stream=stream)  # the pairs those passes evaluated

    # per-output error of the timed results against the stored full FP64 oracle evaluation
    parity = {"reference": "tests/golden/large_N100000.npz (full FP64 oracle evaluation of this workload)",
              "fp32c": parity_report(w, out), "fp32c_st": parity_report(w, band_out)}

    # FP64 GPU path on the same workload (speedup of FP32C over it)
    fp64_ms = []
    for i in range(3):
        ev[0].record(stream)
        hawkes._call("hess", x, y, t, r, w.params, "fp64", stream=stream, check=False)
        ev[1].record(stream)
        ev[1].synchronize()
        if i > 0:
            fp64_ms.append(ev[0].elapsed_time(ev[1]))

    # HMC ESS/s: the preconditioned chains of the HMC configuration (23,422
    # events, 1,610 free log-rates, 20 leapfrog steps, 2,000 iterations after
    # 200 of warm-up, mass from the Hessian diagonal every 100), on space-time
    # tiles, one chain per seed; about 12 s each.  One chain's slowest ESS is
    # itself a noisy statistic (theta0 trades off against the sequenced
    # log-rates along a ridge that a diagonal mass follows slowly, and how
    # often a chain crosses it varies between seeds), so each statistic is
    # reported as the median over the chains, with every chain listed.
    hmc_summary = hmc_tree_summary = None
    if not args.no_hmc:
        from paper_2103_03348_b300 import run_hmc
        keys = ("workload", "n_events", "n_rates", "precision", "mass", "iters", "warmup", "leapfrog_steps",
                "accept_rate", "sampling_seconds", "ms_per_gradient",
                "ess_globals", "ess_rates", "ess_per_s_globals", "ess_per_s_rates")
        seeds = list(range(max(1, args.hmc_seeds)))
        runs = [run_hmc.run("fp32c_st", iters=args.hmc_iters, warmup=args.hmc_warmup, device=str(dev), seed=sd)
                for sd in seeds]
        med = lambda xs: float(np.median(xs))  # noqa: E731
        hmc_summary = {k: runs[0][k] for k in keys[:8]}
        hmc_summary.update({k: med([r[k] for r in runs]) for k in ("accept_rate", "sampling_seconds", "ms_per_gradient")})
        for k in ("ess_globals", "ess_rates", "ess_per_s_globals", "ess_per_s_rates"):
            hmc_summary[k] = {q: med([r[k][q] for r in runs]) for q in ("min", "median", "max")}
        hmc_summary["chains"] = {
            "seeds": seeds, "statistic": "median over the chains of each per-chain statistic",
            "per_chain": [{"seed": sd, "sampling_seconds": r["sampling_seconds"],
                           "ess_per_s_globals": r["ess_per_s_globals"], "ess_per_s_rates": r["ess_per_s_rates"],
                           "ess_each_global": r["ess_each_global"],
                           "slowest_global": min(r["ess_each_global"], key=r["ess_each_global"].get)}
                          for sd, r in zip(seeds, runs)]}
        # one chain with the tree-structured mass on the rates (the prior's
        # full precision plus the likelihood's curvature), seed 0; about 13 s more
        h = run_hmc.run("fp32c_st", iters=args.hmc_iters, warmup=args.hmc_warmup, device=str(dev), mass="tree")
        hmc_tree_summary = {k: h[k] for k in keys}
        hmc_tree_summary["chains"] = {"seeds": [0], "slowest_global": min(h["ess_each_global"],
                                                                           key=h["ess_each_global"].get)}

    pred_summary = None if args.no_predictive else predictive_bench(dev, stream)

    # the learned surrogate at its own configuration: 500,000 events, 20,000 exact
    # warm-up pairs, surrogate HMC (exact accept) against exact HMC from the same
    # state with the same mass and step size, on space-time tiles; a few minutes
    sur_summary = None
    if world == 1 and not args.no_surrogate:
        from paper_2103_03348_b300 import run_surrogate
        sur_summary = run_surrogate.run(n=args.surrogate_n, pairs=20_000, iters=2000, exact_iters=500,
                                        precision="fp32c_st", device=str(dev))
    from paper_2103_03348_b300 import peaks
    alu = peaks.measure(str(dev))

    if rank != 0:
        return 0

    pb = band_pairs(w)
    row_slots = ROW_BG_SLOTS * pairs + ROW_EXC_SLOTS * pb
    col_slots = COL_SLOTS * pb
    row_t = float(np.mean(row_ms)) * 1e-3
    col_t = float(np.mean(col_ms)) * 1e-3
    achieved = row_slots / row_t
    clocks = clk.summary()
    traffic = profile_traffic()
    sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    sm_max_mhz = float(clocks.get("sm_max_mhz") or SM_MAX_MHZ_DEFAULT)
    FP32_PEAK_SLOTS = sms * LANES * sm_max_mhz * 1e6
    peak_t = FP32_PEAK_SLOTS / 1e12
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        # the oracle's OpenMP thread count persists between calls: read the host's count
        # once, before any one-thread run, and pass it explicitly
        all_threads = oracle.max_threads()
        rate, threads, k, dt = oracle_sample_rate(w, target_s=12.0, threads=all_threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{k} whole rows (all {n} sources, with derivative sums) + {k} whole columns of the "
                         f"N={n} workload in {dt:.1f} s; rate = k(N-1)/time (CPU: {cpu_info()})"}
        rate1, _, k1, dt1 = oracle_sample_rate(w, target_s=4.0, rng_seed=1, threads=1)
        cpu["single_thread"] = {"value": rate1, "unit": UNIT, "cores": 1,
                                "sample": f"{k1} whole rows + {k1} whole columns in {dt1:.1f} s on one thread"}
        cpu["small_configs"] = small_config_table(dev, stream, all_threads)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(w),
        "roofline": {"bound": "alu", "kernel": "row32_kernel (row pass)", "achieved": achieved / 1e12,
                     "peak": peak_t, "unit": "T FP32 lane-slots/s", "frac": achieved / FP32_PEAK_SLOTS,
                     "traffic": traffic,
                     "peak_source": f"{sms} SMs (device properties) x 128 FP32 lanes x {sm_max_mhz:.0f} MHz "
                                    f"(maximum SM clock); unit counts, no FP32 figure is measured by the driver",
                     "sms": sms,
                     "algorithmic_slots_per_launch": row_slots,
                     "row_ms": row_t * 1e3, "col_ms": col_t * 1e3,
                     "col_frac": col_slots / col_t / FP32_PEAK_SLOTS,
                     "step_frac": (row_slots + col_slots) / (ms * 1e-3) / FP32_PEAK_SLOTS,
                     "frac_at_sampled_clock": (achieved / (sms * LANES * clocks["sm_mhz"] * 1e6)
                                               if clocks.get("sm_mhz") else None),
                     "band_pairs": pb,
                     "measured_alu_peaks": {"ffma2_T_lane_slots_per_s": alu["ffma2_lane_fma_per_s"] / 1e12,
                                            "ex2_T_per_s": alu["ex2_per_s"] / 1e12,
                                            "dfma_T_per_s": alu["dfma_per_s"] / 1e12,
                                            "source": "the library's f32x2 FMA, MUFU exp2 and FP64 FMA chains"},
                     "frac_of_measured_ffma2": achieved / alu["ffma2_lane_fma_per_s"],
                     # the MUFU bound beside the FP32 one: one ex2 per ordered pair (background)
                     # plus one per causal pair in the band (excitation)
                     "mufu": {"ex2_per_launch": pairs + pb,
                              "achieved_T_per_s": (pairs + pb) / row_t / 1e12,
                              "peak_T_per_s": alu["ex2_per_s"] / 1e12,
                              "frac": (pairs + pb) / row_t / alu["ex2_per_s"],
                              "peak_source": "measured MUFU exp2 chain (measured_alu_peaks)"},
                     "frac_survey": (COARSE_ROW_SLOTS * pairs) / row_t / FP32_PEAK_SLOTS,
                     "col_frac_survey": (COARSE_COL_SLOTS * pb) / col_t / FP32_PEAK_SLOTS,
                     "survey_count": "26 FP32 slots per ordered pair (excitation and masks charged to every "
                                     "pair), 10 per causal column pair in the band"},
        "parity": parity,
        "roofline_st": st_roofline(st_pairs, st_row_ms, st_col_ms, FP32_PEAK_SLOTS),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * 8 * n,
                "d2h_bytes_per_step": 8 + 2 * 8 * (6 + n), "ms_per_step": float(np.mean(e2e_ms))},
        "cpu_baseline": cpu,
        "gpu_launches": hawkes.kernels_per_call("hess", "fp32c") * args.steps,
        "clocks": clocks,
        "band_skip": {"precision": "fp32c_band (tile pairs whose background terms all underflow are skipped; "
                                   "results identical bit for bit)",
                      "ms_per_step": float(np.mean(band_ms)),
                      "pair_interactions_per_s": world * pairs / (float(np.mean(band_ms)) * 1e-3),
                      "speedup_over_fp32c": ms / float(np.mean(band_ms))},
        "spacetime": {"precision": "fp32c_st (events regrouped by Hilbert index inside slabs of 4,096; group pairs "
                                   "whose FP32 terms all underflow are skipped; results equal fp32c's up to "
                                   "summation order)",
                      "ms_per_step": float(np.mean(st_ms)),
                      "pair_interactions_per_s": world * pairs / (float(np.mean(st_ms)) * 1e-3),
                      "speedup_over_fp32c": ms / float(np.mean(st_ms)),
                      "speedup_over_band": float(np.mean(band_ms)) / float(np.mean(st_ms))},
        "fp64_gpu_path": {"ms_per_step": float(np.mean(fp64_ms)),
                          "speedup_fp32c_over_fp64": float(np.mean(fp64_ms)) / ms},
        "wall_s_timed_region": wall,
        "hmc": hmc_summary,
        "hmc_tree_mass": hmc_tree_summary,
        "predictive": pred_summary,
        "surrogate": sur_summary,
    }
    print(json.dumps(line), flush=True)
    return 0


def st_roofline(st_pairs, row_ms, col_ms, peak):
    """The space-time passes (the path the sampler runs) against the FP32 pipe,
    counting the pairs inside the group pairs they evaluate: 14 slots per
    background pair and 7 per excitation pair in the row pass (the per-pair
    counts of the full evaluation), 7 per column pair."""
    row_t, col_t = float(np.mean(row_ms)) * 1e-3, float(np.mean(col_ms)) * 1e-3
    row_slots = ROW_BG_SLOTS * st_pairs["row_background_pairs"] + ROW_EXC_SLOTS * st_pairs["row_excitation_pairs"]
    col_slots = COL_SLOTS * st_pairs["column_pairs"]
    return {"bound": "alu", "kernel": "row32_st_kernel (space-time row pass)", "unit": "T FP32 lane-slots/s",
            "achieved": row_slots / row_t / 1e12, "peak": peak / 1e12, "frac": row_slots / row_t / peak,
            "row_ms": row_t * 1e3, "col_ms": col_t * 1e3, "col_frac": col_slots / col_t / peak,
            "algorithmic_slots_per_launch": row_slots, "col_slots_per_launch": col_slots, **st_pairs,
            "count": "pairs inside the live group pairs, counted on the device by the passes' own "
                     "classification (hawkes_st_live_pairs)"}


def parity_report(w, out):
    """Relative errors of a device result against the stored oracle evaluation:
    loglik, and max / median of the scaled entry errors (denominator
    max(|ref_i|, 1e-3 max|ref|)) of the global and log-rate entries of the
    gradient and Hessian diagonal; None when the fixture is absent or was made
    from other inputs."""
    import hashlib
    path = os.path.join(ROOT, "tests", "golden", "large_N100000.npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    d = hashlib.sha256()
    for a in (w.x, w.y, w.t, w.r, np.asarray(w.params, float)):
        d.update(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    if str(z["input_sha256"]) != d.hexdigest():
        return None
    ll, g, h = float(out["loglik"].item()), out["grad"].cpu().numpy(), out["hdiag"].cpu().numpy()

    def vec(a, b):
        den = np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
        e = np.abs(a - b) / den
        return {"max": float(e.max()), "median": float(np.median(e))}

    nrm = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    return {"loglik": abs(ll - float(z["loglik"])) / abs(float(z["loglik"])),
            "grad_globals": vec(g[:6], z["grad"][:6]), "grad_rates": vec(g[6:], z["grad"][6:]),
            "grad_norm": nrm(g, z["grad"]),
            "hdiag_globals": vec(h[:6], z["hdiag"][:6]), "hdiag_rates": vec(h[6:], z["hdiag"][6:]),
            "hdiag_norm": nrm(h, z["hdiag"])}


def run_sharded(args, rank, world, local_rank):
    """--shards: the evaluation split over the ranks (strong scaling): each
    rank runs its shard's row phase, the per-tile records are all-gathered
    (NCCL), each rank runs its column phase and the per-event entries are
    all-gathered, so that every rank holds the whole result.  value = the
    whole problem's N(N-1) pairs per second (max over ranks of the step time)."""
    import torch
    from paper_2103_03348_b300 import build, hawkes, replicas, shard
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = synth.make("large")
    to_dev = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    x, y, t, r = to_dev(w.x), to_dev(w.y), to_dev(w.t), to_dev(w.r)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sh = shard.Shard(w.n, "fp32c", rank, world, dev) if world > 1 else None

    def step():
        if world > 1:
            return shard.distributed_evaluate(x, y, t, r, w.params, "fp32c", "hess", shard=sh)
        return hawkes.hess_diag(x, y, t, r, w.params, "fp32c")

    ref = hawkes.hess_diag(x, y, t, r, w.params, "fp32c")
    out = step()
    if not all(torch.equal(a, b) for a, b in zip(out, ref)):
        raise RuntimeError("the sharded evaluation differs from the unsharded call")
    for _ in range(args.warmup):
        flush.zero_()
        step()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        replicas.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t_ms = float(np.mean(ms))
    t_max = replicas.max_over_ranks(t_ms, dev)
    if rank == 0:
        pairs = w.n * (w.n - 1)
        print(json.dumps({"metric": METRIC, "value": pairs / (t_max * 1e-3), "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max,
                          "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic", "config": dict(workload_config(w), parallelism=f"shards{world}"),
                          "sharded": {"records_bytes": shard.n_records(w.n) * shard.RECORD_DOUBLES * 8,
                                      "exchange": "per-tile records, then per-event entries (NCCL all-gather)",
                                      "bit_identical_to_unsharded": True}}), flush=True)
    return 0


def predictive_bench(dev, stream):
    """Posterior-predictive simulation: 30 days ahead of the 23,422-event
    history with 1,610 free log-rates, for 4,096 posterior-like parameter
    settings, one block per setting; CUDA events around each batch."""
    from paper_2103_03348_b300 import run_predictive
    return run_predictive.run(samples=4096, horizon=30.0, reps=3, device=str(dev))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hmc", action="store_true", help="skip the short HMC chain (ESS/s)")
    ap.add_argument("--no-predictive", action="store_true", help="skip the posterior-predictive simulation")
    ap.add_argument("--shards", action="store_true",
                    help="time the evaluation split over the ranks (strong scaling) instead of replicas")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate chains (N=500,000)")
    ap.add_argument("--surrogate-n", type=int, default=500_000, help="events of the surrogate block's workload")
    ap.add_argument("--hmc-iters", type=int, default=2000)
    ap.add_argument("--hmc-warmup", type=int, default=200)
    ap.add_argument("--hmc-seeds", type=int, default=3, help="HMC chains (seeds 0..k-1) behind the hmc line")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time the resident-input steps only (no e2e, FP64 path or CPU baseline); for profilers")
    ap.add_argument("--kernel-precision", default="fp32c", choices=["fp32c", "fp32c_band", "fp32c_st"],
                    help="with --kernel-only: the precision of the timed step (to profile the other FP32C forms)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.kernel_precision != "fp32c" and not args.kernel_only:
        ap.error("--kernel-precision applies to --kernel-only runs")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.shards:
            return run_sharded(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
