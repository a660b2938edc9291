#!/usr/bin/env python
"""Baryon-block throughput on GB300 (blocks/s) for the batched L=32 workload, by default.

Default workload ``l32_batch_48t_6noise``: L = 32 (32768 sites), N_ev = 128, 48 time slices
x 6 noise triples whose dilution sizes are drawn from {32, 48, 64}, 9 momenta and a
4-triple baryon operator: 288 jobs of uneven size, 2592 blocks B[t][p][d1][d2][d3] per
step. One step = one ``bblock_compute_batch`` call over every job (projection of the three
quark lines for each spin used, fused diquark + contraction on the tensor cores, slab
reduction), replayed from a CUDA graph from the third identical call on. Inputs are seeded
synthetic draws (``workloads.py``) resident on the device.

The same line reports, on the same inputs:
* the plain FP64 form, timed per dilution size on one job each and extrapolated to the
  batch's job mix (``fp64_form``), and the headline form's speedup over it;
* the other FP64-accurate forms the same way (``fp64_accurate_forms``): double-float on the
  FP32 pipe and the Ozaki digit-product form on the tensor cores;
* per-block relative Frobenius errors of both against the CPU FP64 oracle on sampled
  entries of jobs taken from every wave (``oracle_check``);
* the tile autotuner with and without its learned cost model (``tuning``);
* the other mixed forms on a stated subset of the batch (``forms``);
* the L=24 single-noise workload as a secondary key (``secondary``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload NAME] [--form FORM]

Prints one JSON line (rank 0). Under torchrun every rank computes its own independent
inputs (weak scaling, no data-path collective); the timed region is bracketed by a barrier
and the maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import csv
import dataclasses
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

WORKLOAD = "l32_batch_48t_6noise"
SECONDARY = "l24_nev96_ndil32"
METRIC = "baryon blocks/s"
UNIT = "blocks/s"
# Peak of the FP64 pipe: the nominal 1.25 TFLOP/s of GB300 is 4 FP64 flop/clk/SM
# (2 DFMA) x 152 SMs x the 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 4 * 152 * 2.070e9 / 1e12
# Peak of the FP32 pipe (the double-float form's bound): 128 FP32 instructions/clk/SM x 152
# SMs x 2070 MHz, in tera-instructions per second.
FP32_INST_PEAK = 128 * 152 * 2.070e9 / 1e12


def _measured_peaks():
    """Dense BF16 tensor peak measured on the GB300s (cuBLAS burst), if present."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# BF16 (= FP16 on the same pipe) from the measured burst figure (fallback 1.9 PFLOP/s);
# TF32 = BF16 x the nominal dense ratio 1.1 / 2.25.
BF16_PEAK_TFLOPS = float(_measured_peaks().get("bf16_tflops", 1900.0))
BF16_PEAK_SOURCE = ("measured cuBLAS BF16 burst (MEASURED_PEAKS.json)"
                    if "bf16_tflops" in _measured_peaks() else "fallback 1.9 PFLOP/s")
TF32_PEAK_TFLOPS = BF16_PEAK_TFLOPS * 1.1 / 2.25
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

# name: (precision, BF16 products, MMA piece products, tensor peak TFLOP/s, tolerance)
FORMS = {
    "fp64": ("fp64", 6, 0, None, 1e-12), "df64": ("df64", 6, 0, None, 1e-12),
    "bf16x6": ("bf16", 6, 6, BF16_PEAK_TFLOPS, 1e-6),
    "bf16x9": ("bf16", 9, 9, BF16_PEAK_TFLOPS, 1e-6),
    "tf32x3": ("tf32x3", 6, 3, TF32_PEAK_TFLOPS, 1e-6),
    "bf16x3": ("bf16", 3, 3, BF16_PEAK_TFLOPS, 1e-4),
    "fp16x3": ("fp16x3", 6, 3, BF16_PEAK_TFLOPS, 1e-6),
    # FP64-accurate on the BF16 tensor cores: 28 digit products of the folded complex GEMM
    "ozaki": ("ozaki", 6, 28, BF16_PEAK_TFLOPS, 1e-12),
}
BATCH_HEAD = "fp16x3"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the sampled comparison with the CPU oracle")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU seconds of one oracle sample")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload: skip the tile autotuner (heuristic tiles)")
    ap.add_argument("--no-triplet", action="store_true",
                    help="skip the mode-triplet ordering's measurement")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the forms other than the headline and the FP64 form")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="batched workload: skip the FP64 form's comparison timing")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary single-noise workload")
    ap.add_argument("--form", choices=sorted(FORMS), default=None,
                    help="form of the headline number (default: %s for the batched workload, "
                    "fp64 for the others)" % BATCH_HEAD)
    ap.add_argument("--n-t", type=int, default=None,
                    help="time slices per step (default: the workload's); for profiling runs")
    ap.add_argument("--size-sweep", action="store_true",
                    help="instead of the throughput line: the contraction time's growth with "
                    "L and with N_dil (one JSON line)")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ algorithmic work

def spin_structure(spins):
    spins = [tuple(int(v) for v in s) for s in np.asarray(spins).reshape(-1, 3)]
    n_alpha = len({s[0] for s in spins})
    n_beta = len({s[1] for s in spins})
    pairs = len({(s[0], s[1]) for s in spins})
    return n_alpha, n_beta, pairs


def contraction_flops(X, nd, P, pairs):
    """Complex-arithmetic flops (cmul 6, complex FMA 8) of the contraction of one
    (time slice, noise triple) in the paper's ordering: diquark 42 per (pair, d1, d2, x);
    colour singlet with the spin-pair sum inside, 8 * 3 * pairs per (d1, d2, d3, x);
    momentum projection 8 P per (d1, d2, d3, x)."""
    d1, d2, d3 = nd
    return 42.0 * pairs * d1 * d2 * X + (24.0 * pairs + 8.0 * P) * d1 * d2 * d3 * X


def projection_flops(X, n_ev, nd, n_alpha, n_beta, pairs):
    """Eq. (2) as complex GEMMs: 8 * 3X * n_ev per output column."""
    return 8.0 * 3 * X * n_ev * (n_alpha * nd[0] + n_beta * nd[1] + pairs * nd[2])


def folded_gemm_flops(X, nd, P, pairs):
    """Useful flops of the folded contraction run on the tensor cores: one complex GEMM
    of M = d1 d2, N = P d3, K = 3 pairs X, 8 M N K (phase and colour sum folded in). With
    the row-factored phase P is the number of distinct n0 of the momenta instead."""
    return 8.0 * nd[0] * nd[1] * (P * nd[2]) * (3 * pairs * X)


def phase_columns(path, L, momenta):
    """Phase columns per d3 of the tensor-core GEMM: every momentum, or (row-factored
    path) the distinct x-components n0 mod L."""
    mom = np.asarray(momenta).reshape(-1, 3)
    return len({int(m[0]) % L for m in mom}) if path.startswith("tc_rows") else len(mom)


def contraction_df_inst(X, nd, P, pairs):
    """FP32 instructions of the double-float contraction's inner loops per (time slice,
    noise triple): 12 per double-float FMA (exact product error, TwoSum, lazy error sum),
    three per (pair, colour) in the singlet, four per momentum, 16 for the singlet's real and
    imaginary parts; per (d1, d2, d3, x)."""
    d1, d2, d3 = nd
    return (108.0 * pairs + 16.0 + 48.0 * P) * d1 * d2 * d3 * X


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_QUERY}", "--format=csv",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        time.sleep(0.25)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        if len(rows) < 2:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        head = [h.strip() for h in rows[0]]
        sm, smax, power, reasons = [], [], [], set()
        names = {"clocks_event_reasons.hw_slowdown": "hw_slowdown",
                 "clocks_event_reasons.hw_thermal_slowdown": "hw_thermal_slowdown",
                 "clocks_event_reasons.sw_thermal_slowdown": "sw_thermal_slowdown",
                 "clocks_event_reasons.sw_power_cap": "sw_power_cap"}
        for r in rows[1:]:
            if len(r) != len(head):
                continue
            d = {h.split(" ")[0]: v.strip() for h, v in zip(head, r)}
            try:
                sm.append(float(d["clocks.current.sm"].split()[0]))
                smax.append(float(d["clocks.max.sm"].split()[0]))
                power.append(float(d["power.draw"].split()[0]))
            except (KeyError, ValueError, IndexError):
                continue
            for k, v in names.items():
                if d.get(k, "").lower() == "active":
                    reasons.add(v)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle leg
#
# The CPU FP64 oracle is used in this one leg only: it is timed on a bounded sample (the
# cpu_baseline) and it evaluates sampled entries of GPU-computed blocks (the oracle check).

def samples(nd):
    """A few dilution indices of a line with nd columns: first, interior, last."""
    return sorted({0, nd // 3, (2 * nd) // 3 + 1, nd - 1})


def oracle_check(inp, outs, picks, tol):
    """Per-block relative Frobenius errors against the oracle on sampled entries.

    ``outs[k]`` are the GPU blocks of noise triple k (complex128, [n_t][P][d1][d2][d3], host
    or device); ``picks`` lists the (noise triple, time slice) jobs to check. For each job
    the oracle evaluates Eq. (2) then Eq. (1) on a few dilution columns per line (always the
    last one, in a tile's ragged edge); every momentum's sampled block is compared with the
    GPU's entries. Returns a summary dict."""
    import oracle
    w = inp.workload
    errs, worst = [], None
    t0 = time.perf_counter()
    for (k, t) in picks:
        nd = inp.ndil[k]
        ds = [samples(n) for n in nd]
        ref = oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[k][i][t] for i in range(3)],
                                    inp.momenta, inp.spins, inp.coeffs, *ds)
        o = outs[k][t]
        got = o.cpu().numpy() if hasattr(o, "cpu") else np.asarray(o)
        got = got[:, ds[0]][:, :, ds[1]][:, :, :, ds[2]]
        for p in range(ref.shape[0]):
            e = float(np.linalg.norm(got[p] - ref[p]) / np.linalg.norm(ref[p]))
            errs.append(e)
            if worst is None or e > worst[0]:
                worst = (e, k, t, p)
    return {"blocks_checked": len(errs), "jobs": [list(j) for j in picks],
            "entries_per_block": "4 x 4 x 4 sampled (d1, d2, d3), last index of each line included",
            "max": max(errs), "median": statistics.median(errs), "tolerance": tol,
            "worst_block": {"noise": worst[1], "t": worst[2], "p": worst[3]},
            "pass": bool(max(errs) <= tol), "oracle_seconds": time.perf_counter() - t0}


def oracle_sample(inp, target_s: float, threads=None, k=0):
    """Time the CPU FP64 oracle on a bounded sample of the workload (noise triple k).

    The oracle's OpenMP loop runs over d1, so the sample grows in steps of one d1 value per
    thread: first over d2 values, then over further d1 blocks, then over time slices,
    until it is about ``target_s`` seconds of CPU work. All momenta and all d3 are always
    included. Returns (blocks/s, threads, text)."""
    import oracle
    if threads is not None:
        oracle.set_num_threads(threads)
    w = inp.workload
    nd = inp.ndil[k]
    P = len(inp.momenta)
    n_t = inp.V.shape[0]
    n1 = max(1, min(nd[0], oracle.num_threads()))
    all3 = list(range(nd[2]))

    def run(t, d1s, d2s):
        oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[k][i][t] for i in range(3)],
                              inp.momenta, inp.spins, inp.coeffs, d1s, d2s, all3)

    run(0, list(range(n1)), [0])                 # warm-up (thread pool start)
    t0 = time.perf_counter()
    run(0, list(range(n1)), [0])                 # one d1 block x one d2 value
    t_unit = max(time.perf_counter() - t0, 1e-3)
    units = max(1, round(target_s / t_unit))
    k2 = min(nd[1], units)
    m1 = min(-(-nd[0] // n1), max(1, round(units / k2)))
    d1s = list(range(min(nd[0], m1 * n1)))
    n_ts = 1
    if len(d1s) == nd[0] and k2 == nd[1]:
        n_ts = min(n_t, max(1, round(units / (k2 * m1))))
    t0 = time.perf_counter()
    for t in range(n_ts):
        run(t, d1s, list(range(k2)))
    tk = time.perf_counter() - t0
    blocks = n_ts * P * len(d1s) * k2 / (nd[0] * nd[1])
    text = (f"{w.name} noise triple {k} (N_dil {nd[0]}): {n_ts} time slice(s), {P} momenta, "
            f"d1 in [0,{len(d1s)}) of {nd[0]}, d2 in [0,{k2}) of {nd[1]}, all {nd[2]} d3 = "
            f"{blocks:.4f} blocks in {tk:.2f} s on {n1} thread(s)")
    return blocks / tk, n1, text


def cpu_baseline(w, target_s):
    """The oracle on the host's cores (all, then one), on a bounded sample of workload w
    (for a batch: its largest-dilution noise triple, whose blocks cost the most)."""
    import oracle
    inp = workloads.generate(w, n_t=2)
    k = max(range(len(inp.ndil)), key=lambda q: inp.ndil[q][0])
    cores = oracle.num_threads()
    v, n1, sample = oracle_sample(inp, target_s, threads=cores, k=k)
    v1, _, sample1 = oracle_sample(inp, max(2.0, target_s / 3), threads=1, k=k)
    oracle.set_num_threads(cores)
    return {"value": v, "unit": UNIT, "cores": n1, "kind": "oracle", "sample": sample,
            "build": "gcc -O3 -fopenmp (no -march=native: the same source builds on x86-64 "
                     "and Arm hosts)",
            "one_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workloads.WORKLOADS[args.workload]
    inp = workloads.generate(w, n_t=2)
    k = max(range(len(inp.ndil)), key=lambda q: inp.ndil[q][0])
    oracle.build()
    vals, sample = [], ""
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    cores = oracle.num_threads()
    for i in range(args.warmup + args.steps):
        v, cores, sample = oracle_sample(inp, per_step, k=k)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded, workloads.py)",
        "config": {"workload": w.name, "L": w.L, "n_ev": w.n_ev,
                   "ndil": sorted({nd[0] for nd in inp.ndil}), "n_t": w.n_t,
                   "n_noise": w.n_noise, "n_mom": len(w.momenta), "n_spin": len(w.spins),
                   "form": "fp64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ helpers of our arm

def load_traffic(key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source; (bytes, record) or (None, None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    try:
        from paper_2211_16278_gb300 import build as cb
        rec = json.load(open(path)).get(key)
        if rec and rec.get("source_sha256") == cb.source_digest(rec.get("source")):
            return rec.get("dram_bytes_per_launch_full_workload"), rec
    except Exception:
        return None, None
    return None, None


def rank_inputs(w, rank: int, n_t=None):
    """Inputs of one rank: every rank draws its own time slices (its own seed), so the
    ranks share no work and exchange no data."""
    return workloads.generate(w, n_t=n_t, seed=w.seed + rank)


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (the timing that is reported)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, blocks_per_step: int, steps: int, seconds: float) -> float:
    """Whole-job blocks/s: the blocks of all ranks over the slowest rank's time."""
    return world * blocks_per_step * steps / seconds


def wave_picks(n_noise, n_t, per=3):
    """(noise triple, time slice) jobs spread over a batch in job order (noise-major), so
    that the first, interior and last waves are all represented."""
    n = n_noise * n_t
    idx = sorted({round(i * (n - 1) / (per * n_noise - 1)) for i in range(per * n_noise)}) \
        if n > 1 else [0]
    return [(j // n_t, j % n_t) for j in idx]


class Runner:
    """Device-side measurement of one workload: timed steps of a form on the created stream,
    CUDA events around every launch (graph replays included)."""

    def __init__(self, torch, bb, dev, local, world, barrier, stream):
        self.torch, self.bb, self.dev, self.local = torch, bb, dev, local
        self.world, self.barrier, self.stream = world, barrier, stream

    def context(self, w, form, max_nd):
        precision, products = FORMS[form][:2]
        return self.bb.bblock_create(w.L, w.n_ev, max_nd, precision, bf16_products=products,
                                     device=self.local)

    def measure(self, ctx, step, steps, warmup, sampler=None):
        """W untimed + K timed steps; timing events recorded from the first warm-up on, so
        the captured graph carries them and the timed steps are graph replays."""
        torch, bb = self.torch, self.bb
        bb.bblock_profile_enable(ctx, True)
        for _ in range(warmup):
            step()
        bb.bblock_status(ctx)
        bb.bblock_profile_read(ctx)  # reset
        torch.cuda.synchronize(self.dev)
        self.barrier()
        n_launch = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if sampler is not None:
            sampler.__enter__()
        torch.cuda.synchronize(self.dev)
        self.barrier()
        e0.record(self.stream)
        for _ in range(steps):
            step()
            n_launch += bb.bblock_last_launch_count(ctx)
        e1.record(self.stream)
        torch.cuda.synchronize(self.dev)
        self.barrier()
        if sampler is not None:
            sampler.__exit__(None, None, None)
        bb.bblock_status(ctx)
        t_ms = e0.elapsed_time(e1)
        prof = bb.bblock_profile_read(ctx)
        bb.bblock_profile_enable(ctx, False)
        t_ms = max_over_ranks(t_ms, self.world, self.dev)
        return t_ms, prof, n_launch


def tensor_roofline(form, prof, gemm_flops, alg_flops, steps, traffic, traffic_rec, path):
    """The contraction's algorithmic flops (the paper-ordering count of Eq. 1 per job: diquark,
    colour singlet with the pair sum inside, momentum projection) per launch over its
    average CUDA-event launch duration, against the pipe's measured peak. Beside it: the
    complex GEMM the tensor cores run on this path (N = phase columns x d3) and the MMA
    piece-product flops they execute for it."""
    nprod, peak = FORMS[form][2:4]
    nc, msc = prof.get("contract", (0, 0.0))
    if not nc:
        return None
    sec = msc / 1e3
    alg = alg_flops * steps / sec / 1e12
    execd = gemm_flops * nprod * steps / sec / 1e12
    return {"bound": "tensor", "kernel": "k_contract_oz" if form == "ozaki" else "k_contract_tc",
            "path": path,
            "achieved": alg, "peak": peak, "unit": "TFLOP/s", "frac": alg / peak,
            "flops": "algorithmic: Eq. 1 in the paper's ordering, 42 Pi D1D2 X + (24 Pi + 8 P) "
                     "D1D2D3 X per job (cmul 6, complex FMA 8)",
            "flops_per_launch": alg_flops * steps / nc,
            "traffic": traffic,
            "traffic_capture": traffic_rec.get("captured_workload") if traffic_rec else None,
            "peak_source": BF16_PEAK_SOURCE
                           + ("; TF32 = BF16 x 1.1/2.25 nominal" if form == "tf32x3" else ""),
            "gemm_tflops": gemm_flops * steps / sec / 1e12,
            "gemm_frac": gemm_flops * steps / sec / 1e12 / peak,
            "executed_tflops": execd, "executed_frac": execd / peak,
            "executed": ("MMA digit products: the path's complex GEMM x %d" if form == "ozaki"
                         else "MMA piece products: the path's complex GEMM x %d") % nprod,
            "launches": nc, "avg_launch_ms": msc / nc}


# The FP64 peak of the FP64 form's roofline: the DFMA rate bblock_probe_fp64 measures at the
# start of the run (set by run_ours), else the derived nominal figure.
FP64_PEAK = {"tflops": FP64_PEAK_TFLOPS,
             "source": "derived: 4 FP64 flop/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)"}


def fp64_roofline(prof, alg_flops, steps, traffic, traffic_rec):
    n_c, ms_c = prof.get("contract", (0, 0.0))
    if not n_c:
        return None
    achieved = alg_flops * steps / (ms_c / 1e3) / 1e12
    peak = FP64_PEAK["tflops"]
    return {"bound": "alu", "kernel": "k_contract_fp64", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_capture": traffic_rec.get("captured_workload") if traffic_rec else None,
            "peak_source": FP64_PEAK["source"],
            "flops": "paper-ordering complex count (cmul 6, complex FMA 8); the kernel "
                     "executes about 80/96 of it (three-multiplication complex products)",
            "flops_per_launch": alg_flops * steps / n_c,
            "launches": n_c, "avg_launch_ms": ms_c / n_c}


def df_roofline(prof, inst, alg_flops, steps):
    nc, msc = prof.get("contract", (0, 0.0))
    if not nc:
        return None
    ach = inst * steps / (msc / 1e3) / 1e12
    return {"bound": "alu", "kernel": "k_contract_df", "achieved": ach,
            "peak": FP32_INST_PEAK, "unit": "T FP32-inst/s", "frac": ach / FP32_INST_PEAK,
            "peak_source": "derived: 128 FP32 instructions/clk/SM x 152 SMs x 2070 MHz",
            "flops": "modelled FP32 instructions of the double-float inner loops",
            "complex_count_tflops": alg_flops * steps / (msc / 1e3) / 1e12, "launches": nc,
            "avg_launch_ms": msc / nc}


def kernel_table(prof, ms):
    return {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / ms if ms else None}
            for k, v in prof.items()}


# ------------------------------------------------------------------ batched workload

def run_batched(args, R, w, rank, local, clk):
    torch, bb, dev, stream = R.torch, R.bb, R.dev, R.stream
    head = args.form or BATCH_HEAD
    inp = rank_inputs(w, rank)
    n_t = inp.V.shape[0]
    P = len(inp.momenta)
    n_alpha, n_beta, pairs = spin_structure(inp.spins)
    max_nd = max(max(nd) for nd in inp.ndil)
    V = torch.from_numpy(inp.V).to(dev)
    phis = [[torch.from_numpy(inp.phi[k][i]).to(dev) for i in range(3)]
            for k in range(w.n_noise)]
    job_nd = [inp.ndil[k] for k in range(w.n_noise) for _ in range(n_t)]
    blocks_per_step = len(job_nd) * P
    contract_alg = sum(contraction_flops(w.X, nd, P, pairs) for nd in job_nd)
    project_alg = sum(projection_flops(w.X, w.n_ev, nd, n_alpha, n_beta, pairs) for nd in job_nd)
    torch.cuda.synchronize(dev)

    def outputs(sel_t=None):
        ts = n_t if sel_t is None else sel_t
        return [torch.empty((ts, P, *inp.ndil[k]), dtype=torch.complex128, device=dev)
                for k in range(w.n_noise)]

    def batch_step(ctx, outs, ts=None, noises=None):
        ts = range(n_t) if ts is None else ts
        noises = range(w.n_noise) if noises is None else noises
        jobs = [(V[t], phis[k][0][t], phis[k][1][t], phis[k][2][t], outs[k][i])
                for k in noises for i, t in enumerate(ts)]

        def step():
            bb.bblock_compute_batch(ctx, jobs, inp.momenta, inp.spins, inp.coeffs, stream=stream)
        return step

    # ---- tile autotuner: exhaustive search against the learned cost model's top 3
    ctx = R.context(w, head, max_nd)
    tuning = None
    if not args.no_tune and FORMS[head][2]:
        tuning = tune_batched(R, w, inp, V, phis, ctx, head)

    # ---- headline: the whole batch, graph-replayed
    outs = outputs()
    step = batch_step(ctx, outs)
    ms, prof, launches = R.measure(ctx, step, args.steps, args.warmup, sampler=clk)
    value = job_throughput(R.world, blocks_per_step, args.steps, ms / 1e3)
    path = bb.bblock_last_path(ctx)
    ncols = phase_columns(path, w.L, inp.momenta)
    gemm = sum(folded_gemm_flops(w.X, nd, ncols, pairs) for nd in job_nd)
    tkey = f"k_contract_tc/{head}/{path}/{w.name}"
    traffic, trec = load_traffic(tkey)
    roofline = tensor_roofline(head, prof, gemm, contract_alg, args.steps, traffic, trec, path)

    check = None
    if rank == 0 and not args.no_check:
        check = oracle_check(inp, outs, wave_picks(w.n_noise, n_t), FORMS[head][4])

    # ---- the plain FP64 form on the same inputs: one job per dilution size (one time slice
    # of the first noise triple drawn with that size), timed with graph replays, then
    # extrapolated to the batch's job mix
    fp64 = None
    accurate = {}
    if not args.no_fp64_form:
        fp64 = fp64_form_per_size(R, w, inp, V, phis, ms / args.steps, blocks_per_step,
                                  rank == 0 and not args.no_check)
        # the other FP64-accurate forms (parity 1e-12) the same way: double-float on the FP32
        # pipe, and the Ozaki digit-product form on the tensor cores
        for name in ("df64", "ozaki"):
            r = fp64_form_per_size(R, w, inp, V, phis, ms / args.steps, blocks_per_step,
                                   rank == 0 and not args.no_check, form=name)
            r["speedup_vs_fp64_form"] = fp64["extrapolated_ms_per_step"] / r["extrapolated_ms_per_step"]
            accurate[name] = r
        if accurate:
            accurate["ozaki"]["speedup_vs_df64_form"] = (
                accurate["df64"]["extrapolated_ms_per_step"]
                / accurate["ozaki"]["extrapolated_ms_per_step"])

    # ---- the other mixed forms on a subset of the batch (the first 8 time slices of every
    # noise triple: 48 jobs), default tiles, graph-replayed; the headline form is timed on
    # the same subset for comparison
    forms = {}
    if not args.no_forms:
        sub_t = list(range(min(8, n_t)))
        sub_nd = [inp.ndil[k] for k in range(w.n_noise) for _ in sub_t]
        sub_alg = sum(contraction_flops(w.X, nd, P, pairs) for nd in sub_nd)
        for name in dict.fromkeys([head, "bf16x6", "fp16x3", "tf32x3", "bf16x3"]):
            c2 = R.context(w, name, max_nd)
            o2 = outputs(len(sub_t))
            t_ms, pr, nl = R.measure(c2, batch_step(c2, o2, ts=sub_t), 2, 3)
            blocks = len(sub_nd) * P
            pth = bb.bblock_last_path(c2)
            sub_gemm = sum(folded_gemm_flops(w.X, nd, phase_columns(pth, w.L, inp.momenta), pairs)
                           for nd in sub_nd)
            ent = {"blocks_per_s": job_throughput(R.world, blocks, 2, t_ms / 1e3),
                   "ms_per_step": t_ms / 2, "gpu_launches": nl,
                   "tensor_roofline": tensor_roofline(name, pr, sub_gemm, sub_alg, 2, None, None,
                                                      pth),
                   "kernels": kernel_table(pr, t_ms)}
            if rank == 0 and not args.no_check:
                ent["oracle_check"] = oracle_check(
                    inp, [o.cpu() for o in o2], [(k, sub_t[-1]) for k in range(w.n_noise)],
                    FORMS[name][4])
            forms[name] = ent
            bb.bblock_destroy(c2)
            del o2
        forms["subset"] = (f"time slices 0..{len(sub_t) - 1} of all {w.n_noise} noise triples: "
                           f"{len(sub_nd)} jobs, {len(sub_nd) * P} blocks per step; default "
                           f"tiles; 3 warm-up + 2 timed graph-replayed steps")

    # ---- end to end through the public API: every step copies the inputs from pinned host
    # memory, computes the batch and copies the blocks back
    e2e = None
    if not args.no_e2e:
        e2e = e2e_batched(R, w, inp, ctx, n_t, blocks_per_step, args, outs, head)

    line_extra = {
        "roofline": roofline,
        "kernels": kernel_table(prof, ms),
        "oracle_check": check,
        "fp64_form": fp64,
        "speedup_vs_fp64_form": (fp64["extrapolated_ms_per_step"] / (ms / args.steps)
                                 if fp64 else None),
        "fp64_accurate_forms": accurate or None,
        "tuning": tuning,
        "forms": forms,
        "e2e": e2e,
        "algorithmic_tflops": (contract_alg + project_alg) * args.steps / (ms / 1e3) / 1e12,
    }
    config = {"workload": w.name, "L": w.L, "X": w.X, "n_ev": w.n_ev,
              "ndil": [nd[0] for nd in inp.ndil], "n_t": n_t, "n_noise": w.n_noise,
              "n_mom": P, "n_spin": len(inp.spins), "spin_pairs": pairs, "form": head,
              "jobs_per_step_per_gpu": len(job_nd), "blocks_per_step_per_gpu": blocks_per_step,
              "tiles": {"nc": bb.bblock_get_option(ctx, "tc_nc"),
                        "chunk": bb.bblock_get_option(ctx, "tc_chunk"),
                        "source": "cost-model top 3 timed" if tuning else "heuristic"},
              "timed_steps": "bblock_compute_batch replayed from a CUDA graph, CUDA events "
                             "around every launch (captured as graph event nodes)",
              "l2": "inputs larger than L2 (V %.1f GB on the device; fields %.0f GB per step)" % (
                  inp.V.nbytes / 1e9,
                  sum(3 * w.X * 8 * (n_alpha * nd[0] + n_beta * nd[1] + pairs * nd[2])
                      for nd in job_nd) / 1e9),
              "parallelism": f"{R.world} independent GPU(s), no collective"}
    bb.bblock_destroy(ctx)
    del outs
    torch.cuda.empty_cache()
    return head, value, ms, launches, config, line_extra


def tune_batched(R, w, inp, V, phis, ctx, head):
    """The tile autotuner on two time slices of the largest-dilution noise triple: every
    candidate timed (exhaustive), against the cost model's top 3 timed. The model is trained
    (on the GPU, by the library's own kernels) on exhaustive timings of the workload's other
    dilution sizes and of the L = 24 workload. The context keeps the model's choice."""
    torch, bb, dev, stream = R.torch, R.bb, R.dev, R.stream
    P = len(inp.momenta)
    n_t = inp.V.shape[0]
    nt_s = min(2, n_t)
    order = sorted(range(w.n_noise), key=lambda q: inp.ndil[q][0])
    target = order[-1]
    train_feat, train_ms = [], []

    def tune_on(c, Vs, ph, mom, spins, coeffs, nd, model=None):
        Bs = torch.empty((Vs.shape[0], len(mom), *nd), dtype=torch.complex128, device=dev)
        bb.bblock_compute(c, Vs, *ph, mom, spins, coeffs, B_out=Bs, stream=stream)  # warm
        t0 = time.perf_counter()
        rep = bb.bblock_autotune(c, Vs, *ph, mom, spins, coeffs, Bs, stream=stream,
                                 model=model, top_k=3, repeats=2)
        return rep, time.perf_counter() - t0

    # training data: the other dilution sizes of this workload
    seen = set()
    for k in order[:-1]:
        if inp.ndil[k][0] in seen or inp.ndil[k][0] == inp.ndil[target][0]:
            continue
        seen.add(inp.ndil[k][0])
        c = R.context(w, head, max(inp.ndil[k]))
        rep, _ = tune_on(c, V[:nt_s], [p[:nt_s] for p in phis[k]], inp.momenta, inp.spins,
                         inp.coeffs, inp.ndil[k])
        train_feat += [r["features"] for r in rep]
        train_ms += [r["ms"] for r in rep]
        bb.bblock_destroy(c)
    # and the L = 24 workload (other lattice, dilution, momenta and spin operator)
    w2 = workloads.WORKLOADS[SECONDARY]
    inp2 = workloads.generate(w2, n_t=2)
    V2 = torch.from_numpy(inp2.V).to(dev)
    ph2 = [torch.from_numpy(inp2.phi[0][i]).to(dev) for i in range(3)]
    c = R.context(w2, head, max(inp2.ndil[0]))
    rep, _ = tune_on(c, V2, ph2, inp2.momenta, inp2.spins, inp2.coeffs, inp2.ndil[0])
    train_feat += [r["features"] for r in rep]
    train_ms += [r["ms"] for r in rep]
    bb.bblock_destroy(c)
    del V2, ph2

    t0 = time.perf_counter()
    cm = bb.CostModel(bb.bblock.TUNE_FEATURES, 32, seed=7)
    loss = cm.train(np.asarray(train_feat, np.float32), np.log(np.asarray(train_ms)),
                    epochs=3000, lr=3e-3)
    t_train = time.perf_counter() - t0

    ph_t = [p[:nt_s] for p in phis[target]]
    nd_t = inp.ndil[target]
    c_ex = R.context(w, head, max(nd_t))
    rep_ex, t_ex = tune_on(c_ex, V[:nt_s], ph_t, inp.momenta, inp.spins, inp.coeffs, nd_t)
    bb.bblock_destroy(c_ex)
    rep_m, t_m = tune_on(ctx, V[:nt_s], ph_t, inp.momenta, inp.spins, inp.coeffs, nd_t,
                         model=cm)
    bb.bblock_set_option(ctx, "slabs", 0)   # slab count automatic for the whole batch
    best_ex = min(rep_ex, key=lambda r: r["ms"])
    timed = [r for r in rep_m if r["ms"] > 0]
    best_m = min(timed, key=lambda r: r["ms"])
    # the library's default tile (every tile option automatic), timed the autotuner's way:
    # plain launches, median of the timed calls after one warm-up call
    c_def = R.context(w, head, max(nd_t))
    bb.bblock_set_option(c_def, "graphs", 0)
    Bd = torch.empty((nt_s, P, *nd_t), dtype=torch.complex128, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ts = []
    for k in range(4):
        ev[0].record(stream)
        bb.bblock_compute(c_def, V[:nt_s], *ph_t, inp.momenta, inp.spins, inp.coeffs, B_out=Bd,
                          stream=stream)
        ev[1].record(stream)
        bb.bblock_status(c_def)
        if k:
            ts.append(ev[0].elapsed_time(ev[1]))
    bb.bblock_destroy(c_def)
    default_ms = statistics.median(ts)
    return {
        "tuned_on": f"time slices 0..{nt_s - 1} of noise triple {target} (N_dil {nd_t[0]})",
        "training": {"samples": len(train_ms), "loss": loss, "seconds": t_train,
                     "from": f"exhaustive timings of N_dil {sorted(seen)} of this workload "
                             f"and of {SECONDARY}"},
        "exhaustive": {"candidates_timed": len(rep_ex), "best_ms": best_ex["ms"],
                       "best": {k: best_ex[k] for k in ("nc", "chunk", "slabs")},
                       "wall_s": t_ex},
        "model_top3": {"candidates_timed": len(timed), "best_ms": best_m["ms"],
                       "best": {k: best_m[k] for k in ("nc", "chunk", "slabs")},
                       "wall_s": t_m, "vs_exhaustive_best": best_m["ms"] / best_ex["ms"]},
        "default_tile_ms": default_ms,
        "model_vs_default": best_m["ms"] / default_ms,
        "exhaustive_table": [[r["nc"], r["chunk"], r["slabs"], round(r["ms"], 3)] for r in rep_ex],
    }


def fp64_form_per_size(R, w, inp, V, phis, head_ms_per_step, blocks_per_step, check,
                       form="fp64"):
    """An FP64-accurate form (the plain FP64 form, double-float or the Ozaki tensor-core
    form) on one job per dilution size of the batch (graph-replayed, 3 warm-up + 2 timed
    calls each); the batch's time in that form is the sum over its jobs of the time of a
    job of that size."""
    torch, bb, dev = R.torch, R.bb, R.dev
    n_t = inp.V.shape[0]
    P = len(inp.momenta)
    per_size = {}
    outs_chk, picks = {}, []
    for k in range(w.n_noise):
        nd = inp.ndil[k]
        if nd[0] in per_size:
            continue
        c = R.context(w, form, max(nd))
        B = torch.empty((1, P, *nd), dtype=torch.complex128, device=dev)
        jobs = [(V[0], phis[k][0][0], phis[k][1][0], phis[k][2][0], B[0])]

        def step():
            bb.bblock_compute_batch(c, jobs, inp.momenta, inp.spins, inp.coeffs,
                                    stream=R.stream)
        t_ms, pr, nl = R.measure(c, step, 2, 3)
        n_alpha, n_beta, pairs = spin_structure(inp.spins)
        alg = contraction_flops(w.X, nd, P, pairs)
        if form == "fp64":
            roof = fp64_roofline(pr, alg, 2, None, None)
        elif form == "df64":
            roof = df_roofline(pr, contraction_df_inst(w.X, nd, P, pairs), alg, 2)
        else:
            roof = tensor_roofline(form, pr, folded_gemm_flops(w.X, nd, P, pairs), alg, 2,
                                   None, None, bb.bblock_last_path(c))
        per_size[nd[0]] = {"noise": k, "ms_per_job": t_ms / 2, "blocks_per_s": 2 * P / (t_ms / 1e3),
                           "roofline": roof, "kernels": kernel_table(pr, t_ms)}
        if form == "ozaki":
            per_size[nd[0]]["cluster"] = bb.bblock_get_option(c, "tc_cluster")
        if check:
            full = [None] * w.n_noise
            full[k] = B.cpu()
            outs_chk[k] = full
            picks.append(k)
        bb.bblock_destroy(c)
    counts = {}
    for k in range(w.n_noise):
        counts[inp.ndil[k][0]] = counts.get(inp.ndil[k][0], 0) + n_t
    ext_ms = sum(cnt * per_size[d]["ms_per_job"] for d, cnt in counts.items())
    res = {"per_dilution_size": {str(d): v for d, v in per_size.items()},
           "jobs_per_size_in_batch": {str(d): c for d, c in counts.items()},
           "extrapolated_ms_per_step": ext_ms,
           "extrapolated_blocks_per_s": R.world * blocks_per_step / (ext_ms / 1e3),
           "method": "one job (time slice 0 of the first noise triple of each dilution size) "
                     "per size, 3 warm-up + 2 timed graph-replayed calls; batch time = sum over "
                     "the batch's jobs of the measured time of a job of that size"}
    if check:
        errs = []
        for k in picks:
            r = oracle_check(inp, outs_chk[k], [(k, 0)], FORMS[form][4])
            errs.append(r)
        res["oracle_check"] = {"blocks_checked": sum(r["blocks_checked"] for r in errs),
                               "max": max(r["max"] for r in errs),
                               "median": statistics.median([r["median"] for r in errs]),
                               "tolerance": FORMS[form][4],
                               "pass": all(r["pass"] for r in errs)}
    return res


def e2e_batched(R, w, inp, ctx, n_t, blocks_per_step, args, outs, head):
    torch, bb, dev, stream = R.torch, R.bb, R.dev, R.stream
    hV = torch.from_numpy(inp.V).pin_memory()
    hphi = [[torch.from_numpy(inp.phi[k][i]).pin_memory() for i in range(3)]
            for k in range(w.n_noise)]
    hB = [torch.empty(tuple(o.shape), dtype=torch.complex128).pin_memory() for o in outs]
    dV = torch.empty(tuple(hV.shape), dtype=torch.complex128, device=dev)
    dphi = [[torch.empty(tuple(p.shape), dtype=torch.complex128, device=dev) for p in ph]
            for ph in hphi]
    douts = [torch.empty(tuple(o.shape), dtype=torch.complex128, device=dev) for o in outs]
    jobs = [(dV[t], dphi[k][0][t], dphi[k][1][t], dphi[k][2][t], douts[k][t])
            for k in range(w.n_noise) for t in range(n_t)]

    def e2e_step():
        with torch.cuda.stream(stream):
            dV.copy_(hV, non_blocking=True)
            for k in range(w.n_noise):
                for i in range(3):
                    dphi[k][i].copy_(hphi[k][i], non_blocking=True)
        bb.bblock_compute_batch(ctx, jobs, inp.momenta, inp.spins, inp.coeffs, stream=stream)
        with torch.cuda.stream(stream):
            for k in range(w.n_noise):
                hB[k].copy_(douts[k], non_blocking=True)
        stream.synchronize()

    # one plain warm-up call; the first timed call captures the graph, the others replay it
    e2e_steps = min(args.steps, 3)
    e2e_step()
    R.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    dt = max_over_ranks(time.perf_counter() - t0, R.world, dev)
    # same tiles, same job list: the host-copy path reproduces the device path's blocks
    for h, o in zip(hB, outs):
        ref = o.cpu().numpy()
        err = np.linalg.norm(h.numpy() - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= 1e-12, f"host-copy and resident-input steps differ by {err:.2e}"
    h2d = hV.numel() * 16 + sum(p.numel() * 16 for ph in hphi for p in ph)
    res = {"value": job_throughput(R.world, blocks_per_step, e2e_steps, dt), "unit": UNIT,
           "steps": e2e_steps,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": sum(h.numel() * 16 for h in hB),
           "path": "pinned host -> device copies, bblock_compute_batch (graph replay), device "
                   "-> pinned host copies, stream synchronised; wall clock per step"}
    del dV, dphi, douts
    return res


# ------------------------------------------------------------------ single-noise workloads

def run_single(args, R, w, rank, head, clk, steps, warmup, extras=True):
    torch, bb, dev, stream = R.torch, R.bb, R.dev, R.stream
    inp = rank_inputs(w, rank, n_t=args.n_t if extras else None)
    n_t = inp.V.shape[0]
    P = len(inp.momenta)
    n_alpha, n_beta, pairs = spin_structure(inp.spins)
    nd = inp.ndil[0]
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    blocks_per_step = n_t * P
    contract_alg = n_t * contraction_flops(w.X, nd, P, pairs)
    project_alg = n_t * projection_flops(w.X, w.n_ev, nd, n_alpha, n_beta, pairs)
    full_shape = args.n_t is None or not extras

    def measure(form, sampler=None, k=steps, wu=warmup):
        c = R.context(w, form, max(nd))
        B = torch.empty((n_t, P, *nd), dtype=torch.complex128, device=dev)

        def step():
            bb.bblock_compute(c, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B,
                              stream=stream)
        t_ms, prof, nl = R.measure(c, step, k, wu, sampler=sampler)
        return c, B, t_ms, prof, nl

    ctx, B, ms, prof, launches = measure(head, clk)
    value = job_throughput(R.world, blocks_per_step, steps, ms / 1e3)

    def gemm_of(c):
        return n_t * folded_gemm_flops(w.X, nd, phase_columns(bb.bblock_last_path(c), w.L,
                                                              inp.momenta), pairs)
    if head == "fp64":
        traffic, trec = load_traffic(f"k_contract_fp64/fp64/{w.name}") if full_shape else (None, None)
        roofline = fp64_roofline(prof, contract_alg, steps, traffic, trec)
    elif head == "df64":
        roofline = df_roofline(prof, n_t * contraction_df_inst(w.X, nd, P, pairs), contract_alg,
                               steps)
    else:
        path = bb.bblock_last_path(ctx)
        traffic, trec = (load_traffic(f"k_contract_tc/{head}/{path}/{w.name}") if full_shape
                         else (None, None))
        roofline = tensor_roofline(head, prof, gemm_of(ctx), contract_alg, steps, traffic, trec,
                                   path)

    forms = {}
    if extras and not args.no_forms:
        B0 = B.cpu().numpy()
        nrm = np.linalg.norm(B0)
        for name in FORMS:
            if name == head:
                continue
            c2, B2, t_ms, pr, nl = measure(name)
            err = float(np.linalg.norm(B2.cpu().numpy() - B0) / nrm)
            ent = {"blocks_per_s": job_throughput(R.world, blocks_per_step, steps, t_ms / 1e3),
                   "ms_per_step": t_ms / steps, "gpu_launches": nl,
                   f"rel_frobenius_err_vs_{head}_form": err,
                   f"speedup_vs_{head}_form": ms / t_ms,
                   "kernels": kernel_table(pr, t_ms)}
            if name == "df64":
                ent["alu_roofline"] = df_roofline(pr, n_t * contraction_df_inst(w.X, nd, P, pairs),
                                                  contract_alg, steps)
            elif name == "fp64":
                ent["alu_roofline"] = fp64_roofline(pr, contract_alg, steps, None, None)
            else:
                ent["tensor_roofline"] = tensor_roofline(name, pr, gemm_of(c2), contract_alg, steps,
                                                         None, None, bb.bblock_last_path(c2))
            forms[name] = ent
            bb.bblock_destroy(c2)

    check = None
    if rank == 0 and not args.no_check:
        check = oracle_check(inp, [B.cpu()], [(0, t) for t in sorted({0, n_t - 1})],
                             FORMS[head][4])

    triplet = None
    if extras and not args.no_triplet and max(nd) <= w.n_ev <= 256:
        triplet = mode_triplet_timing(R, w, inp, V, phis, B, ms / steps, forms, steps, warmup)

    e2e = None
    if extras and not args.no_e2e:
        hV = torch.from_numpy(inp.V).pin_memory()
        hphi = [torch.from_numpy(inp.phi[0][i]).pin_memory() for i in range(3)]
        hB = torch.empty(tuple(B.shape), dtype=torch.complex128).pin_memory()

        def e2e_step():
            bb.bblock_compute_host(ctx, hV, *hphi, inp.momenta, inp.spins, inp.coeffs, hB, stream)
        for _ in range(max(1, warmup // 2)):
            e2e_step()
        R.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0, R.world, dev)
        # the host path computes in chunks of time slices, whose site slabs may differ from
        # the device call's: the two agree to the form's rounding, not bit for bit
        tol = 1e-12 if head in ("fp64", "df64", "ozaki") else 1e-5
        ref = B.cpu().numpy()
        err = np.linalg.norm(hB.numpy() - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= tol, f"host and device paths differ by {err:.2e}"
        h2d = hV.numel() * 16 + sum(p.numel() * 16 for p in hphi)
        e2e = {"value": job_throughput(R.world, blocks_per_step, steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": hB.numel() * 16,
               "path": "bblock_compute_host (pinned host buffers, copies inside, chunked)"}

    line_extra = {"roofline": roofline, "kernels": kernel_table(prof, ms), "oracle_check": check,
                  "forms": forms, "mode_triplet": triplet, "e2e": e2e,
                  "algorithmic_tflops": (contract_alg + project_alg) * steps / (ms / 1e3) / 1e12}
    config = {"workload": w.name, "L": w.L, "X": w.X, "n_ev": w.n_ev, "ndil": nd[0],
              "n_t": n_t, "n_noise": 1, "n_mom": P, "n_spin": len(inp.spins),
              "spin_pairs": pairs, "form": head, "blocks_per_step_per_gpu": blocks_per_step,
              "timed_steps": "bblock_compute replayed from a CUDA graph, CUDA events around "
                             "every launch (captured as graph event nodes)",
              "l2": "inputs larger than L2 (V %.0f MB)" % (inp.V.nbytes / 1e6),
              "parallelism": f"{R.world} independent GPU(s), no collective"}
    bb.bblock_destroy(ctx)
    return value, ms, launches, config, line_extra


def mode_triplet_timing(R, w, inp, V, phis, B, direct_ms, forms, steps, warmup):
    """The mode-triplet ordering (Sec. 2, Eq. 4): T per time slice (noise-independent), then
    blocks from T by three FP64 mode products; the crossover is the number of noise triples
    per time slice above which T + n * (blocks from T) beats n * (direct blocks)."""
    torch, bb, dev, stream = R.torch, R.bb, R.dev, R.stream
    n_t = inp.V.shape[0]
    P = len(inp.momenta)
    triplet = {}
    Tbuf = torch.empty((n_t, P, w.n_ev, w.n_ev, w.n_ev), dtype=torch.complex128, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name in ("fp64", "df64"):
        c3 = bb.bblock_create(w.L, w.n_ev, w.n_ev, FORMS[name][0], device=R.local)
        bb.bblock_mode_triplet(c3, V, inp.momenta, T_out=Tbuf, stream=stream)    # warm-up
        bb.bblock_status(c3)
        ev0.record(stream)
        bb.bblock_mode_triplet(c3, V, inp.momenta, T_out=Tbuf, stream=stream)
        ev1.record(stream)
        bb.bblock_status(c3)
        triplet[f"T_ms_per_time_slice_{name}"] = ev0.elapsed_time(ev1) / n_t
        if name == "df64":
            Bt = torch.empty_like(B)
            for _ in range(max(1, warmup)):
                bb.bblock_from_triplet(c3, Tbuf, *phis, inp.spins, inp.coeffs, B_out=Bt,
                                       stream=stream)
            bb.bblock_status(c3)
            ev0.record(stream)
            for _ in range(steps):
                bb.bblock_from_triplet(c3, Tbuf, *phis, inp.spins, inp.coeffs, B_out=Bt,
                                       stream=stream)
            ev1.record(stream)
            bb.bblock_status(c3)
            triplet["blocks_from_T_ms_per_time_slice"] = ev0.elapsed_time(ev1) / steps / n_t
            triplet["rel_frobenius_err_vs_headline"] = float(
                np.linalg.norm(Bt.cpu().numpy() - B.cpu().numpy()) /
                np.linalg.norm(B.cpu().numpy()))
        bb.bblock_destroy(c3)
    direct = {"fp64": direct_ms / n_t}
    if "df64" in forms:
        direct["df64"] = forms["df64"]["ms_per_step"] / n_t
    triplet["direct_ms_per_time_slice"] = direct
    ft = triplet["blocks_from_T_ms_per_time_slice"]
    triplet["crossover_noise_triples"] = {
        k: (triplet[f"T_ms_per_time_slice_{k}"] / (v - ft) if v > ft else None)
        for k, v in direct.items()}
    return triplet


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2211_16278_gb300 as bb

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    # a created stream: repeated calls are then replayed from a CUDA graph by the library
    R = Runner(torch, bb, dev, local, world, barrier, torch.cuda.Stream(dev))
    # the FP64 pipe's measured peaks: DFMA (the FP64 form's roofline) and the FP64 MMA
    probe = bb.bblock_probe_fp64(local, stream=R.stream)
    if probe["dfma_tflops"] > 0:
        FP64_PEAK["tflops"] = probe["dfma_tflops"]
        FP64_PEAK["source"] = ("measured in this run: DFMA loop over every SM "
                               "(bblock_probe_fp64), best of 3")
    w = workloads.WORKLOADS[args.workload]
    if args.n_t is not None:
        w = dataclasses.replace(w, n_t=args.n_t)
    clk = ClockSampler(local)
    if w.n_noise > 1:
        head, value, ms, launches, config, extra = run_batched(args, R, w, rank, local, clk)
        dtype = {"tf32x3": "tf32", "fp64": "f64", "df64": "f32 pairs",
                 "fp16x3": "fp16"}.get(head, "bf16")
    else:
        head = args.form or "fp64"
        value, ms, launches, config, extra = run_single(args, R, w, rank, head, clk,
                                                        args.steps, args.warmup)
        dtype = {"tf32x3": "tf32", "fp64": "f64", "df64": "f32 pairs",
                 "fp16x3": "fp16"}.get(head, "bf16")

    secondary = None
    if w.n_noise > 1 and not args.no_secondary:
        w2 = workloads.WORKLOADS[SECONDARY]
        secondary = {}
        for form in ("fp64", head):
            a2 = parse_args(["--no-forms", "--no-e2e", "--no-triplet"] +
                            (["--no-check"] if args.no_check else []))
            v2, ms2, nl2, cfg2, ex2 = run_single(a2, R, w2, rank, form, None, 3, 3, extras=False)
            secondary[form] = {"workload": w2.name, "blocks_per_s": v2, "ms_per_step": ms2 / 3,
                               "gpu_launches": nl2, "roofline": ex2["roofline"],
                               "oracle_check": ex2["oracle_check"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic (seeded, workloads.py)",
            "config": config,
            "gpu_launches": launches,
        }
        line.update(extra)
        line["fp64_probe"] = dict(probe, note="FP64 form runs on DFMA: the measured DFMA rate "
                                  "is its roofline peak; the FP64 MMA (mma.sync m8n8k4) rate "
                                  "is the alternative it was chosen over")
        line["cpu_baseline"] = cpu
        line["clocks"] = clk.summary()
        line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


SWEEP_N_EV = 96
SWEEP_POINTS = [(16, 32), (24, 32), (32, 32), (48, 32), (32, 16), (32, 48), (32, 64)]


def loglog_slope(xs, ys):
    """Least-squares slope of log y against log x."""
    lx = [math.log(x) for x in xs]
    ly = [math.log(y) for y in ys]
    mx, my = statistics.fmean(lx), statistics.fmean(ly)
    return sum((a - mx) * (b - my) for a, b in zip(lx, ly)) / sum((a - mx) ** 2 for a in lx)


def run_size_sweep(args):
    """Problem-size scaling of the contraction (the paper's observation, Sec. 4, that its
    time grows as L^3 and as N_dil^3): one time slice of the 9-momentum, 4-triple operator of
    the batched workload, N_ev = 96, for L in {16, 24, 32, 48} at N_dil = 32 and for N_dil in
    {16, 32, 48, 64} at L = 32, in the FP16 form and the FP64 form. Contraction time per call
    from CUDA events (3 warm-up, 3 timed graph replays); exponents fitted on log-log."""
    import torch

    import paper_2211_16278_gb300 as bb

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    R = Runner(torch, bb, dev, 0, 1, lambda: None, torch.cuda.Stream(dev))
    mom = workloads.MOM_C4
    spins, coeffs = workloads.SPIN_C3
    points = []
    for i, (L, D) in enumerate(SWEEP_POINTS):
        inp = workloads.custom(L, SWEEP_N_EV, (D, D, D), 1, mom, spins, coeffs, seed=9000 + i)
        V = torch.from_numpy(inp.V).to(dev)
        phis = [torch.from_numpy(inp.phi[0][k]).to(dev) for k in range(3)]
        for form in ("fp16x3", "fp64"):
            precision, products = FORMS[form][:2]
            ctx = bb.bblock_create(L, SWEEP_N_EV, D, precision, bf16_products=products)
            B = torch.empty((1, len(mom), D, D, D), dtype=torch.complex128, device=dev)

            def step():
                bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B,
                                  stream=R.stream)
            t_ms, prof, _ = R.measure(ctx, step, 3, 3)
            points.append({"L": L, "n_dil": D, "form": form, "path": bb.bblock_last_path(ctx),
                           "contract_ms": prof["contract"][1] / 3, "call_ms": t_ms / 3})
            bb.bblock_destroy(ctx)
    fits = {}
    for form in ("fp16x3", "fp64"):
        lp = [p for p in points if p["form"] == form and p["n_dil"] == 32]
        dp = [p for p in points if p["form"] == form and p["L"] == 32]
        fits[form] = {
            "L_exponent": loglog_slope([p["L"] for p in lp], [p["contract_ms"] for p in lp]),
            "n_dil_exponent": loglog_slope([p["n_dil"] for p in dp], [p["contract_ms"] for p in dp]),
        }
    print(json.dumps({"size_sweep": {"n_ev": SWEEP_N_EV, "momenta": len(mom),
                                     "spin_triples": len(spins), "time_slices": 1,
                                     "points": points, "fits": fits,
                                     "expected": "exponent 3 in L (sites) and in N_dil"}}),
          flush=True)
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.size_sweep:
        return run_size_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
