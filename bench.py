#!/usr/bin/env python
"""Baryon-block throughput on GB300 (blocks/s), by default for the L=24, N_ev=96, N_dil=32
workload in the FP64 form.

One step = the whole hot path (phase table from cache, projection of the three quark
lines for every spin used, fused diquark + contraction, slab reduction) over every block
of the workload; for the default workload 8 time slices x 3 momenta x one 3-triple baryon
operator, i.e. 24 blocks B[t][p][d1][d2][d3]. Inputs are seeded synthetic draws
(``workloads.py``) resident on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload NAME] [--form fp64|bf16x6|bf16x9|tf32x3|bf16x3]

``--workload`` selects another named workload (the batched one, with six noise triples of
uneven dilution size, runs as one batched call per step and defaults to the bf16x6 form).
Prints one JSON line (rank 0). Under torchrun every rank computes its own independent
time slices (weak scaling, no data-path collective); the timed region is bracketed by a
barrier and the maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import csv
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

WORKLOAD = "l24_nev96_ndil32"
METRIC = "baryon blocks/s"
UNIT = "blocks/s"
# Peak of the FP64 pipe: the nominal 1.25 TFLOP/s of GB300 is 4 FP64 flop/clk/SM
# (2 DFMA) x 152 SMs x the 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 4 * 152 * 2.070e9 / 1e12


def _measured_peaks():
    """Dense BF16 tensor peak measured on the GB300s (cuBLAS burst), if present."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# BF16 from the measured burst figure (fallback 1.9 PFLOP/s); TF32 = BF16 x the nominal
# dense ratio 1.1 / 2.25.
BF16_PEAK_TFLOPS = float(_measured_peaks().get("bf16_tflops", 1900.0))
TF32_PEAK_TFLOPS = BF16_PEAK_TFLOPS * 1.1 / 2.25
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU seconds of one oracle sample")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workload: skip the tile autotuner (heuristic tiles)")
    ap.add_argument("--no-triplet", action="store_true",
                    help="skip the mode-triplet ordering's measurement")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the tensor-core forms (time the FP64 form only)")
    ap.add_argument("--form", choices=["fp64", "df64", "bf16x6", "bf16x9", "tf32x3", "bf16x3"],
                    default=None, help="form of the headline number (default: fp64; bf16x6 "
                    "for the batched workload)")
    ap.add_argument("--n-t", type=int, default=None,
                    help="time slices per step (default: the workload's); for profiling runs")
    return ap.parse_args()


# ------------------------------------------------------------------ algorithmic work

def spin_structure(spins):
    spins = [tuple(int(v) for v in s) for s in np.asarray(spins).reshape(-1, 3)]
    n_alpha = len({s[0] for s in spins})
    n_beta = len({s[1] for s in spins})
    pairs = len({(s[0], s[1]) for s in spins})
    return n_alpha, n_beta, pairs


def contraction_flops(X, nd, P, pairs):
    """Complex-arithmetic flops (cmul 6, complex FMA 8) of the contraction of one
    (time slice, noise triple): diquark 42 per (pair, d1, d2, x); colour singlet with the
    spin-pair sum inside, 8 * 3 * pairs per (d1, d2, d3, x); momentum projection 8 P per
    (d1, d2, d3, x)."""
    d1, d2, d3 = nd
    return 42.0 * pairs * d1 * d2 * X + (24.0 * pairs + 8.0 * P) * d1 * d2 * d3 * X


def projection_flops(X, n_ev, nd, n_alpha, n_beta, pairs):
    """Eq. (2) as complex GEMMs: 8 * 3X * n_ev per output column."""
    return 8.0 * 3 * X * n_ev * (n_alpha * nd[0] + n_beta * nd[1] + pairs * nd[2])


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
        sm, smax, reasons = [], [], set()
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
            except (KeyError, ValueError, IndexError):
                continue
            for k, v in names.items():
                if d.get(k, "").lower() == "active":
                    reasons.add(v)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle sample

def oracle_sample(inp, target_s: float):
    """Time the CPU FP64 oracle on a bounded sample of the workload.

    The oracle's OpenMP loop runs over d1, so the sample grows in steps of one d1 value per
    thread: first over d2 values, then over further d1 blocks, then over time slices,
    until it is about ``target_s`` seconds of CPU work. All momenta and all d3 are always
    included. Returns (blocks/s, threads, text)."""
    import oracle
    w = inp.workload
    nd = inp.ndil[0]
    P = len(inp.momenta)
    n_t = inp.V.shape[0]
    n1 = max(1, min(nd[0], oracle.num_threads()))
    all3 = list(range(nd[2]))

    def run(t, d1s, d2s):
        oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
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
    text = (f"{n_ts} time slice(s), {P} momenta, d1 in [0,{len(d1s)}) of {nd[0]}, d2 in "
            f"[0,{k2}) of {nd[1]}, all {nd[2]} d3 = {blocks:.4f} blocks in {tk:.2f} s on "
            f"{n1} threads")
    return blocks / tk, n1, text


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workloads.WORKLOADS[args.workload]
    inp = workloads.generate(w, n_t=4)
    oracle.build()
    vals, sample = [], ""
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        v, cores, sample = oracle_sample(inp, per_step)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded, workloads.py)",
        "config": {"workload": w.name, "L": w.L, "n_ev": w.n_ev, "ndil": w.ndil, "n_t": w.n_t,
                   "n_mom": len(w.momenta), "n_spin": len(w.spins), "form": "fp64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def load_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        from paper_2211_16278_gb300 import build as cb
        rec = json.load(open(path)).get(kernel)
        if rec and rec.get("source_sha256") == cb.source_digest(rec.get("source")):
            return rec.get("dram_bytes_per_launch_full_workload")
    except Exception:
        return None
    return None


def rank_inputs(w, rank: int):
    """Inputs of one rank: every rank draws its own time slices (its own seed), so the
    ranks share no work and exchange no data."""
    return workloads.generate(w, seed=w.seed + rank)


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


# Peak of the FP32 pipe (the double-float form's bound): 128 FP32 instructions/clk/SM x 152
# SMs x 2070 MHz, in tera-instructions per second.
FP32_INST_PEAK = 128 * 152 * 2.070e9 / 1e12


def contraction_df_inst(X, nd, P, pairs):
    """FP32 instructions of the double-float contraction's inner loops per (time slice,
    noise triple): 12 per double-float FMA (exact product error, TwoSum, lazy error sum),
    three per (pair, colour) in the singlet, four per momentum, 16 for the singlet's real and
    imaginary parts; per (d1, d2, d3, x)."""
    d1, d2, d3 = nd
    return (108.0 * pairs + 16.0 + 48.0 * P) * d1 * d2 * d3 * X


FORMS = {  # name: (precision, bf16 products, MMA piece products, tensor peak TFLOP/s)
    "fp64": ("fp64", 6, 0, None), "df64": ("df64", 6, 0, None),
    "bf16x6": ("bf16", 6, 6, BF16_PEAK_TFLOPS), "bf16x9": ("bf16", 9, 9, BF16_PEAK_TFLOPS),
    "tf32x3": ("tf32x3", 6, 3, TF32_PEAK_TFLOPS), "bf16x3": ("bf16", 3, 3, BF16_PEAK_TFLOPS),
}


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

    w = workloads.WORKLOADS[args.workload]
    if args.n_t is not None:
        import dataclasses
        w = dataclasses.replace(w, n_t=args.n_t)
    batched = w.n_noise > 1
    # the committed DRAM-traffic captures are of the default workload at full size
    default_shape = w.name == WORKLOAD and args.n_t is None
    head = args.form or ("bf16x6" if batched else "fp64")
    inp = rank_inputs(w, rank)
    P = len(inp.momenta)
    n_alpha, n_beta, pairs = spin_structure(inp.spins)
    max_nd = max(max(nd) for nd in inp.ndil)
    V = torch.from_numpy(inp.V).to(dev)
    phis = [[torch.from_numpy(inp.phi[k][i]).to(dev) for i in range(3)] for k in range(w.n_noise)]
    # jobs: (noise triple, time slice); a single-noise workload is one call over all slices
    job_nd = [inp.ndil[k] for k in range(w.n_noise) for _ in range(w.n_t)]
    # a created stream: repeated calls are then replayed from a CUDA graph by the library
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    blocks_per_step = len(job_nd) * P
    contract_alg = sum(contraction_flops(w.X, nd, P, pairs) for nd in job_nd)
    project_alg = sum(projection_flops(w.X, w.n_ev, nd, n_alpha, n_beta, pairs) for nd in job_nd)
    # useful complex GEMM work of the folded contraction: 8 M N K per job, K = 3 pairs X
    gemm_flops = sum(8.0 * nd[0] * nd[1] * (P * nd[2]) * (3 * pairs * w.X) for nd in job_nd)

    tuned = {}

    def outputs():
        return [torch.empty((w.n_t, P, *inp.ndil[k]), dtype=torch.complex128, device=dev)
                for k in range(w.n_noise)]

    def measure(form, sampler=None):
        """W untimed + K timed steps of one form; CUDA events on the launching stream."""
        precision, products = FORMS[form][:2]
        c = bb.bblock_create(w.L, w.n_ev, max_nd, precision, bf16_products=products,
                             device=local)
        outs = outputs()
        if batched and not args.no_tune:
            # tile shapes from the autotuner, timed on two time slices of the noise triple with
            # the largest dilution; the slab count stays automatic for the whole batch
            k = max(range(w.n_noise), key=lambda q: inp.ndil[q][0])
            nt_s = min(2, w.n_t)
            Bs = torch.empty((nt_s, P, *inp.ndil[k]), dtype=torch.complex128, device=dev)
            rep = bb.bblock_autotune(c, V[:nt_s], *[p[:nt_s] for p in phis[k]], inp.momenta,
                                     inp.spins, inp.coeffs, Bs, stream=stream, repeats=2)
            bb.bblock_set_option(c, "slabs", 0)
            tuned[form] = {"nc": bb.bblock_get_option(c, "tc_nc"),
                           "chunk": bb.bblock_get_option(c, "tc_chunk"),
                           "candidates_timed": sum(1 for r in rep if r["ms"] > 0)}
            del Bs
        if batched:
            jobs = [(V[t], phis[k][0][t], phis[k][1][t], phis[k][2][t], outs[k][t])
                    for k in range(w.n_noise) for t in range(w.n_t)]

            def step():
                bb.bblock_compute_batch(c, jobs, inp.momenta, inp.spins, inp.coeffs,
                                        stream=stream)
        else:
            def step():
                bb.bblock_compute(c, V, *phis[0], inp.momenta, inp.spins, inp.coeffs,
                                  B_out=outs[0], stream=stream)

        for _ in range(args.warmup):
            step()
        bb.bblock_status(c)
        torch.cuda.synchronize(dev)
        barrier()
        bb.bblock_profile_enable(c, True)
        bb.bblock_profile_read(c)  # reset
        n_launch = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if sampler is not None:
            sampler.__enter__()
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
            n_launch += bb.bblock_last_launch_count(c)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        if sampler is not None:
            sampler.__exit__(None, None, None)
        bb.bblock_status(c)
        t_ms = e0.elapsed_time(e1)
        prof = bb.bblock_profile_read(c)
        bb.bblock_profile_enable(c, False)
        t_ms = max_over_ranks(t_ms, world, dev)
        return c, outs, t_ms, prof, n_launch

    def tensor_roofline(form, prof):
        nprod, peak = FORMS[form][2:]
        # DRAM bytes per launch were captured for the BF16x6 variant on this workload
        traffic = (load_traffic("k_contract_tc")
                   if form == "bf16x6" and default_shape else None)
        nc, msc = prof.get("contract", (0, 0.0))
        # executed MMA flops of the timed steps / the contraction launches' summed time
        execd = gemm_flops * nprod * args.steps / (msc / 1e3) / 1e12 if nc else None
        return {"bound": "tensor", "kernel": "k_contract_tc", "achieved": execd, "peak": peak,
                "unit": "TFLOP/s", "frac": execd / peak if execd else None, "traffic": traffic,
                "peak_source": "measured cuBLAS BF16 burst (MEASURED_PEAKS.json)"
                               + ("; TF32 = BF16 x 1.1/2.25 nominal" if form == "tf32x3" else ""),
                "flops": "executed split-product MMA flops", "launches": nc,
                "avg_launch_ms": msc / nc if nc else None}

    def df_roofline(prof):
        nc, msc = prof.get("contract", (0, 0.0))
        inst = sum(contraction_df_inst(w.X, nd, P, pairs) for nd in job_nd)
        ach = inst * args.steps / (msc / 1e3) / 1e12 if nc else None
        flops = contract_alg * args.steps / (msc / 1e3) / 1e12 if nc else None
        return {"bound": "alu", "kernel": "k_contract_df", "achieved": ach,
                "peak": FP32_INST_PEAK, "unit": "T FP32-inst/s",
                "frac": ach / FP32_INST_PEAK if ach else None,
                "traffic": load_traffic("k_contract_df") if default_shape else None,
                "peak_source": "derived: 128 FP32 instructions/clk/SM x 152 SMs x 2070 MHz",
                "flops": "modelled FP32 instructions of the double-float inner loops",
                "complex_count_tflops": flops, "launches": nc,
                "avg_launch_ms": msc / nc if nc else None}

    clk = ClockSampler(local)
    ctx, outs, ms, prof, launches = measure(head, clk)
    value = job_throughput(world, blocks_per_step, args.steps, ms / 1e3)

    # roofline of the dominant kernel (the contraction): algorithmic flops / event time
    if head == "fp64":
        n_c, ms_c = prof.get("contract", (0, 0.0))
        flops_per_launch = contract_alg * args.steps / n_c if n_c else None
        achieved = contract_alg * args.steps / (ms_c / 1e3) / 1e12 if n_c else None
        roofline = {
            "bound": "alu", "kernel": "k_contract_fp64", "achieved": achieved,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
            "traffic": load_traffic("k_contract_fp64") if default_shape else None,
            "peak_source": "derived: 4 FP64 flop/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
            "flops_per_launch": flops_per_launch,
            "launches": n_c, "avg_launch_ms": ms_c / n_c if n_c else None,
        }
    else:
        roofline = tensor_roofline(head, prof)
    kernels = {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / ms if ms else None}
               for k, v in prof.items()}

    # the tensor-core forms on the same inputs; error against the FP64 form's blocks
    forms = {}
    if not args.no_forms and head == "fp64":
        B64 = [o.cpu().numpy() for o in outs]
        nrm = math.sqrt(sum(np.linalg.norm(b) ** 2 for b in B64))
        for name in ("df64", "bf16x6", "bf16x9", "tf32x3", "bf16x3"):
            c2, o2, t_ms, pr, nl = measure(name)
            err = math.sqrt(sum(np.linalg.norm(a.cpu().numpy() - b) ** 2
                                for a, b in zip(o2, B64))) / nrm
            nc, msc = pr.get("contract", (0, 0.0))
            forms[name] = {
                "blocks_per_s": job_throughput(world, blocks_per_step, args.steps, t_ms / 1e3),
                "ms_per_step": t_ms / args.steps, "gpu_launches": nl,
                "rel_frobenius_err_vs_fp64_form": err,
                "speedup_vs_fp64_form": ms / t_ms,
                "contract_ms_per_launch": msc / nc if nc else None,
                ("alu_roofline" if name == "df64" else "tensor_roofline"):
                    df_roofline(pr) if name == "df64" else tensor_roofline(name, pr),
                "kernels": {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / t_ms}
                            for k, v in pr.items()},
            }
            bb.bblock_destroy(c2)

    # the mode-triplet ordering (Sec. 2, Eq. 4): T per time slice (noise-independent), then
    # blocks from T by three FP64 mode products; the crossover is the number of noise
    # triples per time slice above which T + n * (blocks from T) beats n * (direct blocks)
    triplet = None
    if not args.no_triplet and not batched and max(nd0 := inp.ndil[0]) <= w.n_ev <= 256:
        triplet = {}
        mom = inp.momenta
        Tbuf = torch.empty((w.n_t, P, w.n_ev, w.n_ev, w.n_ev), dtype=torch.complex128, device=dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for name in ("fp64", "df64"):
            c3 = bb.bblock_create(w.L, w.n_ev, w.n_ev, FORMS[name][0], device=local)
            bb.bblock_mode_triplet(c3, V, mom, T_out=Tbuf, stream=stream)    # warm-up
            bb.bblock_status(c3)
            ev0.record(stream)
            bb.bblock_mode_triplet(c3, V, mom, T_out=Tbuf, stream=stream)
            ev1.record(stream)
            bb.bblock_status(c3)
            triplet[f"T_ms_per_time_slice_{name}"] = ev0.elapsed_time(ev1) / w.n_t
            if name == "df64":
                Bt = torch.empty_like(outs[0])
                for k in range(max(1, args.warmup)):
                    bb.bblock_from_triplet(c3, Tbuf, *phis[0], inp.spins, inp.coeffs, B_out=Bt,
                                           stream=stream)
                bb.bblock_status(c3)
                ev0.record(stream)
                for k in range(args.steps):
                    bb.bblock_from_triplet(c3, Tbuf, *phis[0], inp.spins, inp.coeffs, B_out=Bt,
                                           stream=stream)
                ev1.record(stream)
                bb.bblock_status(c3)
                ft = ev0.elapsed_time(ev1) / args.steps / w.n_t
                triplet["blocks_from_T_ms_per_time_slice"] = ft
                triplet["rel_frobenius_err_vs_fp64_form"] = float(
                    np.linalg.norm(Bt.cpu().numpy() - outs[0].cpu().numpy()) /
                    np.linalg.norm(outs[0].cpu().numpy()))
            bb.bblock_destroy(c3)
        direct = {"fp64": ms / args.steps / w.n_t}
        if "df64" in forms:
            direct["df64"] = forms["df64"]["ms_per_step"] / w.n_t
        triplet["direct_ms_per_time_slice"] = direct
        ft = triplet["blocks_from_T_ms_per_time_slice"]
        triplet["crossover_noise_triples"] = {
            k: (triplet[f"T_ms_per_time_slice_{k}"] / (v - ft) if v > ft else None)
            for k, v in direct.items()}
        del Tbuf

    # end to end through the public API with host buffers: every step copies the inputs
    # from pinned host memory, computes, and copies the blocks back
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(inp.V).pin_memory()
        hphi = [[torch.from_numpy(inp.phi[k][i]).pin_memory() for i in range(3)]
                for k in range(w.n_noise)]
        hB = [torch.empty(tuple(o.shape), dtype=torch.complex128).pin_memory() for o in outs]
        if batched:
            dV = torch.empty_like(V)
            dphi = [[torch.empty_like(p) for p in ph] for ph in phis]
            douts = outputs()
            jobs = [(dV[t], dphi[k][0][t], dphi[k][1][t], dphi[k][2][t], douts[k][t])
                    for k in range(w.n_noise) for t in range(w.n_t)]

            def e2e_step():
                with torch.cuda.stream(stream):
                    dV.copy_(hV, non_blocking=True)
                    for k in range(w.n_noise):
                        for i in range(3):
                            dphi[k][i].copy_(hphi[k][i], non_blocking=True)
                bb.bblock_compute_batch(ctx, jobs, inp.momenta, inp.spins, inp.coeffs,
                                        stream=stream)
                with torch.cuda.stream(stream):
                    for k in range(w.n_noise):
                        hB[k].copy_(douts[k], non_blocking=True)
                stream.synchronize()
        else:
            def e2e_step():
                bb.bblock_compute_host(ctx, hV, *hphi[0], inp.momenta, inp.spins, inp.coeffs,
                                       hB[0], stream)
        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        # the host path computes in chunks of time slices, whose site slabs may differ from
        # the device call's: the two agree to the form's rounding, not bit for bit
        tol = 1e-12 if head in ("fp64", "df64") else 1e-5
        for h, o in zip(hB, outs):
            ref = o.cpu().numpy()
            err = np.linalg.norm(h.numpy() - ref) / max(np.linalg.norm(ref), 1e-300)
            assert err <= tol, f"host and device paths differ by {err:.2e}"
        h2d = hV.numel() * 16 + sum(p.numel() * 16 for ph in hphi for p in ph)
        e2e = {"value": job_throughput(world, blocks_per_step, args.steps, dt), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": sum(h.numel() * 16 for h in hB)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(workloads.generate(w, n_t=4), args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        nd0 = inp.ndil[0]
        field_bytes = sum(3 * w.X * 16 * (n_alpha * nd[0] + n_beta * nd[1] + pairs * nd[2])
                          for nd in job_nd)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if head == "fp64" else ("tf32" if head == "tf32x3" else "bf16"),
            "data": "synthetic (seeded, workloads.py)",
            "config": {"workload": w.name, "L": w.L, "X": w.X, "n_ev": w.n_ev,
                       "ndil": nd0[0] if not batched else sorted({nd[0] for nd in inp.ndil}),
                       "n_t": w.n_t, "n_noise": w.n_noise, "n_mom": P,
                       "n_spin": len(inp.spins), "spin_pairs": pairs, "form": head,
                       "blocks_per_step_per_gpu": blocks_per_step,
                       "l2": "inputs larger than L2 (V %.0f MB, fields %.0f MB per step)" % (
                           inp.V.nbytes / 1e6, field_bytes / 1e6),
                       "parallelism": f"{world} independent GPU(s), no collective",
                       "tuned_tiles": tuned.get(head)},
            "algorithmic_tflops": (contract_alg + project_alg) * args.steps / (ms / 1e3) / 1e12,
            "gpu_launches": launches,
            "kernels": kernels,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "forms": forms,
            "mode_triplet": triplet,
        }
        print(json.dumps(line), flush=True)
    bb.bblock_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
