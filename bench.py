#!/usr/bin/env python
"""Baryon-block throughput on GB300: blocks/s of the L=24, N_ev=96, N_dil=32 workload.

One step = the whole hot path (phase table from cache, projection of the three quark
lines for every spin used, fused diquark + contraction, slab reduction) over 8 time
slices x 3 momenta x one 3-triple baryon operator, i.e. 24 blocks B[t][p][d1][d2][d3].
Inputs are seeded synthetic draws (``workloads.py``) resident on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

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
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the tensor-core forms (time the FP64 form only)")
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
    """Time the CPU FP64 oracle on a bounded sample of the workload: time slice 0, all
    momenta, the first n_thr values of d1 (the oracle's OpenMP loop runs over d1, so each
    thread gets one), the first k values of d2, all d3. Returns (blocks/s, threads, text)."""
    import oracle
    w = inp.workload
    nd = inp.ndil[0]
    phis = [inp.phi[0][i][0] for i in range(3)]
    n1 = max(1, min(nd[0], oracle.num_threads()))
    d1s, all3 = list(range(n1)), list(range(nd[2]))

    def run(k):
        t0 = time.perf_counter()
        oracle.bblock_sampled(w.L, inp.V[0], *phis, inp.momenta, inp.spins, inp.coeffs,
                              d1s, list(range(k)), all3)
        return time.perf_counter() - t0

    t1 = run(1)
    k = int(max(1, min(nd[1], round(target_s / max(t1, 1e-3)))))
    tk = run(k) if k > 1 else t1
    blocks = len(inp.momenta) * n1 * k / (nd[0] * nd[1])
    text = (f"time slice 0, {len(inp.momenta)} momenta, d1 in [0,{n1}), d2 in [0,{k}) of "
            f"{nd[1]}, all {nd[2]} d3 = {blocks:.5f} blocks in {tk:.2f} s on {n1} threads")
    return blocks / tk, n1, text


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workloads.WORKLOADS[args.workload]
    inp = workloads.generate(w, n_t=1)
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
    inp = workloads.generate(w, seed=w.seed + rank)  # each rank: its own time slices
    nd = inp.ndil[0]
    P = len(inp.momenta)
    n_alpha, n_beta, pairs = spin_structure(inp.spins)
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    # a created stream: repeated calls are then replayed from a CUDA graph by the library
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    blocks_per_step = w.n_t * P

    def measure(precision, products, sampler=None):
        """W untimed + K timed steps of one form; CUDA events on the launching stream."""
        c = bb.bblock_create(w.L, w.n_ev, max(nd), precision, bf16_products=products,
                             device=local)
        out = torch.empty((w.n_t, P, *nd), dtype=torch.complex128, device=dev)

        def step():
            bb.bblock_compute(c, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=out,
                              stream=stream)

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
        if world > 1:
            t = torch.tensor([t_ms], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_ms = float(t.item())
        return c, out, t_ms, prof, n_launch

    clk = ClockSampler(local)
    ctx, B, ms, prof, launches = measure("fp64", 6, clk)
    value = world * blocks_per_step * args.steps / (ms / 1e3)

    # roofline of the dominant kernel (the contraction): algorithmic flops / event time
    n_c, ms_c = prof.get("contract", (0, 0.0))
    groups = math.ceil(P / 8)
    flops_per_launch = w.n_t * contraction_flops(w.X, nd, P, pairs) / groups
    achieved = flops_per_launch / (ms_c / n_c / 1e3) / 1e12 if n_c else None
    roofline = {
        "bound": "alu", "kernel": "k_contract_fp64", "achieved": achieved,
        "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
        "traffic": load_traffic("k_contract_fp64"),
        "peak_source": "derived: 4 FP64 flop/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
        "flops_per_launch": flops_per_launch,
        "launches": n_c, "avg_launch_ms": ms_c / n_c if n_c else None,
    }
    kernels = {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / ms if ms else None}
               for k, v in prof.items()}

    # the tensor-core forms on the same inputs; error against the FP64 form's blocks
    forms = {}
    if not args.no_forms:
        B64 = B.cpu().numpy()
        nrm = np.linalg.norm(B64)
        # useful complex GEMM work of the folded contraction: 8 M N K per job, K = 3 pairs X
        gemm_flops = w.n_t * 8.0 * nd[0] * nd[1] * (P * nd[2]) * (3 * pairs * w.X)
        for name, prec, prods, nprod, peak in (
                ("bf16x6", "bf16", 6, 6, BF16_PEAK_TFLOPS), ("bf16x9", "bf16", 9, 9, BF16_PEAK_TFLOPS),
                ("tf32x3", "tf32x3", 6, 3, TF32_PEAK_TFLOPS), ("bf16x3", "bf16", 3, 3, BF16_PEAK_TFLOPS)):
            c2, out, t_ms, pr, nl = measure(prec, prods)
            err = float(np.linalg.norm(out.cpu().numpy() - B64) / nrm)
            nc, msc = pr.get("contract", (0, 0.0))
            execd = gemm_flops * nprod / (msc / nc / 1e3) / 1e12 if nc else None
            forms[name] = {
                "blocks_per_s": world * blocks_per_step * args.steps / (t_ms / 1e3),
                "ms_per_step": t_ms / args.steps, "gpu_launches": nl,
                "rel_frobenius_err_vs_fp64_form": err,
                "speedup_vs_fp64_form": ms / t_ms,
                "contract_ms_per_launch": msc / nc if nc else None,
                "tensor_roofline": {"bound": "tensor", "achieved": execd, "peak": peak,
                                    "unit": "TFLOP/s", "frac": execd / peak if execd else None,
                                    "flops": "executed split-product MMA flops"},
                "kernels": {k: {"launches": v[0], "total_ms": v[1], "share": v[1] / t_ms}
                            for k, v in pr.items()},
            }
            bb.bblock_destroy(c2)

    # end to end through the host-buffer entry point: H2D inputs + compute + D2H blocks
    e2e = None
    if not args.no_e2e:
        hV = torch.from_numpy(inp.V).pin_memory()
        hphi = [torch.from_numpy(inp.phi[0][i]).pin_memory() for i in range(3)]
        hB = torch.empty((w.n_t, P, *nd), dtype=torch.complex128).pin_memory()
        for _ in range(max(1, args.warmup // 2)):
            bb.bblock_compute_host(ctx, hV, *hphi, inp.momenta, inp.spins, inp.coeffs, hB, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            bb.bblock_compute_host(ctx, hV, *hphi, inp.momenta, inp.spins, inp.coeffs, hB, stream)
        dt = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        assert np.array_equal(hB.numpy(), B.cpu().numpy()), "host and device entry points differ"
        h2d = hV.numel() * 16 + sum(p.numel() * 16 for p in hphi)
        e2e = {"value": world * blocks_per_step * args.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": hB.numel() * 16}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(workloads.generate(w, n_t=1), args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        total_flops = w.n_t * (contraction_flops(w.X, nd, P, pairs) +
                               projection_flops(w.X, w.n_ev, nd, n_alpha, n_beta, pairs))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded, workloads.py)",
            "config": {"workload": w.name, "L": w.L, "X": w.X, "n_ev": w.n_ev, "ndil": nd[0],
                       "n_t": w.n_t, "n_mom": P, "n_spin": len(inp.spins), "spin_pairs": pairs,
                       "form": "fp64", "blocks_per_step_per_gpu": blocks_per_step,
                       "l2": "inputs larger than L2 (V %.0f MB, fields %.0f MB per step)" % (
                           inp.V.nbytes / 1e6, 3 * w.X * 16 * w.n_t *
                           (n_alpha * nd[0] + n_beta * nd[1] + pairs * nd[2]) / 1e6),
                       "parallelism": f"{world} independent GPU(s), no collective"},
            "algorithmic_tflops": total_flops * args.steps / (ms / 1e3) / 1e12,
            "gpu_launches": launches,
            "kernels": kernels,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "forms": forms,
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
