"""The benchmark's reference arm on the CPU: `bench.py --impl reference` times the FP64
oracle on a bounded sample and prints one JSON line with the same metric and keys as the
GPU arm, plus its CPU-baseline description; ranks other than 0 print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
       "--warmup", "0", "--cpu-seconds", "2", "--workload", "l4_nev8_ndil8"]


def run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == "baryon blocks/s" and d["unit"] == "blocks/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "l4_nev8_ndil8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_size_sweep_fit_recovers_power_laws():
    """The size sweep's exponent fit (least squares on log-log) returns the power of an exact
    power law, and the sweep's points span both series it fits."""
    sys.path.insert(0, ROOT)
    import bench
    for k in (2.0, 3.0):
        assert abs(bench.loglog_slope([16, 24, 32, 48], [7.0 * L ** k for L in (16, 24, 32, 48)]) - k) < 1e-12
    assert bench.parse_args(["--size-sweep"]).size_sweep
    Ls = sorted({L for L, D in bench.SWEEP_POINTS if D == 32})
    Ds = sorted({D for L, D in bench.SWEEP_POINTS if L == 32})
    assert len(Ls) >= 3 and len(Ds) >= 3
