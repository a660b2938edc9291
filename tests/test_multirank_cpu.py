"""The multi-rank host logic of ``bench.py``, as two ``gloo`` ranks on the CPU.

Time slices are independent units, so ranks shard them with no data-path collective:
every rank draws its own inputs and the only exchange is the maximum of the timings. Two
processes check that the ranks' inputs differ, that the reported time is the slowest rank's,
and that the whole-job value counts the blocks of every rank. The oracle stands in for the
GPU path: each rank computes its own blocks on the CPU and agrees with the blocks
recomputed from its seed alone.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import workloads
    w = workloads.WORKLOADS["l4_nev8_ndil8"]
    inp = bench.rank_inputs(w, rank)
    B = oracle.bblock(w.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)], inp.momenta,
                      inp.spins, inp.coeffs)
    t_local = 1.0 + rank                        # rank 1 is the slower one
    t_max = bench.max_over_ranks(t_local, world)
    value = bench.job_throughput(world, len(inp.momenta), 5, t_max)
    # gather every rank's first input entry to rank 0 to compare draws
    v0 = torch.tensor([inp.V[0].real.flat[0], inp.V[0].imag.flat[0]], dtype=torch.float64)
    got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, v0)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            {"B": B, "t_max": t_max, "value": value,
             "v0": [g.numpy() for g in got]}, allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import oracle
    oracle.build()
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npy", allow_pickle=True).item() for r in range(world)]
    for r in res:
        assert r["t_max"] == 2.0                 # the slower rank's time
        assert r["value"] == pytest.approx(world * 1 * 5 / 2.0)
    v0 = res[0]["v0"]
    assert not np.array_equal(v0[0], v0[1])       # each rank drew its own time slices
    assert not np.allclose(res[0]["B"], res[1]["B"])
    import bench
    import workloads
    w = workloads.WORKLOADS["l4_nev8_ndil8"]
    for rank, r in enumerate(res):                # a rank's blocks follow from its seed alone
        inp = bench.rank_inputs(w, rank)
        ref = oracle.bblock(w.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)], inp.momenta,
                            inp.spins, inp.coeffs)
        assert np.array_equal(r["B"], ref)
