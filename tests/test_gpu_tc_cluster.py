"""The tensor-core contraction with thread-block clusters (BF16 forms), through the C ABI.

With C CTAs per cluster each CTA builds 128/C rows of the diquark tile and pushes them into
its peers' stage buffers. The cluster run must equal the plain kernel bit for bit when the
N tile and slab count are the same: every output column is still computed by one CTA, from
identical operand pieces, in the same MMA order. It must also match the oracle, including
ragged shapes where some CTAs of a cluster get an empty N tile. It must replay unchanged
from a CUDA graph.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = [("bf16", 6, 1e-6), ("bf16", 9, 1e-6), ("bf16", 3, 1e-4)]
FORM_IDS = ["bf16x6", "bf16x9", "bf16x3"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_16278_gb300 as bb
    bb.load()
    return torch, bb


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    (5, 12, (12, 11, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    (6, 16, (16, 16, 20), 1, [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
    (4, 10, (24, 20, 30), 1, [(0, 0, 0), (-1, 2, 1), (1, 1, 1), (0, 0, 1)],
     [(1, 2, 3), (0, 1, 3)], [0.3 - 0.2j, 1.0]),
]


def blocks(torch, bb, inp, precision, products, cluster, nc=0, slabs=0, stream=None):
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), precision, bf16_products=products)
    bb.bblock_set_option(ctx, "tc_cluster", cluster)
    bb.bblock_set_option(ctx, "tc_nc", nc)
    bb.bblock_set_option(ctx, "slabs", slabs)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, stream=stream)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    bb.bblock_destroy(ctx)
    return out


@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("form", range(len(FORMS)), ids=FORM_IDS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_cluster_equals_plain_kernel_and_oracle(env, case, form, cluster):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    precision, products, tol = FORMS[form]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=8000 + case)
    plain = blocks(torch, bb, inp, precision, products, 1, nc=16, slabs=3)
    clustered = blocks(torch, bb, inp, precision, products, cluster, nc=16, slabs=3)
    assert np.array_equal(clustered, plain)
    ref = np.stack([oracle.bblock(L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)], mom, spins,
                                  coeffs) for t in range(n_t)])
    assert rel(clustered, ref) <= tol


def test_benchmarked_shape_with_clusters_of_two(env):
    """L = 24, N_ev = 96, N_dil = 32 with clusters of 2 (its two N tiles per cluster):
    sampled entries against the oracle, and equality with a plain run of the same tiles."""
    torch, bb = env
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w, n_t=2)
    clustered = blocks(torch, bb, inp, "bf16", 6, 2, nc=48, slabs=8)
    plain = blocks(torch, bb, inp, "bf16", 6, 1, nc=48, slabs=8)
    assert np.array_equal(clustered, plain)
    d1s, d2s, d3s = [0, 13, 31], [5, 31], [0, 30, 31]
    for t in range(2):
        ref = oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                    inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
        assert rel(clustered[t][:, d1s][:, :, d2s][:, :, :, d3s], ref) <= 1e-6


def test_cluster_graph_replay_is_bitwise_equal(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[1]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=8100)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(L, n_ev, max(nd), "bf16", bf16_products=6)
    bb.bblock_set_option(ctx, "tc_cluster", 4)
    stream = torch.cuda.Stream()
    B = torch.empty((n_t, len(mom), *nd), dtype=torch.complex128, device=dev)
    outs = []
    for call in range(4):          # plain launches, capture + replay, replays
        with torch.cuda.stream(stream):
            B.zero_()
        bb.bblock_compute(ctx, V, *phis, mom, spins, coeffs, B_out=B, stream=stream)
        bb.bblock_status(ctx)
        outs.append(B.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    bb.bblock_destroy(ctx)
