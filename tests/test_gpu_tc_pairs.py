"""The FP16 form's CTA pairs, through the C ABI.

Two CTAs of a cluster take adjacent 128-pair tiles of one N tile. Each builds its own
diquark rows and half of the third-quark rows, and copies that half into the peer's stage;
each then multiplies its diquark rows by the whole third-quark tile, which may be up to 80
complex columns wide (the accumulators are single-buffered beyond 48). These tests compare
every N tile width against the CPU oracle, on shapes with an odd number of 128-pair tiles
(the second CTA of the last pair has no rows), with N tiles that do not divide the (p, d3)
columns, and with fewer third-quark rows than a copy group; the pairs must also agree with
the plain FP16 kernel to the form's tolerance and replay bitwise from a CUDA graph.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-6


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
    # 144 pairs: two 128-pair tiles; 3 x 13 = 39 (p, d3) columns
    (5, 12, (12, 12, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    # 320 pairs: three 128-pair tiles (an odd count); 5 x 20 = 100 columns
    (6, 16, (16, 20, 20), 1, [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
    # 480 pairs: four tiles, the last one ragged; 4 x 30 = 120 columns
    (4, 10, (24, 20, 30), 1, [(0, 0, 0), (-1, 2, 1), (1, 1, 1), (0, 0, 1)],
     [(1, 2, 3), (0, 1, 3)], [0.3 - 0.2j, 1.0]),
    # a single small tile: 72 pairs, 1 x 7 columns (fewer third-quark rows than one N tile)
    (3, 9, (9, 8, 7), 1, [(0, 0, 0)], [(0, 0, 0)], [1.0]),
]


def blocks(torch, bb, inp, cluster, nc=0, stream=None, ctx=None):
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), "fp16x3")
        bb.bblock_set_option(ctx, "tc_cluster", cluster)
        bb.bblock_set_option(ctx, "tc_nc", nc)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, stream=stream)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    if own:
        bb.bblock_destroy(ctx)
    return out


def oracle_blocks(inp):
    w = inp.workload
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, inp.coeffs)
                     for t in range(inp.V.shape[0])])


@pytest.mark.parametrize("nc", [16, 32, 48, 64, 80])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_pairs_match_oracle_at_every_tile_width(env, case, nc):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=8000 + case)
    got = blocks(torch, bb, inp, cluster=2, nc=nc)
    err = rel(got, oracle_blocks(inp))
    print(f"fp16x3 pairs case {case} nc {nc}: rel. Frobenius error {err:.3e}")
    assert np.all(np.isfinite(got)) and err <= TOL


@pytest.mark.parametrize("case", range(len(CASES)))
def test_pairs_agree_with_plain_kernel(env, case):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=8100 + case)
    pairs = blocks(torch, bb, inp, cluster=0)           # the default: CTA pairs
    plain = blocks(torch, bb, inp, cluster=1)
    ref = oracle_blocks(inp)
    assert rel(pairs, ref) <= TOL and rel(plain, ref) <= TOL
    assert rel(pairs, plain) <= 2 * TOL


def test_pairs_replay_bitwise_from_graph(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[1]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=8200)
    ctx = bb.bblock_create(L, n_ev, max(nd), "fp16x3")
    bb.bblock_set_option(ctx, "tc_nc", 80)
    stream = torch.cuda.Stream()
    outs = [blocks(torch, bb, inp, 0, stream=stream, ctx=ctx) for _ in range(4)]
    bb.bblock_destroy(ctx)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert rel(outs[0], oracle_blocks(inp)) <= TOL


def test_tile_option_limits(env):
    """N tiles of 64 and 80 columns are the FP16 form's (its CTA pairs); the other forms
    reject them."""
    torch, bb = env
    ctx = bb.bblock_create(4, 8, 16, "fp16x3")
    for nc in (16, 32, 48, 64, 80):
        bb.bblock_set_option(ctx, "tc_nc", nc)
        assert bb.bblock_get_option(ctx, "tc_nc") == nc
    bb.bblock_destroy(ctx)
    ctx = bb.bblock_create(4, 8, 16, "bf16", bf16_products=6)
    with pytest.raises(bb.BblockError):
        bb.bblock_set_option(ctx, "tc_nc", 64)
    bb.bblock_destroy(ctx)
