"""The mode-triplet ordering on the GPU (Sec. 2, Eq. 4), through the C ABI.

* T from each form against the oracle's Eq. (4), which is written out independently of the
  direct contraction.
* Blocks from T (three FP64 mode products) against the oracle's direct Eq. (1)/(3). The
  cases cover several spin pairs, several gamma spins sharing a pair, per-momentum
  coefficients and unequal dilution sizes.
* The two orderings on the GPU agree at the benchmarked shape (L = 24, N_ev = 96).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("precision,products,tol", [("fp64", 6, 1e-12), ("df64", 6, 1e-12),
                                                    ("bf16", 6, 1e-6), ("tf32x3", 6, 1e-6),
                                                    ("fp16x3", 6, 1e-6)])
def test_mode_triplet_matches_eq4(env, precision, products, tol):
    torch, bb = env
    mom = [(0, 0, 0), (1, 0, 0), (-1, 1, 2)]
    inp = workloads.custom(4, 8, (8, 8, 8), 2, mom, [(0, 0, 0)], [1.0], seed=6000)
    V = torch.from_numpy(inp.V).to("cuda:0")
    ctx = bb.bblock_create(4, 8, 8, precision, bf16_products=products)
    T = bb.bblock_mode_triplet(ctx, V, mom)
    bb.bblock_status(ctx)
    got = T.cpu().numpy()
    for t in range(2):
        ref = oracle.mode_triplet(4, inp.V[t], mom)
        assert rel(got[t], ref) <= tol
    bb.bblock_destroy(ctx)


CASES = [
    # L, n_ev, (nd1, nd2, nd3), momenta, spins, coeffs
    (3, 6, (5, 4, 7), [(0, 0, 0), (1, 0, 0)], [(0, 1, 0), (1, 0, 0), (2, 3, 2)],
     [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    (4, 9, (6, 6, 6), [(0, 0, 0), (0, 1, 1), (1, 1, 0)],
     [(0, 1, 2), (0, 1, 3), (0, 1, 0), (2, 2, 1), (3, 1, 2)], [0.5, -0.25j, 1.0, 0.3 + 0.1j, -0.7]),
    (2, 5, (3, 9, 2), [(0, 0, 0), (1, 1, 1)], [(3, 3, 3)], [1.0]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_blocks_through_the_triplet_match_the_definition(env, case):
    torch, bb = env
    L, n_ev, nd, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, 2, mom, spins, coeffs, seed=6100 + case)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(L, n_ev, max(max(nd), n_ev), "fp64")
    T = bb.bblock_mode_triplet(ctx, V, mom)
    B = bb.bblock_from_triplet(ctx, T, *phis, spins, coeffs)
    bb.bblock_status(ctx)
    got = B.cpu().numpy()
    for t in range(2):
        ref = oracle.bblock(L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)], mom, spins, coeffs)
        assert rel(got[t], ref) <= 1e-12
    bb.bblock_destroy(ctx)


def test_momentum_dependent_coefficients_through_the_triplet(env):
    torch, bb = env
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    rng = np.random.default_rng(6200)
    coeffs = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    inp = workloads.custom(3, 7, (6, 5, 4), 1, mom, spins, np.ones(3), seed=6201)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(3, 7, 7, "fp64")
    T = bb.bblock_mode_triplet(ctx, V, mom)
    B = bb.bblock_from_triplet(ctx, T, *phis, spins, coeffs)
    bb.bblock_status(ctx)
    ref = oracle.bblock(3, inp.V[0], *[inp.phi[0][i][0] for i in range(3)], mom, spins, coeffs)
    assert rel(B.cpu().numpy()[0], ref) <= 1e-12
    bb.bblock_destroy(ctx)


def test_both_orderings_agree_at_l24_nev96(env):
    """One time slice of the benchmarked workload: direct path and mode-triplet path in the
    FP64 form agree, and sampled entries match the oracle."""
    torch, bb = env
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w, n_t=1)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(w.L, w.n_ev, w.n_ev, "fp64")
    direct = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    T = bb.bblock_mode_triplet(ctx, V, inp.momenta)
    via = bb.bblock_from_triplet(ctx, T, *phis, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    a, b = direct.cpu().numpy(), via.cpu().numpy()
    assert rel(b, a) <= 1e-12
    d1s, d2s, d3s = [0, 17, 31], [2, 31], [0, 31]
    ref = oracle.bblock_sampled(w.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)],
                                inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
    assert rel(b[0][:, d1s][:, :, d2s][:, :, :, d3s], ref) <= 1e-12
    bb.bblock_destroy(ctx)


def test_triplet_needs_max_ndil_of_at_least_n_ev(env):
    torch, bb = env
    inp = workloads.custom(2, 6, (4, 4, 4), 1, [(0, 0, 0)], [(0, 0, 0)], [1.0], seed=6300)
    V = torch.from_numpy(inp.V).to("cuda:0")
    ctx = bb.bblock_create(2, 6, 4, "fp64")
    with pytest.raises(bb.BblockError, match="INVALID_ARG"):
        bb.bblock_mode_triplet(ctx, V, [(0, 0, 0)])
    bb.bblock_destroy(ctx)
