"""The FP64-accurate tensor-core form (BBLOCK_OZAKI), through the C ABI, against the oracle.

The form splits the double-float diquark and phase-folded third quark into seven BF16
digits per entry, scaled per row (d1, d2) and column d3 of every site slab by a power of
two, and sums the digit products exactly on the tensor cores. These tests hold it to the
FP64 forms' parity target, 1e-12 relative Frobenius error, on:

* shapes with ragged M tiles (nd1 nd2 not a multiple of 128), ragged N tiles (P nd3 not a
  multiple of the tile width), ragged K (sites x pairs x 3 not a multiple of 16) and
  several site slabs, at every N tile width (16, 32, 48 complex columns);
* per-momentum spin coefficients (one launch per momentum);
* fields whose columns span 2^-40 .. 2^40: every (d1, d3) sub-block must keep its own
  relative accuracy, which a single per-job scale could not give;
* all-zero inputs (exact zeros) and a job of one site;
* agreement with the FP64 form, and bitwise-identical graph replays.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


C4_MOM = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 0), (-1, -1, 0)]
CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    # 144 rows (2 M tiles), 9 x 13 = 117 columns, K = 64 x 4 x 3
    (4, 10, (12, 12, 13), 2, C4_MOM,
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
    # 320 rows, 5 x 20 columns, 3 pairs: K = 125 x 9 (not a multiple of 16)
    (5, 12, (16, 20, 20), 1, [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    # momenta beyond L and negative, complex coefficients, 2 pairs
    (6, 14, (10, 9, 17), 1, [(7, 0, 0), (1, 2, -3), (-5, 4, 1)],
     [(1, 2, 3), (0, 1, 3)], [0.3 - 0.2j, 1.0]),
    # one pair, one momentum, a single tile of 72 rows and 7 columns
    (3, 9, (9, 8, 7), 1, [(0, 0, 0)], [(0, 0, 0)], [1.0]),
]


def device_inputs(torch, inp, scale=None):
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i] if scale is None else scale[i]).to(dev)
            for i in range(3)]
    return V, phis


def reference(inp, coeffs=None, phis=None):
    w = inp.workload
    c = inp.coeffs if coeffs is None else coeffs
    ph = inp.phi[0] if phis is None else phis
    return np.stack([oracle.bblock(w.L, inp.V[t], *[ph[i][t] for i in range(3)],
                                   inp.momenta, inp.spins, c) for t in range(inp.V.shape[0])])


def compute(torch, bb, inp, precision="ozaki", nc=0, slabs=0, coeffs=None, phis=None,
            stream=None, ctx=None, cluster=0):
    w = inp.workload
    V, ph = device_inputs(torch, inp, phis)
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), precision)
        bb.bblock_set_option(ctx, "tc_nc", nc)
        bb.bblock_set_option(ctx, "slabs", slabs)
        if precision == "ozaki":
            bb.bblock_set_option(ctx, "tc_cluster", cluster)
    B = bb.bblock_compute(ctx, V, *ph, inp.momenta, inp.spins,
                          inp.coeffs if coeffs is None else coeffs, stream=stream)
    bb.bblock_status(ctx)
    if own:
        assert bb.bblock_last_path(ctx) == ("ozaki" if precision == "ozaki" else "fp64")
        bb.bblock_destroy(ctx)
    return B.cpu().numpy()


@pytest.mark.parametrize("cluster", [1, 2, 3, 4])
@pytest.mark.parametrize("slabs", [0, 3])
@pytest.mark.parametrize("nc", [16, 32, 48])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_matches_oracle(env, case, nc, slabs, cluster):
    """Clusters of 2-4 CTAs share each diquark tile; ragged last clusters (N tiles not a
    multiple of the cluster size) compute zero third-quark rows and write nothing."""
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12000 + case)
    got = compute(torch, bb, inp, nc=nc, slabs=slabs, cluster=cluster)
    err = rel(got, reference(inp))
    print(f"ozaki case {case} nc {nc} slabs {slabs} cluster {cluster}: rel. error {err:.3e}")
    assert np.all(np.isfinite(got)) and err <= TOL


@pytest.mark.parametrize("cluster", [2, 3, 4])
def test_clusters_are_bitwise_the_plain_kernel(env, cluster):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[0]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12050)
    plain = compute(torch, bb, inp, cluster=1)
    assert np.array_equal(compute(torch, bb, inp, cluster=cluster), plain)


def test_per_momentum_coefficients(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, _ = CASES[0]
    rng = np.random.default_rng(12100)
    coeffs = rng.standard_normal((len(mom), len(spins))) + 1j * rng.standard_normal((len(mom), len(spins)))
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs[0], seed=12100)
    got = compute(torch, bb, inp, coeffs=coeffs)
    err = rel(got, reference(inp, coeffs))
    print(f"ozaki per-momentum coefficients: rel. Frobenius error {err:.3e}")
    assert err <= TOL


def test_wide_dynamic_range_per_row_and_column(env):
    """Columns of phi1 scaled by 2^k1(d1), k1 in [-20, 20], and of phi3 by 2^k3(d3), k3 in
    [-40, 40]: block (d1, d3) scales by 2^(k1 + k3). Each (d1, d3) sub-block (all p, d2)
    must meet the tolerance relative to its own norm."""
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[0]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12200)
    k1 = np.linspace(-20, 20, nd[0]).round().astype(int)
    k3 = np.linspace(-40, 40, nd[2]).round().astype(int)
    phis = [inp.phi[0][0] * np.ldexp(1.0, k1)[None, None, :], inp.phi[0][1],
            inp.phi[0][2] * np.ldexp(1.0, k3)[None, None, :]]
    phis = [np.ascontiguousarray(p) for p in phis]
    got = compute(torch, bb, inp, phis=phis)
    ref = reference(inp, phis=phis)
    worst = 0.0
    for d1 in range(nd[0]):
        for d3 in range(nd[2]):
            worst = max(worst, rel(got[:, :, d1, :, d3], ref[:, :, d1, :, d3]))
    print(f"ozaki dynamic range: worst (d1, d3) sub-block rel. error {worst:.3e}")
    assert worst <= TOL


def test_zero_inputs_give_exact_zeros(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[1]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12300)
    zeros = [np.zeros_like(inp.phi[0][i]) for i in range(3)]
    got = compute(torch, bb, inp, phis=zeros)
    assert np.array_equal(got, np.zeros_like(got))


def test_single_site_lattice(env):
    torch, bb = env
    inp = workloads.custom(1, 3, (5, 4, 6), 2, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (1, 0, 0)], [0.6, -0.8], seed=12400)
    got = compute(torch, bb, inp)
    assert rel(got, reference(inp)) <= TOL


@pytest.mark.parametrize("case", range(len(CASES)))
def test_agrees_with_fp64_form(env, case):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12500 + case)
    oz = compute(torch, bb, inp)
    f64 = compute(torch, bb, inp, precision="fp64")
    assert rel(oz, f64) <= 2 * TOL


def test_graph_replay_is_bitwise(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[0]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=12600)
    ctx = bb.bblock_create(L, n_ev, max(nd), "ozaki")
    stream = torch.cuda.Stream()
    outs = [compute(torch, bb, inp, stream=stream, ctx=ctx) for _ in range(4)]
    bb.bblock_destroy(ctx)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert rel(outs[0], reference(inp)) <= TOL
