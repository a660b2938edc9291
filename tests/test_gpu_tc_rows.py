"""The FP16 form's row-factored momentum phase, through the C ABI.

The phase of Eq. 1 factorises along the lattice, e^{-i p.x} = w^{n0 x0} w^{n1 x1 + n2 x2}
with w = e^{-2 pi i / L}. The tensor cores sum each lattice row (x1, x2 fixed) against the
third quark times w^{n0 x0} for every distinct n0 of the momenta; the epilogue multiplies
each row's sums by w^{n1 x1 + n2 x2} into one running sum per momentum. These tests compare
it with the CPU oracle for momenta with negative components, components beyond L, several
momenta sharing one n0, pair counts whose groups do not fill a row's last stage, dilution
sizes that do not fill the last tile, and every d3 tile width the tensor memory allows; it
must also agree with the CTA-pair path and replay bitwise from a CUDA graph.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-6
C4_MOM = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
          (1, 1, 0), (-1, -1, 0)]


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
    # the batched workload's 9 momenta (3 distinct n0), 4 pairs: 16 groups per 4-site row
    (4, 10, (12, 11, 13), 2, C4_MOM,
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
    # 3 pairs (a row of 5 sites is 15 groups: the stage is padded), d3 = 20 (ragged tile)
    (5, 12, (16, 9, 20), 1, C4_MOM[:7],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    # components beyond L and negative; 6 momenta sharing two n0 (mod 6)
    (6, 14, (10, 10, 17), 1, [(7, 0, 0), (1, 2, -3), (-5, 4, 1), (1, -1, 8), (0, 3, 3), (6, 1, 1)],
     [(1, 2, 3), (0, 1, 3)], [0.3 - 0.2j, 1.0]),
    # one spin pair (a row of 3 sites is 3 groups of a 16-group stage), 12 momenta
    (3, 9, (8, 8, 33), 1, [(a, b, c) for a in (0, 1) for b in (0, 1, 2) for c in (0, 1)],
     [(0, 0, 0)], [1.0]),
]


def blocks(torch, bb, inp, rows, nc=0, stream=None, ctx=None, cluster=0):
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), "fp16x3")
        bb.bblock_set_option(ctx, "tc_rows", rows)
        bb.bblock_set_option(ctx, "tc_nc", nc)
        bb.bblock_set_option(ctx, "tc_cluster", cluster)
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


def distinct_n0(L, mom):
    return len({m[0] % L for m in mom})


@pytest.mark.parametrize("nc", [0, 16, 32, 48])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("cluster", [1, 0])
def test_rows_match_oracle(env, case, nc, cluster):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    k = distinct_n0(L, mom)
    if nc and (k * nc > 48 or 4 * k * nc + 2 * len(mom) * nc > 512):
        pytest.skip("tile does not fit the row-factored layout")
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9000 + case)
    got = blocks(torch, bb, inp, rows=1, nc=nc, cluster=cluster)
    err = rel(got, oracle_blocks(inp))
    print(f"fp16x3 rows case {case} nc {nc} cluster {cluster}: rel. Frobenius error {err:.3e}")
    assert np.all(np.isfinite(got)) and err <= TOL


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rows_agree_with_pairs(env, case):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9100 + case)
    rows = blocks(torch, bb, inp, rows=1)
    pairs = blocks(torch, bb, inp, rows=2)
    ref = oracle_blocks(inp)
    assert rel(rows, ref) <= TOL and rel(pairs, ref) <= TOL
    assert rel(rows, pairs) <= 2 * TOL


def test_rows_replay_bitwise_from_graph(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[0]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9200)
    ctx = bb.bblock_create(L, n_ev, max(nd), "fp16x3")
    bb.bblock_set_option(ctx, "tc_rows", 1)
    stream = torch.cuda.Stream()
    outs = [blocks(torch, bb, inp, 1, stream=stream, ctx=ctx) for _ in range(4)]
    bb.bblock_destroy(ctx)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert rel(outs[0], oracle_blocks(inp)) <= TOL


def test_rows_batch_uneven_dilution(env):
    """A batch of jobs with different dilution sizes in one row-factored launch."""
    torch, bb = env
    dev = torch.device("cuda:0")
    L, n_ev = 4, 10
    spins, coeffs = [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]
    rng = np.random.Generator(np.random.PCG64(9300))
    jobs, host = [], []
    for nd in [(8, 8, 8), (12, 12, 12), (16, 16, 16), (20, 20, 20)]:
        V = workloads.eigenvectors(rng, L, n_ev)
        ph = [workloads.coefficients(rng, n_ev, d) for d in nd]
        host.append((V, ph))
        B = torch.zeros((len(C4_MOM), *nd), dtype=torch.complex128, device=dev)
        jobs.append((torch.from_numpy(V).to(dev), *[torch.from_numpy(p).to(dev) for p in ph], B))
    ctx = bb.bblock_create(L, n_ev, 20, "fp16x3")
    bb.bblock_set_option(ctx, "tc_rows", 1)
    bb.bblock_compute_batch(ctx, jobs, C4_MOM, spins, coeffs)
    bb.bblock_status(ctx)
    for (V, ph), job in zip(host, jobs):
        ref = oracle.bblock(L, V, *ph, C4_MOM, spins, coeffs)
        assert rel(job[4].cpu().numpy(), ref) <= TOL
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rows_in_clusters_sharing_the_diquark_tile(env, case):
    """Clusters of two CTAs that build half of each diquark tile each and take adjacent d3
    tiles (BBLOCK_OPT_TC_CLUSTER = 2): the same blocks as the plain row-factored CTAs, to the
    form's tolerance, including jobs with an odd number of d3 tiles."""
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9400 + case)
    w = inp.workload
    ctx = bb.bblock_create(w.L, w.n_ev, max(nd), "fp16x3")
    bb.bblock_set_option(ctx, "tc_rows", 1)
    bb.bblock_set_option(ctx, "tc_cluster", 2)
    got = blocks(torch, bb, inp, 1, ctx=ctx)
    assert bb.bblock_last_path(ctx) == "tc_rows_cluster"
    bb.bblock_destroy(ctx)
    ref = oracle_blocks(inp)
    err = rel(got, ref)
    print(f"fp16x3 rows in clusters case {case}: rel. Frobenius error {err:.3e}")
    assert np.all(np.isfinite(got)) and err <= TOL
    plain = blocks(torch, bb, inp, rows=1, cluster=1)
    assert rel(got, plain) <= 2 * TOL
