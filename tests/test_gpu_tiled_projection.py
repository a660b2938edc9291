"""The tiled tensor-core projection (Eq. 2; BBLOCK_OPT_TC_PROJECTION = 0, the default), through
the C ABI.

V (once per distinct V of a wave) and every field's coefficient-folded phi are split into
three BF16 pieces (exact for FP32) and written in the MMA's core-matrix layout; the
projection kernel stages them with bulk copies and sums the six piece products i + j <= 2
on the tensor cores. Its fields feed every mixed contraction, so the blocks must meet each
form's parity target against the oracle on shapes at the projection's edges:

* odd L (3 L^3 rows, the last 128-row tile ragged);
* N_ev not a multiple of the 32-deep K stage;
* dilution sizes that are not multiples of 16 and above the 64-column N tile;
* line-3 fields folding several gamma spins, and per-momentum coefficient sets;
* a batch whose jobs share V (one tile set per distinct V) and whose dilution sizes differ.

It must also agree with the FP32 projection to the forms' rounding and replay bitwise from a
CUDA graph.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = [("bf16", 6, 1e-6), ("bf16", 9, 1e-6), ("tf32x3", 3, 1e-6), ("bf16", 3, 1e-4),
         ("fp16x3", 6, 1e-6)]
FORM_IDS = ["bf16x6", "bf16x9", "tf32x3", "bf16x3", "fp16x3"]

CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    (5, 50, (12, 11, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (0, 1, 3)],
     [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2), 0.25j]),
    (4, 60, (33, 20, 70), 1, [(0, 0, 0), (-1, 2, 1)],
     [(1, 2, 3), (0, 1, 3), (1, 2, 0)], [0.3 - 0.2j, 1.0, -0.5]),
    (3, 27, (8, 9, 10), 3, [(0, 0, 0), (0, 1, 1)], [(0, 1, 0), (1, 0, 2)], [0.5, -0.5]),
    # the batched workload's momenta and spins at a small L
    (6, 40, (16, 16, 16), 1, [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1),
                             (0, 0, -1), (1, 1, 0), (-1, -1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
]


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


def reference(inp, coeffs=None):
    w = inp.workload
    c = inp.coeffs if coeffs is None else coeffs
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, c) for t in range(inp.V.shape[0])])


def run(torch, bb, inp, form, proj, coeffs=None, stream=None, ctx=None):
    precision, products, _ = FORMS[form]
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), precision, bf16_products=products)
        bb.bblock_set_option(ctx, "tc_projection", proj)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins,
                          inp.coeffs if coeffs is None else coeffs, stream=stream)
    bb.bblock_status(ctx)
    if own:
        bb.bblock_destroy(ctx)
    return B.cpu().numpy()


@pytest.mark.parametrize("form", range(len(FORMS)), ids=FORM_IDS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tiled_projection_matches_oracle(env, case, form):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=13000 + case)
    got = run(torch, bb, inp, form, 0)
    ref = reference(inp)
    err = rel(got, ref)
    fp32 = run(torch, bb, inp, form, 2)
    print(f"{FORM_IDS[form]} case {case}: tiled projection {err:.3e}, FP32 projection "
          f"{rel(fp32, ref):.3e}, difference {rel(got, fp32):.3e}")
    assert np.all(np.isfinite(got)) and err <= FORMS[form][2]


def test_per_momentum_coefficients(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, _ = CASES[0]
    coeffs = np.array([[0.5, -0.5, 0.5j, 0.1], [1.0, 0.2, -0.3, 0.0], [0.0, 1.0j, 0.5, -0.5]])
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs[0], seed=13100)
    got = run(torch, bb, inp, 0, 0, coeffs=coeffs)
    assert rel(got, reference(inp, coeffs)) <= 1e-6


def test_batch_sharing_v_with_uneven_dilution(env):
    """Jobs of several noise triples per time slice share V: one tile set per distinct V."""
    torch, bb = env
    dev = torch.device("cuda:0")
    L, n_ev = 5, 36
    mom = [(0, 0, 0), (1, 0, 0), (0, 1, 1)]
    spins, coeffs = [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7]
    rng = np.random.Generator(np.random.PCG64(13200))
    Vs = [workloads.eigenvectors(rng, L, n_ev) for _ in range(2)]
    dVs = [torch.from_numpy(V).to(dev) for V in Vs]
    jobs, host = [], []
    for t in range(2):
        for nd in [(8, 8, 8), (20, 17, 12), (33, 30, 40)]:
            ph = [workloads.coefficients(rng, n_ev, d) for d in nd]
            host.append((Vs[t], ph))
            B = torch.zeros((len(mom), *nd), dtype=torch.complex128, device=dev)
            jobs.append((dVs[t], *[torch.from_numpy(p).to(dev) for p in ph], B))
    for form in (0, 4):
        precision, products, tol = FORMS[form]
        ctx = bb.bblock_create(L, n_ev, 40, precision, bf16_products=products)
        assert bb.bblock_get_option(ctx, "tc_projection") == 0
        bb.bblock_compute_batch(ctx, jobs, mom, spins, coeffs)
        bb.bblock_status(ctx)
        for (V, ph), job in zip(host, jobs):
            ref = oracle.bblock(L, V, *ph, mom, spins, coeffs)
            assert rel(job[4].cpu().numpy(), ref) <= tol
        bb.bblock_destroy(ctx)


def test_graph_replay_is_bitwise(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[1]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=13300)
    ctx = bb.bblock_create(L, n_ev, max(nd), "fp16x3")
    stream = torch.cuda.Stream()
    outs = [run(torch, bb, inp, 4, 0, stream=stream, ctx=ctx) for _ in range(4)]
    bb.bblock_destroy(ctx)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert rel(outs[0], reference(inp)) <= 1e-6
