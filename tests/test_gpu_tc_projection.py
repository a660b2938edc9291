"""The projection (Eq. 2) on the tensor cores (BBLOCK_OPT_TC_PROJECTION = 1), through the C ABI.

In this mode the mixed forms split V and the coefficient-folded phi columns into the form's
BF16 or TF32 pieces and accumulate them as the contraction does. Checked against the oracle
on shapes that exercise its edges:

* odd L, so that V's rows (3 L^3) are odd in number and its row segments start off a
  16-byte boundary;
* dilution sizes that are not multiples of the N tile;
* N_ev that is not a multiple of the stage depth (48 BF16 or 24 TF32 eigenvectors);
* line-3 fields folding several gamma spins, and per-momentum coefficient sets.

Replays of a captured graph must be bitwise equal, and switching the option must not replay
a graph captured with the other projection.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

# (precision, products, tolerance): the TF32 and 2-piece projections add their own rounding
FORMS = [("bf16", 6, 1e-6), ("bf16", 9, 1e-6), ("tf32x3", 3, 2e-6), ("bf16", 3, 1e-4)]
FORM_IDS = ["bf16x6", "bf16x9", "tf32x3", "bf16x3"]

CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    (5, 50, (12, 11, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (0, 1, 3)],
     [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2), 0.25j]),
    (4, 60, (33, 20, 17), 1, [(0, 0, 0), (-1, 2, 1)],
     [(1, 2, 3), (0, 1, 3), (1, 2, 0)], [0.3 - 0.2j, 1.0, -0.5]),
    (3, 27, (8, 9, 10), 3, [(0, 0, 0), (0, 1, 1)], [(0, 1, 0), (1, 0, 2)], [0.5, -0.5]),
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


def device_inputs(torch, inp):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(inp.V).to(dev),
            [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)])


def reference(inp, coeffs=None):
    w = inp.workload
    c = inp.coeffs if coeffs is None else coeffs
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, c) for t in range(inp.V.shape[0])])


@pytest.mark.parametrize("form", range(len(FORMS)), ids=FORM_IDS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_tensor_core_projection_matches_oracle(env, case, form):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    precision, products, tol = FORMS[form]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9000 + case)
    V, phis = device_inputs(torch, inp)
    ctx = bb.bblock_create(L, n_ev, max(nd), precision, bf16_products=products)
    bb.bblock_set_option(ctx, "tc_projection", 1)
    assert bb.bblock_get_option(ctx, "tc_projection") == 1
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), reference(inp)) <= tol
    bb.bblock_destroy(ctx)


def test_tensor_core_projection_with_per_momentum_coefficients(env):
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, _ = CASES[0]
    coeffs = np.array([[0.5, -0.5, 0.5j, 0.1], [1.0, 0.2, -0.3, 0.0], [0.0, 1.0j, 0.5, -0.5]])
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs[0], seed=9100)
    V, phis = device_inputs(torch, inp)
    ctx = bb.bblock_create(L, n_ev, max(nd), "bf16", bf16_products=6)
    bb.bblock_set_option(ctx, "tc_projection", 1)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), reference(inp, coeffs)) <= 1e-6
    bb.bblock_destroy(ctx)


def test_graph_replay_and_switching_the_projection(env):
    """Four identical calls (plain, captured, replayed twice) are bitwise equal; after the
    option changes, the next call runs the FP32 projection (a different rounding), not the
    graph captured with the tensor-core one."""
    torch, bb = env
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[1]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=9200)
    V, phis = device_inputs(torch, inp)
    dev = torch.device("cuda:0")
    ctx = bb.bblock_create(L, n_ev, max(nd), "bf16", bf16_products=6)
    bb.bblock_set_option(ctx, "tc_projection", 1)
    stream = torch.cuda.Stream()
    B = torch.empty((n_t, len(mom), *nd), dtype=torch.complex128, device=dev)
    outs = []
    for _ in range(4):
        bb.bblock_compute(ctx, V, *phis, mom, spins, coeffs, B_out=B, stream=stream)
        bb.bblock_status(ctx)
        outs.append(B.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    bb.bblock_set_option(ctx, "tc_projection", 2)
    bb.bblock_compute(ctx, V, *phis, mom, spins, coeffs, B_out=B, stream=stream)
    bb.bblock_status(ctx)
    fp32 = B.cpu().numpy()
    assert not np.array_equal(fp32, outs[0])
    ref = reference(inp)
    assert rel(fp32, ref) <= 1e-6 and rel(outs[0], ref) <= 1e-6
    with pytest.raises(bb.BblockError):
        bb.bblock_set_option(ctx, "tc_projection", 3)
    bb.bblock_destroy(ctx)
