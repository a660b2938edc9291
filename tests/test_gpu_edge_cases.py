"""Edge cases at the limits of the interface, in every form, against the oracle.

* The largest dilution size a context accepts (nd = 256 = max_ndil) on a two-site-per-axis
  lattice: the largest tiles and the most N tiles per unit.
* The largest eigenvector count (N_ev = 3 L^3: V is a full orthonormal basis).
* One lattice site (L = 1): a single slab of a single site.
* One dilution column per line (nd = 1): every tile is a ragged tail.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = [("fp64", 6, 1e-12), ("df64", 6, 1e-12), ("bf16", 6, 1e-6), ("tf32x3", 6, 1e-6),
         ("bf16", 9, 1e-6), ("fp16x3", 6, 1e-6), ("ozaki", 6, 1e-12)]
IDS = ["fp64", "df64", "bf16x6", "tf32x3", "bf16x9", "fp16x3", "ozaki"]


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


def run(torch, bb, inp, form, max_nd=None):
    precision, products, _ = FORMS[form]
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ctx = bb.bblock_create(w.L, w.n_ev, max_nd or max(inp.ndil[0]), precision,
                           bf16_products=products)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    bb.bblock_destroy(ctx)
    return out


def reference(inp):
    w = inp.workload
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, inp.coeffs)
                     for t in range(inp.V.shape[0])])


@pytest.fixture(scope="module")
def max_dilution():
    inp = workloads.custom(2, 4, (256, 256, 256), 1, [(0, 0, 0), (1, 0, 1)],
                           [(0, 1, 0), (1, 0, 2)], [0.6, -0.8j], seed=7000)
    return inp, reference(inp)


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_largest_dilution_size(env, max_dilution, form):
    torch, bb = env
    inp, ref = max_dilution
    got = run(torch, bb, inp, form, max_nd=256)
    assert rel(got, ref) <= FORMS[form][2]


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_full_eigenvector_basis(env, form):
    torch, bb = env
    inp = workloads.custom(2, 24, (7, 9, 5), 2, [(0, 0, 0), (1, 1, 0)],
                           [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7], seed=7100)
    assert rel(run(torch, bb, inp, form), reference(inp)) <= FORMS[form][2]


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_single_site_lattice(env, form):
    torch, bb = env
    inp = workloads.custom(1, 3, (5, 4, 6), 2, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (2, 3, 1)], [1.0, 0.5j], seed=7200)
    assert rel(run(torch, bb, inp, form), reference(inp)) <= FORMS[form][2]


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_single_column_lines(env, form):
    torch, bb = env
    inp = workloads.custom(3, 6, (1, 1, 1), 3, [(0, 0, 0), (0, 1, 0), (1, 1, 1)],
                           [(0, 1, 0), (1, 0, 0), (3, 2, 1)], [0.5, -0.5, 1.0], seed=7300)
    assert rel(run(torch, bb, inp, form), reference(inp)) <= FORMS[form][2]
