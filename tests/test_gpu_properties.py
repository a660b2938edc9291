"""Properties of Eq. (1)/(3) checked on the GPU at the benchmarked size (L = 24, N_ev = 96,
N_dil = 32, all 8 time slices), where the oracle cannot compute whole blocks.

* Antisymmetry under exchange of quark lines 1 and 2 (the epsilon tensor), with the spin
  labels exchanged as well: B[phi1, phi2, phi3; (a, b, g)]_{d1 d2 d3}
  = -B[phi2, phi1, phi3; (b, a, g)]_{d2 d1 d3}.
* Linearity in line 3: B[.., phi3 + z phi3'] = B[.., phi3] + z B[.., phi3'].
* The degenerate case of equal lines: phi1 = phi2 with alpha = beta in every triple gives
  B_{d d d3} = 0 on the d1 = d2 diagonal.

Tolerances are relative to the largest block entry: 1e-12 for the FP64 and double-float
forms, 5e-6 for the split-BF16 form with 6 products.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

FORMS = [("fp64", 6, 1e-12), ("df64", 6, 1e-12), ("bf16", 6, 5e-6)]
IDS = ["fp64", "df64", "bf16x6"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_16278_gb300 as bb
    bb.load()
    return torch, bb


@pytest.fixture(scope="module")
def inputs(env):
    torch, bb = env
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    return w, inp, V, phis


def blocks(bb, w, form, V, p1, p2, p3, mom, spins, coeffs):
    precision, products, _ = FORMS[form]
    ctx = bb.bblock_create(w.L, w.n_ev, w.ndil, precision, bf16_products=products)
    B = bb.bblock_compute(ctx, V, p1, p2, p3, mom, spins, coeffs)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    bb.bblock_destroy(ctx)
    return out


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_antisymmetry_under_exchange_of_lines_1_and_2(env, inputs, form):
    torch, bb = env
    w, inp, V, phis = inputs
    spins = np.asarray(inp.spins)
    swapped = spins[:, [1, 0, 2]]
    a = blocks(bb, w, form, V, phis[0], phis[1], phis[2], inp.momenta, spins, inp.coeffs)
    b = blocks(bb, w, form, V, phis[1], phis[0], phis[2], inp.momenta, swapped, inp.coeffs)
    b = np.swapaxes(b, 2, 3)                          # [t][p][d2][d1][d3] -> [t][p][d1][d2][d3]
    assert np.abs(a + b).max() <= FORMS[form][2] * np.abs(a).max()


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_linearity_in_line_3(env, inputs, form):
    torch, bb = env
    w, inp, V, phis = inputs
    z = 0.6 - 0.8j
    other = torch.roll(phis[2], shifts=1, dims=2) * 0.5
    mixed = phis[2] + z * other
    a = blocks(bb, w, form, V, phis[0], phis[1], phis[2], inp.momenta, inp.spins, inp.coeffs)
    b = blocks(bb, w, form, V, phis[0], phis[1], other, inp.momenta, inp.spins, inp.coeffs)
    c = blocks(bb, w, form, V, phis[0], phis[1], mixed, inp.momenta, inp.spins, inp.coeffs)
    assert np.abs(c - (a + z * b)).max() <= FORMS[form][2] * np.abs(c).max()


@pytest.mark.parametrize("form", range(len(FORMS)), ids=IDS)
def test_equal_lines_vanish_on_the_diagonal(env, inputs, form):
    torch, bb = env
    w, inp, V, phis = inputs
    spins = [(0, 0, 1), (2, 2, 3), (1, 1, 1)]
    coeffs = [0.5, -0.25j, 1.0]
    B = blocks(bb, w, form, V, phis[0], phis[0], phis[2], inp.momenta, spins, coeffs)
    d = np.arange(w.ndil)
    diag = B[:, :, d, d, :]
    assert np.abs(diag).max() <= FORMS[form][2] * np.abs(B).max()
    assert np.abs(B).max() > 0
