"""GPU parity of the tensor-core forms (tcgen05, split operands, FP32 accumulation) against
the CPU FP64 oracle, through the C ABI.

Tolerances (relative Frobenius error of the whole block set):
  * BF16 split with 6 or 9 piece products, TF32 split with 3, FP16 split with 3 (operands
    scaled into FP16's range by powers of two): <= 1e-6;
  * BF16 split with 3 piece products: <= 1e-4 (the dropped products are ~3 * 2^-16
    relative, so this form is reported, not claimed at 1e-6).
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = [("bf16", 6, 1e-6), ("bf16", 9, 1e-6), ("tf32x3", 6, 1e-6), ("bf16", 3, 1e-4),
         ("fp16x3", 6, 1e-6)]
FORM_IDS = ["bf16x6", "bf16x9", "tf32x3", "bf16x3", "fp16x3"]


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


def gpu_blocks(torch, bb, inp, precision, products, coeffs=None, ctx=None):
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max(inp.ndil[0]), precision, bf16_products=products)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins,
                          inp.coeffs if coeffs is None else coeffs)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    if own:
        bb.bblock_destroy(ctx)
    return out


def oracle_blocks(inp, coeffs=None):
    w = inp.workload
    c = inp.coeffs if coeffs is None else coeffs
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, c) for t in range(inp.V.shape[0])])


CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    (4, 8, (8, 8, 8), 1, [(0, 0, 0)], [(0, 0, 0)], [1.0]),
    (5, 12, (12, 11, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [1 / math.sqrt(2), -1 / math.sqrt(2), 1 / math.sqrt(2)]),
    (6, 16, (16, 16, 16), 1, [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
    (3, 9, (20, 7, 5), 1, [(0, 0, 0), (-1, 2, 1)], [(1, 2, 3), (0, 1, 3)], [0.3 - 0.2j, 1.0]),
]


@pytest.mark.parametrize("form", range(len(FORMS)), ids=FORM_IDS)
@pytest.mark.parametrize("case", range(len(CASES)))
def test_small_shapes_against_oracle(env, form, case):
    torch, bb = env
    precision, products, tol = FORMS[form]
    L, n_ev, nd, n_t, mom, spins, coeffs = CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=2000 + case)
    got = gpu_blocks(torch, bb, inp, precision, products)
    err = rel(got, oracle_blocks(inp))
    print(f"{FORM_IDS[form]} case {case}: rel. Frobenius error {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("form", [0, 2, 4], ids=["bf16x6", "tf32x3", "fp16x3"])
def test_momentum_dependent_coefficients(env, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    rng = np.random.default_rng(3)
    coeffs = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    inp = workloads.custom(4, 10, (9, 8, 7), 2, mom, spins, np.ones(3), seed=2100)
    got = gpu_blocks(torch, bb, inp, precision, products, coeffs=coeffs)
    assert rel(got, oracle_blocks(inp, coeffs=coeffs)) <= tol


def test_bitwise_deterministic(env):
    torch, bb = env
    inp = workloads.custom(5, 12, (12, 12, 12), 2, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (1, 0, 0)], [0.5, -0.5], seed=2200)
    ctx = bb.bblock_create(5, 12, 12, "bf16", bf16_products=6)
    a = gpu_blocks(torch, bb, inp, "bf16", 6, ctx=ctx)
    b = gpu_blocks(torch, bb, inp, "bf16", 6, ctx=ctx)
    assert np.array_equal(a, b)
    bb.bblock_destroy(ctx)


def test_batch_with_uneven_dilution(env):
    torch, bb = env
    dev = torch.device("cuda:0")
    L, n_ev = 4, 10
    mom = [(0, 0, 0), (1, 0, 0), (0, 1, 1)]
    spins, coeffs = [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.5, -0.5, 0.7]
    rng = np.random.Generator(np.random.PCG64(2300))
    jobs, host = [], []
    for nd in [(8, 8, 8), (12, 12, 12), (16, 16, 16), (8, 8, 8)]:
        V = workloads.eigenvectors(rng, L, n_ev)
        ph = [workloads.coefficients(rng, n_ev, d) for d in nd]
        host.append((V, ph))
        B = torch.zeros((len(mom), *nd), dtype=torch.complex128, device=dev)
        jobs.append((torch.from_numpy(V).to(dev), *[torch.from_numpy(p).to(dev) for p in ph], B))
    ctx = bb.bblock_create(L, n_ev, 16, "bf16", bf16_products=6)
    bb.bblock_compute_batch(ctx, jobs, mom, spins, coeffs)
    bb.bblock_status(ctx)
    for (V, ph), job in zip(host, jobs):
        ref = oracle.bblock(L, V, *ph, mom, spins, coeffs)
        assert rel(job[4].cpu().numpy(), ref) <= 1e-6
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("form", [0, 2, 3, 4], ids=["bf16x6", "tf32x3", "bf16x3", "fp16x3"])
def test_l24_nev96_ndil32_sampled(env, form):
    """The benchmarked workload at full size in the mixed forms: sampled entries vs oracle."""
    torch, bb = env
    precision, products, tol = FORMS[form]
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w)
    got = gpu_blocks(torch, bb, inp, precision, products)
    d1s, d2s, d3s = [0, 13, 31], [5, 31], [0, 30, 31]
    for t in (0, 7):
        ref = oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                    inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
        sub = got[t][:, d1s][:, :, d2s][:, :, :, d3s]
        err = rel(sub, ref)
        print(f"{FORM_IDS[form]} L=24 t={t}: sampled rel. error {err:.3e}")
        assert err <= tol


@pytest.mark.parametrize("scales", [(2.0 ** 40, 2.0 ** -30, 2.0 ** 20),
                                    (2.0 ** -50, 2.0 ** -45, 2.0 ** -40),
                                    (1e20, 1e15, 1e-20)], ids=["mixed", "tiny", "wide"])
def test_fp16_form_scales_operands_into_range(env, scales):
    """The FP16 form holds 1e-6 whatever the magnitude of the inputs. Each quark line's
    coefficients are scaled by a factor far outside FP16's range (largest finite 65504,
    smallest normal 2^-14); the blocks must be the oracle's blocks of the scaled inputs,
    because the operands are brought into range by powers of two chosen per job."""
    torch, bb = env
    inp = workloads.custom(5, 12, (12, 11, 13), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
                           [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7], seed=2400)
    for i in range(3):
        inp.phi[0][i] *= scales[i]
    got = gpu_blocks(torch, bb, inp, "fp16x3", 6)
    ref = oracle_blocks(inp)
    err = rel(got, ref)
    print(f"fp16x3 scales {scales}: rel. Frobenius error {err:.3e}")
    assert np.all(np.isfinite(got)) and err <= 1e-6


def test_fp16_form_zero_line_gives_zero_blocks(env):
    """A quark line that is identically zero has no largest entry to scale by: the blocks
    are exactly zero, not NaN."""
    torch, bb = env
    inp = workloads.custom(4, 8, (8, 9, 10), 1, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (1, 0, 0)], [0.5, -0.5], seed=2500)
    inp.phi[0][2][:] = 0.0
    got = gpu_blocks(torch, bb, inp, "fp16x3", 6)
    assert np.array_equal(got, np.zeros_like(got))
