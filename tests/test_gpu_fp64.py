"""GPU parity of the FP64-accurate forms against the CPU FP64 oracle (relative Frobenius
<= 1e-12): the FP64 form (IEEE double on the FP64 pipe) and the double-float form (pairs of
FP32 on the FP32 pipe). The parity tests run for both forms; the tests of host logic
(argument checks, empty calls, the host-buffer entry point) use the FP64 form.

All calls go through the C ABI (``paper_2211_16278_gb300.bblock``). Inputs are
seeded synthetic draws from ``workloads``; expected values come from ``oracle``.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(params=["fp64", "df64"])
def form(request):
    return request.param


@pytest.fixture(scope="module")
def bb(torch_cuda):
    import paper_2211_16278_gb300 as pkg
    pkg.load()
    return pkg


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def run_gpu(bb, torch, inp, precision="fp64", noise=0, ctx=None, coeffs=None):
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[noise][i]).to(dev) for i in range(3)]
    max_nd = max(inp.ndil[noise])
    own = ctx is None
    if own:
        ctx = bb.bblock_create(w.L, w.n_ev, max_nd, precision)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins,
                          inp.coeffs if coeffs is None else coeffs)
    bb.bblock_status(ctx)
    out = B.cpu().numpy()
    if own:
        bb.bblock_destroy(ctx)
    return out


def oracle_blocks(inp, noise=0, coeffs=None):
    w = inp.workload
    c = inp.coeffs if coeffs is None else coeffs
    return np.stack([oracle.bblock(w.L, inp.V[t], *[inp.phi[noise][i][t] for i in range(3)],
                                   inp.momenta, inp.spins, c) for t in range(inp.V.shape[0])])


def test_l4_nev8_ndil8_full(bb, torch_cuda, form):
    inp = workloads.generate(workloads.WORKLOADS["l4_nev8_ndil8"])
    got = run_gpu(bb, torch_cuda, inp, form)
    ref = oracle_blocks(inp)
    assert got.shape == ref.shape == (1, 1, 8, 8, 8)
    assert rel(got, ref) <= TOL_FP64


RAGGED_CASES = [
    # L, n_ev, (nd1, nd2, nd3), n_t, momenta, spins, coeffs
    (3, 7, (5, 3, 7), 2, [(0, 0, 0), (1, 0, 0), (-1, 2, 0), (1, 1, 1)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (0, 1, 3)], [0.5, -0.5, 0.5j, 0.25 - 0.1j]),
    (5, 20, (9, 7, 37), 1, [(0, 0, 0), (2, -1, 0)], [(3, 2, 1)], [1.0]),
    (2, 24, (33, 2, 1), 3, [(0, 0, 0)], [(0, 0, 0), (1, 1, 1)], [1.0, -1.0]),
    (1, 3, (1, 1, 1), 1, [(0, 0, 0), (1, 0, 0)], [(0, 1, 2)], [1.0]),
    (4, 9, (17, 16, 33), 1, [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2)], [0.5, -0.5, 0.5, -0.5]),
]


@pytest.mark.parametrize("case", range(len(RAGGED_CASES)))
def test_ragged_small_shapes(bb, torch_cuda, case, form):
    L, n_ev, nd, n_t, mom, spins, coeffs = RAGGED_CASES[case]
    inp = workloads.custom(L, n_ev, nd, n_t, mom, spins, coeffs, seed=1000 + case)
    got = run_gpu(bb, torch_cuda, inp, form)
    ref = oracle_blocks(inp)
    assert rel(got, ref) <= TOL_FP64


def test_many_momenta_use_several_launch_groups(bb, torch_cuda, form):
    mom = [(a, b, c) for a in (-1, 0, 1) for b in (0, 1) for c in (0, 1)][:11]
    inp = workloads.custom(3, 6, (4, 5, 6), 1, mom, [(0, 1, 0), (2, 2, 3)], [1.0, -0.5j], seed=7)
    assert rel(run_gpu(bb, torch_cuda, inp, form), oracle_blocks(inp)) <= TOL_FP64


def test_momentum_dependent_spin_coefficients(bb, torch_cuda, form):
    mom = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    rng = np.random.default_rng(3)
    coeffs = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    inp = workloads.custom(3, 8, (6, 5, 7), 2, mom, spins, np.ones(3), seed=8)
    got = run_gpu(bb, torch_cuda, inp, form, coeffs=coeffs)
    assert rel(got, oracle_blocks(inp, coeffs=coeffs)) <= TOL_FP64


def test_all_sixteen_spin_pairs(bb, torch_cuda, form):
    spins = [(a, b, (a + b) % 4) for a in range(4) for b in range(4)]
    coeffs = [complex(math.cos(k), math.sin(k)) for k in range(16)]
    inp = workloads.custom(2, 5, (3, 4, 5), 1, [(0, 0, 0), (1, 0, 1)], spins, coeffs, seed=9)
    assert rel(run_gpu(bb, torch_cuda, inp, form), oracle_blocks(inp)) <= TOL_FP64


def test_repeated_triples_fold_into_one_field(bb, torch_cuda, form):
    spins = [(0, 1, 2), (0, 1, 2), (0, 1, 3), (0, 1, 0), (0, 1, 1)]
    coeffs = [0.25, 0.25, -1.0, 0.5j, 2.0]
    inp = workloads.custom(3, 6, (4, 4, 4), 1, [(0, 0, 0), (0, 1, 0)], spins, coeffs, seed=10)
    assert rel(run_gpu(bb, torch_cuda, inp, form), oracle_blocks(inp)) <= TOL_FP64


def test_deterministic_across_runs(bb, torch_cuda, form):
    inp = workloads.custom(4, 10, (8, 8, 8), 2, [(0, 0, 0), (1, 0, 0)], [(0, 1, 0)], [1.0], seed=11)
    torch = torch_cuda
    ctx = bb.bblock_create(4, 10, 8, form)
    a = run_gpu(bb, torch, inp, form, ctx=ctx)
    b = run_gpu(bb, torch, inp, form, ctx=ctx)
    assert np.array_equal(a, b)
    bb.bblock_destroy(ctx)


def test_empty_run_is_a_noop(bb, torch_cuda):
    torch = torch_cuda
    ctx = bb.bblock_create(2, 4, 4, "fp64")
    dev = torch.device("cuda:0")
    V = torch.zeros((0, 4, 8, 3), dtype=torch.complex128, device=dev)
    phi = torch.zeros((0, 16, 4), dtype=torch.complex128, device=dev)
    B = bb.bblock_compute(ctx, V, phi, phi, phi, [(0, 0, 0)], [(0, 0, 0)], [1.0])
    assert B.shape == (0, 1, 4, 4, 4)
    assert bb.bblock_last_launch_count(ctx) == 0
    V1 = torch.zeros((1, 4, 8, 3), dtype=torch.complex128, device=dev)
    phi1 = torch.zeros((1, 16, 4), dtype=torch.complex128, device=dev)
    B = bb.bblock_compute(ctx, V1, phi1, phi1, phi1, np.zeros((0, 3)), [(0, 0, 0)], [1.0])
    assert B.shape == (1, 0, 4, 4, 4)
    bb.bblock_status(ctx)
    bb.bblock_destroy(ctx)


def test_host_entry_point_matches_device_entry_point(bb, torch_cuda):
    inp = workloads.custom(3, 7, (6, 5, 4), 2, [(0, 0, 0), (1, 1, 0)], [(0, 1, 0), (1, 0, 0)],
                           [0.5, -0.5], seed=12)
    dev_out = run_gpu(bb, torch_cuda, inp)
    ctx = bb.bblock_create(3, 7, 6, "fp64")
    B = np.zeros((2, 2, 6, 5, 4), np.complex128)
    bb.bblock_compute_host(ctx, inp.V, *[inp.phi[0][i] for i in range(3)], inp.momenta,
                           inp.spins, inp.coeffs, B)
    assert np.array_equal(B, dev_out)
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("n_t", [3, 11])
@pytest.mark.parametrize("precision", ["fp64", "df64", "bf16"])
def test_host_entry_point_in_uneven_chunks(bb, torch_cuda, n_t, precision):
    """The host entry point moves the time slices in up to 8 chunks on its own copy stream:
    11 slices make chunks of 1 and 2, 3 slices one chunk each. A chunk may split its sites
    into other slabs than a call over all slices, so the blocks agree with the device entry
    point and the oracle to the form's tolerance; repeated host calls agree bit for bit.
    Per-momentum coefficients check that each chunk pairs its slices with the right set."""
    mom = [(0, 0, 0), (1, 1, 0), (0, 0, 1)]
    inp = workloads.custom(3, 7, (6, 5, 4), n_t, mom, [(0, 1, 0), (1, 0, 0)], [0.5, -0.5],
                           seed=40 + n_t)
    coeffs = np.array([[0.5, -0.5], [0.3 + 0.1j, 0.7], [-1.0j, 0.25]])
    tol = 1e-6 if precision == "bf16" else 1e-12
    dev_out = run_gpu(bb, torch_cuda, inp, precision=precision, coeffs=coeffs)
    ref = oracle_blocks(inp, coeffs=coeffs)
    ctx = bb.bblock_create(3, 7, 6, precision)
    stream = torch_cuda.cuda.Stream()
    first = None
    for _ in range(3):
        B = np.full((n_t, 3, 6, 5, 4), np.nan, np.complex128)
        bb.bblock_compute_host(ctx, inp.V, *[inp.phi[0][i] for i in range(3)], inp.momenta,
                               inp.spins, coeffs, B, stream)
        for t in range(n_t):
            assert np.linalg.norm(B[t] - ref[t]) <= tol * np.linalg.norm(ref[t])
        assert np.linalg.norm(B - dev_out) <= tol * np.linalg.norm(ref)
        if first is None:
            first = B
        assert np.array_equal(B, first)
    assert bb.bblock_last_launch_count(ctx) > 0
    # one chunk: the same launches as the device call, so the same bits
    bb.bblock_set_option(ctx, "host_chunks", 1)
    B = np.full((n_t, 3, 6, 5, 4), np.nan, np.complex128)
    bb.bblock_compute_host(ctx, inp.V, *[inp.phi[0][i] for i in range(3)], inp.momenta,
                           inp.spins, coeffs, B, stream)
    assert np.array_equal(B, dev_out)
    with pytest.raises(bb.BblockError):
        bb.bblock_set_option(ctx, "host_chunks", 65)
    bb.bblock_destroy(ctx)


def test_batch_with_uneven_dilution_matches_single_calls(bb, torch_cuda, form):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    L, n_ev = 3, 8
    mom = [(0, 0, 0), (1, 0, 0), (0, 1, 1)]
    spins, coeffs = [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.5, -0.5, 0.7]
    rng = np.random.Generator(np.random.PCG64(13))
    jobs, host = [], []
    for t, nd in enumerate([(4, 4, 4), (7, 7, 7), (5, 3, 9), (4, 4, 4)]):
        V = workloads.eigenvectors(rng, L, n_ev)
        ph = [workloads.coefficients(rng, n_ev, d) for d in nd]
        host.append((V, ph))
        B = torch.zeros((len(mom), *nd), dtype=torch.complex128, device=dev)
        jobs.append((torch.from_numpy(V).to(dev), *[torch.from_numpy(p).to(dev) for p in ph], B))
    ctx = bb.bblock_create(L, n_ev, 9, form)
    bb.bblock_compute_batch(ctx, jobs, mom, spins, coeffs)
    bb.bblock_status(ctx)
    for (V, ph), job in zip(host, jobs):
        ref = oracle.bblock(L, V, *ph, mom, spins, coeffs)
        assert rel(job[4].cpu().numpy(), ref) <= TOL_FP64
    bb.bblock_destroy(ctx)


def test_invalid_arguments_are_rejected(bb, torch_cuda):
    torch = torch_cuda
    dev = torch.device("cuda:0")
    ctx = bb.bblock_create(2, 4, 4, "fp64")
    V = torch.zeros((1, 4, 8, 3), dtype=torch.complex128, device=dev)
    phi = torch.zeros((1, 16, 4), dtype=torch.complex128, device=dev)
    with pytest.raises(bb.BblockError, match="INVALID_ARG"):
        bb.bblock_compute(ctx, V, phi, phi, phi, [(0, 0, 0)], [(0, 4, 0)], [1.0])   # spin 4
    big = torch.zeros((1, 16, 5), dtype=torch.complex128, device=dev)
    with pytest.raises(bb.BblockError, match="INVALID_ARG"):
        bb.bblock_compute(ctx, V, big, phi, phi, [(0, 0, 0)], [(0, 0, 0)], [1.0])   # nd > max
    # a host buffer where a device buffer is required
    lib = bb.load()
    import ctypes
    host = np.zeros(1 << 12, np.complex128)
    mom = np.zeros((1, 3), np.int32)
    sp = np.zeros((1, 3), np.int32)
    cf = np.ones(1, np.complex128)
    rc = lib.bblock_compute(ctx.handle, 1, host.ctypes.data, phi.data_ptr(), phi.data_ptr(),
                            phi.data_ptr(), 4, 4, 4, mom.ctypes.data, 1, sp.ctypes.data,
                            cf.ctypes.data, 1, 0, phi.data_ptr(), None)
    assert rc == -1 and "device memory" in bb.bblock_last_error(ctx)
    rc = lib.bblock_compute(ctx.handle, 1, V.data_ptr() + 8, phi.data_ptr(), phi.data_ptr(),
                            phi.data_ptr(), 4, 4, 4, mom.ctypes.data, 1, sp.ctypes.data,
                            cf.ctypes.data, 1, 0, phi.data_ptr(), None)
    assert rc == -1 and "aligned" in bb.bblock_last_error(ctx)
    bb.bblock_status(ctx)
    bb.bblock_destroy(ctx)


# ---------------------------------------------------------------- full-size workload, sampled

def test_l24_nev96_ndil32_sampled_entries(bb, torch_cuda, form):
    """The benchmarked workload (L=24, N_ev=96, N_dil=32, 8 time slices) at full size;
    sampled (t, d1, d2, d3) entries against the oracle, which evaluates them one by one."""
    w = workloads.WORKLOADS["l24_nev96_ndil32"]
    inp = workloads.generate(w)
    got = run_gpu(bb, torch_cuda, inp, form)
    assert got.shape == (8, 3, 32, 32, 32)
    d1s, d2s, d3s = [0, 13, 31], [5, 31], [0, 30, 31]
    for t in (0, 7):
        ref = oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                    inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
        sub = got[t][:, d1s][:, :, d2s][:, :, :, d3s]
        assert rel(sub, ref) <= TOL_FP64


def test_fp64_probe_measures_both_paths(bb, torch_cuda):
    """The FP64 throughput probe returns positive rates for DFMA and the FP64 MMA, within a
    plausible range of a GPU's FP64 capability (0.05-20 TFLOP/s); the FP64 form's roofline
    takes the DFMA rate as its peak."""
    r = bb.bblock_probe_fp64(0)
    print(f"FP64 probe: DFMA {r['dfma_tflops']:.3f} TFLOP/s, DMMA {r['dmma_tflops']:.3f} TFLOP/s")
    for k in ("dfma_tflops", "dmma_tflops"):
        assert 0.05 < r[k] < 20.0, r
