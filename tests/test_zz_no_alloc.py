"""The allocation-free contraction entry point gives the blocks of the regular one.

``bblock_contract_noalloc`` is for callers that must not allocate device memory (an
application whose memory manager has already reserved the device, or a hot loop where
cudaMalloc/cudaFree and their device-wide synchronisation are not allowed). Its partial
sums live in a fixed device array shared by all calls, so this test makes two calls in
a row, on different shapes, and checks each against ``bblock_compute`` through the C ABI.
It sits in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12


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
    # L, n_ev, (nd1, nd2, nd3), momenta, spin triples, coefficients
    (4, 10, (9, 7, 11), [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7071, -0.7071, 0.7071]),
    (5, 12, (16, 16, 33), [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 2)],
     [(0, 1, 0), (1, 0, 0), (2, 3, 2), (3, 2, 2), (0, 1, 3)], [0.5, -0.5, 0.5, -0.5, 0.25j]),
]


def regular_entry_point(torch, bb, case, seed):
    """Blocks from bblock_compute (context workspace) and the fields the other entry
    point takes: q_i[alpha][x][a][d] reconstructed on the CPU (Eq. 2)."""
    L, n_ev, nd, mom, spins, coeffs = case
    inp = workloads.custom(L, n_ev, nd, 1, mom, spins, coeffs, seed=seed)
    dev = torch.device("cuda:0")
    phis = [inp.phi[0][i] for i in range(3)]
    ctx = bb.bblock_create(L, n_ev, max(nd), "fp64")
    B_ref = bb.bblock_compute(ctx, torch.from_numpy(inp.V).to(dev),
                              *[torch.from_numpy(p).to(dev) for p in phis],
                              inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    bb.bblock_destroy(ctx)
    qs = [torch.from_numpy(oracle.reconstruct_all(inp.V[0], p[0])).to(dev) for p in phis]
    return inp, qs, B_ref.cpu().numpy()[0]


def test_two_calls_in_a_row_match_the_regular_entry_point(env):
    torch, bb = env
    dev = torch.device("cuda:0")
    prepared = [regular_entry_point(torch, bb, case, seed=500 + k) for k, case in enumerate(CASES)]
    outs = []
    for (inp, qs, _), case in zip(prepared, CASES):       # two calls back to back
        L, _, nd, mom, _, _ = case
        B = torch.full((len(mom), *nd), complex(np.nan, np.nan), dtype=torch.complex128,
                       device=dev)
        bb.bblock_contract_noalloc(L, *qs, inp.momenta, inp.spins, inp.coeffs, B)
        outs.append(B)
    torch.cuda.synchronize()
    for k, ((inp, _, ref), B) in enumerate(zip(prepared, outs)):
        got = B.cpu().numpy()
        assert np.isfinite(got).all(), f"call {k}"
        assert rel(got, ref) <= TOL_FP64, f"call {k}"
        # and against the oracle directly
        ref_o = oracle.bblock(inp.workload.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)],
                              inp.momenta, inp.spins, inp.coeffs)
        assert rel(got, ref_o) <= TOL_FP64, f"call {k}"


def test_request_that_fills_the_static_scratch(env):
    """Shapes whose blocks fill the fixed scratch exactly (one slab of partial sums) or half
    of it (two slabs): the slab count is capped by the scratch, and the blocks still match
    the regular entry point. Two calls in a row again, the larger first."""
    torch, bb = env
    dev = torch.device("cuda:0")
    L, n_ev, nd = 2, 6, (64, 64, 64)
    spins, coeffs = [(0, 1, 0), (1, 0, 2)], [0.6, -0.8j]
    moms = [[(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
             (1, 1, 1)],                                    # 8 * 64^3 * 16 B = 32 MiB
            [(0, 0, 0), (1, 0, 0), (0, 1, 1), (1, 1, 1)]]   # 16 MiB: two slabs fit
    for k, mom in enumerate(moms):
        assert len(mom) * 64 ** 3 * 16 <= 32 * 1024 * 1024
        prepared = regular_entry_point(torch, bb, (L, n_ev, nd, mom, spins, coeffs), seed=600 + k)
        inp, qs, ref = prepared
        B = torch.full((len(mom), *nd), complex(np.nan, np.nan), dtype=torch.complex128,
                       device=dev)
        bb.bblock_contract_noalloc(L, *qs, inp.momenta, inp.spins, inp.coeffs, B)
        torch.cuda.synchronize()
        got = B.cpu().numpy()
        assert np.isfinite(got).all(), f"case {k}"
        assert rel(got, ref) <= TOL_FP64, f"case {k}"
        # and against the oracle directly, on sampled entries
        d = [0, 31, 63]
        ref_o = oracle.bblock_sampled(L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)],
                                      inp.momenta, inp.spins, inp.coeffs, d, d, d)
        assert rel(got[:, d][:, :, d][:, :, :, d], ref_o) <= TOL_FP64, f"case {k}"


def test_requests_beyond_the_static_scratch_are_rejected(env):
    torch, bb = env
    dev = torch.device("cuda:0")
    L, nd = 1, 128
    q = torch.zeros((4, 1, 3, nd), dtype=torch.complex128, device=dev)
    mom = [(0, 0, 0)] * 2                     # 2 * 128^3 * 16 bytes = 64 MiB > 32 MiB
    B = torch.zeros((2, nd, nd, nd), dtype=torch.complex128, device=dev)
    with pytest.raises(bb.BblockError, match="TOO_LARGE"):
        bb.bblock_contract_noalloc(L, q, q, q, mom, [(0, 0, 0)], [1.0], B)
    q4 = torch.zeros((4, 1, 3, 2), dtype=torch.complex128, device=dev)
    B9 = torch.zeros((9, 2, 2, 2), dtype=torch.complex128, device=dev)
    with pytest.raises(bb.BblockError, match="TOO_LARGE"):
        bb.bblock_contract_noalloc(L, q4, q4, q4, [(0, 0, 0)] * 9, [(0, 0, 0)], [1.0], B9)
