"""Failure paths, forced on the host side, without faulting the GPU.

* Timeout: a test hook shortens the tensor-core contraction's bounded waits to one
  microsecond, so the first wait runs out. The kernel must raise its abort flag and stop
  early, and `bblock_status` must report BBLOCK_ERR_TIMEOUT, with no hang. The MMA thread
  still waits for its own MMAs before TMEM is freed. The context then runs the same call
  correctly with the default limit.
* Allocation failure: a test hook makes the next device allocation fail. The call reports
  BBLOCK_ERR_OOM and the context recovers on the next call.
* Invalid sizes: a line with no (or negative, or too many) dilution columns is rejected
  before any launch.
* Workspace canaries (checks option): in every form the canaries after the fields, the
  converted inputs and the partial blocks stay intact. A test hook overwrites one from the
  host, in stream order and inside the library's own workspace, so no kernel misbehaves;
  the check kernel must report it, and the context must then compute correct blocks.
"""
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


def _case(torch):
    inp = workloads.custom(6, 16, (16, 12, 16), 2, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7], seed=5100)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    ref = np.stack([oracle.bblock(6, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                  inp.momenta, inp.spins, inp.coeffs) for t in range(2)])
    return inp, V, phis, ref


@pytest.mark.parametrize("precision,products", [("bf16", 6), ("tf32x3", 6)])
def test_wait_timeout_is_reported_and_the_context_recovers(env, precision, products):
    torch, bb = env
    inp, V, phis, ref = _case(torch)
    ctx = bb.bblock_create(6, 16, 16, precision, bf16_products=products)
    bb.bblock_set_option(ctx, "wait_limit_us", 1)
    assert bb.bblock_get_option(ctx, "wait_limit_us") == 1
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    with pytest.raises(bb.BblockError, match="TIMEOUT"):
        bb.bblock_status(ctx)
    bb.bblock_set_option(ctx, "wait_limit_us", 0)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)                     # the status word was cleared when reported
    assert rel(B.cpu().numpy(), ref) <= 1e-6
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("df64", 1e-12), ("bf16", 1e-6)])
def test_forced_allocation_failure_reports_oom_and_the_context_recovers(env, precision, tol):
    torch, bb = env
    inp, V, phis, ref = _case(torch)
    ctx = bb.bblock_create(6, 16, 16, precision)
    bb.bblock_set_option(ctx, "fail_next_alloc", 1)
    with pytest.raises(bb.BblockError, match="OOM"):
        bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    assert "forced" in bb.bblock_last_error(ctx)
    assert bb.bblock_get_option(ctx, "fail_next_alloc") == 0    # fires once
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), ref) <= tol
    bb.bblock_destroy(ctx)


def test_a_line_without_dilution_columns_is_rejected(env):
    torch, bb = env
    inp, V, phis, ref = _case(torch)
    ctx = bb.bblock_create(6, 16, 16, "fp64")
    lib = bb.load()
    mom = np.ascontiguousarray(inp.momenta, np.int32)
    sp = np.ascontiguousarray(inp.spins, np.int32)
    cf = np.ascontiguousarray(inp.coeffs, np.complex128)
    out = torch.zeros(1 << 16, dtype=torch.complex128, device="cuda:0")
    for nds in ((16, 12, 0), (0, 12, 16), (16, -3, 16), (17, 12, 16)):   # 17 > max_ndil
        rc = lib.bblock_compute(ctx.handle, 2, V.data_ptr(), phis[0].data_ptr(), phis[1].data_ptr(),
                                phis[2].data_ptr(), *nds, mom.ctypes.data, mom.shape[0],
                                sp.ctypes.data, cf.ctypes.data, sp.shape[0], 0, out.data_ptr(), None)
        assert rc == -1 and "max_ndil" in bb.bblock_last_error(ctx), nds
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), ref) <= 1e-12
    bb.bblock_destroy(ctx)


FORMS = [("fp64", 6, 1e-12), ("df64", 6, 1e-12), ("bf16", 6, 1e-6), ("tf32x3", 6, 1e-6),
         ("bf16", 3, 1e-4), ("fp16x3", 6, 1e-6)]


@pytest.mark.parametrize("form", range(len(FORMS)))
def test_workspace_canaries_stay_intact(env, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    inp, V, phis, ref = _case(torch)
    ctx = bb.bblock_create(6, 16, 16, precision, bf16_products=products)
    bb.bblock_set_option(ctx, "checks", 1)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), ref) <= tol
    assert bb.bblock_last_launch_count(ctx) >= 2          # fill and check launches included
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_an_overwritten_canary_is_reported(env, precision):
    torch, bb = env
    inp, V, phis, ref = _case(torch)
    ctx = bb.bblock_create(6, 16, 16, precision)
    bb.bblock_set_option(ctx, "checks", 1)
    bb.bblock_set_option(ctx, "corrupt_canary", 1)
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    with pytest.raises(bb.BblockError, match="DEVICE_FLAG"):
        bb.bblock_status(ctx)
    assert "canary" in bb.bblock_last_error(ctx)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy(), ref) <= (1e-12 if precision == "fp64" else 1e-6)
    bb.bblock_destroy(ctx)
