"""CUDA-graph replay of repeated calls and the tuning options, through the C ABI.

A call repeated with identical arguments is captured as a CUDA graph on its second
occurrence and replayed afterwards; the replayed blocks must be bitwise equal to the plain
launches, and any change of arguments must fall back to plain launches. The tile options
(N tile, drain interval, slab count) change only how the work is cut, so every setting must
stay within the form's tolerance of the oracle.
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


def setup(torch, inp):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(inp.V).to(dev), [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)])


@pytest.mark.parametrize("precision,products", [("fp64", 6), ("df64", 6), ("bf16", 6), ("tf32x3", 6),
                                                ("fp16x3", 6)])
def test_graph_replay_is_bitwise_equal_to_plain_launches(env, precision, products):
    torch, bb = env
    inp = workloads.custom(4, 10, (9, 8, 12), 2, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
                           [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7], seed=3000)
    V, phis = setup(torch, inp)
    plain = bb.bblock_create(4, 10, 12, precision, bf16_products=products)
    bb.bblock_set_option(plain, "graphs", 0)
    ref = bb.bblock_compute(plain, V, *phis, inp.momenta, inp.spins, inp.coeffs).cpu().numpy()
    first_launches = bb.bblock_last_launch_count(plain)   # includes the phase-table kernel
    bb.bblock_compute(plain, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    n_plain = bb.bblock_last_launch_count(plain)           # phase table cached
    assert first_launches == n_plain + 1
    ctx = bb.bblock_create(4, 10, 12, precision, bf16_products=products)
    assert bb.bblock_get_option(ctx, "graphs") == 1
    B = torch.empty_like(torch.from_numpy(ref)).to("cuda:0")
    stream = torch.cuda.Stream()       # graphs need a created (capturable) stream
    torch.cuda.synchronize()
    for call in range(4):          # plain, capture + replay, replay, replay
        with torch.cuda.stream(stream):
            B.zero_()
        bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B,
                          stream=stream)
        bb.bblock_status(ctx)
        assert np.array_equal(B.cpu().numpy(), ref), f"call {call}"
        assert bb.bblock_last_launch_count(ctx) == (first_launches if call == 0 else n_plain)
    # the inputs change in place: a replay reads them afresh
    phis[0].mul_(2.0)
    torch.cuda.synchronize()
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B, stream=stream)
    bb.bblock_status(ctx)
    assert np.allclose(B.cpu().numpy(), 2.0 * ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # different arguments (another output buffer, other momenta) fall back to plain launches
    B2 = torch.zeros_like(B)
    torch.cuda.synchronize()
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B2, stream=stream)
    mom2 = inp.momenta[:2]
    B3 = bb.bblock_compute(ctx, V, *phis, mom2, inp.spins, inp.coeffs, stream=stream)
    bb.bblock_status(ctx)
    B_ref2 = B.cpu().numpy()
    assert np.array_equal(B2.cpu().numpy(), B_ref2)
    assert np.array_equal(B3.cpu().numpy(), B_ref2[:, :2])
    # back to the captured arguments: the replay finds the phase table of other momenta
    # in the context and must restore it first
    with torch.cuda.stream(stream):
        B.zero_()
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B, stream=stream)
    bb.bblock_status(ctx)
    assert np.array_equal(B.cpu().numpy(), B_ref2)
    bb.bblock_destroy(ctx)
    bb.bblock_destroy(plain)


@pytest.mark.parametrize("nc,chunk,slabs", [(16, 1, 0), (32, 3, 0), (48, 2, 5), (0, 4, 1), (0, 0, 17)])
def test_tile_options_keep_parity(env, nc, chunk, slabs):
    torch, bb = env
    inp = workloads.custom(5, 12, (12, 11, 13), 1, [(0, 0, 0), (1, 0, 0), (1, 1, 0)],
                           [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7], seed=3100)
    V, phis = setup(torch, inp)
    ref = oracle.bblock(5, inp.V[0], *[inp.phi[0][i][0] for i in range(3)], inp.momenta,
                        inp.spins, inp.coeffs)
    ctx = bb.bblock_create(5, 12, 13, "bf16", bf16_products=6)
    bb.bblock_set_option(ctx, "tc_nc", nc)
    bb.bblock_set_option(ctx, "tc_chunk", chunk)
    bb.bblock_set_option(ctx, "slabs", slabs)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy()[0], ref) <= 1e-6
    bb.bblock_destroy(ctx)
    ctx = bb.bblock_create(5, 12, 13, "fp64")
    bb.bblock_set_option(ctx, "slabs", slabs)
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs)
    bb.bblock_status(ctx)
    assert rel(B.cpu().numpy()[0], ref) <= 1e-12
    bb.bblock_destroy(ctx)


def test_bad_option_values_are_rejected(env):
    torch, bb = env
    ctx = bb.bblock_create(2, 4, 4, "fp64")
    for opt, val in (("tc_nc", 40), ("tc_chunk", 9), ("graphs", 2), ("slabs", -1)):
        with pytest.raises(bb.BblockError, match="INVALID_ARG"):
            bb.bblock_set_option(ctx, opt, val)
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("precision,products,tol", [("fp64", 6, 1e-12), ("df64", 6, 1e-12), ("bf16", 6, 1e-6),
                                                    ("tf32x3", 6, 1e-6), ("fp16x3", 6, 1e-6)])
def test_multi_wave_batch_graph_replay(env, precision, products, tol):
    """A batch that runs as several waves of launches (a small workspace budget per wave),
    with mixed dilution sizes, captured and replayed: each wave's table copy in the graph
    must carry that wave's jobs."""
    torch, bb = env
    L, n_ev, mom = 6, 16, [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    spins, coeffs = [(0, 1, 0), (1, 0, 0), (2, 3, 2)], [0.7, -0.7, 0.7]
    dev = torch.device("cuda:0")
    inps = [workloads.custom(L, n_ev, nd, 3, mom, spins, coeffs, seed=3200 + k)
            for k, nd in enumerate([(16, 16, 16), (12, 12, 16), (16, 12, 8)])]
    jobs_dev, outs = [], []
    for inp in inps:
        V = torch.from_numpy(inp.V).to(dev)
        phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
        Bk = torch.zeros((inp.workload.n_t, len(mom), *inp.ndil[0]), dtype=torch.complex128, device=dev)
        outs.append(Bk)
        for t in range(inp.workload.n_t):
            jobs_dev.append((V[t], phis[0][t], phis[1][t], phis[2][t], Bk[t]))
    stream = torch.cuda.Stream()

    def run(ctx):
        with torch.cuda.stream(stream):
            for Bk in outs:
                Bk.zero_()
        bb.bblock_compute_batch(ctx, jobs_dev, mom, spins, coeffs, stream=stream)
        bb.bblock_status(ctx)
        stream.synchronize()
        return [Bk.cpu().numpy() for Bk in outs], bb.bblock_last_launch_count(ctx)

    one_wave = bb.bblock_create(L, n_ev, 16, precision, bf16_products=products)
    bb.bblock_set_option(one_wave, "graphs", 0)
    _, n_one = run(one_wave)
    plain = bb.bblock_create(L, n_ev, 16, precision, bf16_products=products)
    bb.bblock_set_option(plain, "graphs", 0)
    bb.bblock_set_option(plain, "wave_mb", 16)
    assert bb.bblock_get_option(plain, "wave_mb") == 16
    ref, n_plain = run(plain)
    assert n_plain - 1 >= 3 * (n_one - 1)     # at least 3 waves (the first launch: phase table)
    for k, inp in enumerate(inps):
        for t in (0, inp.workload.n_t - 1):
            want = oracle.bblock(L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)], mom, spins, coeffs)
            assert rel(ref[k][t], want) <= tol, (k, t)
    ctx = bb.bblock_create(L, n_ev, 16, precision, bf16_products=products)
    bb.bblock_set_option(ctx, "wave_mb", 16)
    for call in range(4):          # plain, capture + replay, replay, replay
        got, n = run(ctx)
        for k in range(len(inps)):
            assert np.array_equal(got[k], ref[k]), (call, k)
        assert n == (n_plain if call == 0 else n_plain - 1)   # phase table cached after call 0
    for c in (one_wave, plain, ctx):
        bb.bblock_destroy(c)


@pytest.mark.parametrize("precision,products", [("fp64", 6), ("bf16", 6), ("fp16x3", 6)])
def test_launch_timing_covers_graph_replays(env, precision, products):
    """With launch timing on, the captured graph carries the timing events, so replays are
    timed launch by launch: every replay adds its launches to the per-kernel totals, and
    the replayed blocks stay bitwise those of the plain launches."""
    torch, bb = env
    inp = workloads.custom(4, 10, (9, 8, 12), 2, [(0, 0, 0), (1, 0, 0)],
                           [(0, 1, 0), (1, 0, 0)], [0.7, -0.7], seed=3100)
    V, phis = setup(torch, inp)
    ctx = bb.bblock_create(4, 10, 12, precision, bf16_products=products)
    stream = torch.cuda.Stream()
    B = torch.empty((2, 2, 9, 8, 12), dtype=torch.complex128, device="cuda:0")
    bb.bblock_profile_enable(ctx, True)
    outs = []
    for call in range(5):      # plain, capture + first replay, three replays
        bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B,
                          stream=stream)
        bb.bblock_status(ctx)
        outs.append(B.cpu().numpy())
        if call == 0:
            n_plain = bb.bblock_last_launch_count(ctx) - 1     # without the phase table
            bb.bblock_profile_read(ctx)                        # reset
    prof = bb.bblock_profile_read(ctx)
    bb.bblock_profile_enable(ctx, False)
    assert sum(v[0] for v in prof.values()) == 4 * n_plain, prof
    assert prof["contract"][0] >= 4 and all(v[1] > 0 for v in prof.values())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    ref = oracle.bblock(4, inp.V[0], *[inp.phi[0][i][0] for i in range(3)], inp.momenta,
                        inp.spins, inp.coeffs)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert rel(outs[-1][0], ref) <= tol
    bb.bblock_destroy(ctx)
