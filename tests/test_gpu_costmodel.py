"""The autotuner and its learned cost model, on the GPU through the C ABI.

* The cost model's forward and backward kernels give the loss and gradient of the FP64
  reference network (``oracle.mlp``), within FP32 rounding.
* Training (Adam, on the GPU) fits a smooth target and is bitwise reproducible.
* Gain: trained on the autotuner's timings of two workloads, the model ranks the candidate
  tiles of a third workload; timing only its top 3 of 27 candidates must find a tile within
  10 % of the exhaustive search's best, with 9x fewer timed candidates and less tuning
  wall time.
* Tuning never changes the arithmetic: tuned blocks still match the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import workloads
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_16278_gb300 as bb
    bb.load()
    return torch, bb


def test_gradient_matches_reference_network(env):
    torch, bb = env
    F, H, n = 12, 32, 100
    cm = bb.CostModel(F, H, seed=3)
    rng = np.random.default_rng(4)
    p = (rng.standard_normal(cm.num_params()) * 0.3).astype(np.float32)
    cm.set_params(p)
    assert np.array_equal(cm.get_params(), p)
    X = rng.standard_normal((n, F)).astype(np.float32)
    y = rng.standard_normal(n).astype(np.float32)
    loss, grad = cm.gradient(X, y)
    ref_loss = mlp.loss(p.astype(np.float64), X, y, F, H)
    ref_grad = mlp.gradient(p.astype(np.float64), X, y, F, H)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.linalg.norm(grad - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad)
    pred = cm.predict(X)
    f, _, _ = mlp.forward(p.astype(np.float64), X, F, H)
    assert np.abs(pred - f).max() <= 1e-5 * max(1.0, np.abs(f).max())


def test_training_fits_and_is_reproducible(env):
    torch, bb = env
    F, H, n = 4, 16, 256
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (n, F)).astype(np.float32)
    y = (np.sin(2 * X[:, 0]) + 0.5 * X[:, 1] ** 2 - 0.3 * X[:, 2] * X[:, 3]).astype(np.float32)
    runs = []
    for _ in range(2):
        cm = bb.CostModel(F, H, seed=11)
        l0, _ = cm.gradient(X, y)
        l1 = cm.train(X, y, epochs=1500, lr=1e-2)
        runs.append((l0, l1, cm.get_params()))
    assert runs[0][1] < 0.02 * runs[0][0]
    assert np.array_equal(runs[0][2], runs[1][2])


def _workload(torch, L, n_ev, nd, n_t, mom, seed):
    spins = [(0, 1, 0), (1, 0, 0), (2, 3, 2)]
    inp = workloads.custom(L, n_ev, (nd, nd, nd), n_t, mom, spins, [0.7, -0.7, 0.7], seed=seed)
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    B = torch.empty((n_t, len(mom), nd, nd, nd), dtype=torch.complex128, device=dev)
    return inp, V, phis, B


def test_model_ranking_gains_over_exhaustive_search(env):
    torch, bb = env
    mom3 = [(0, 0, 0), (1, 0, 0), (1, 1, 0)]
    mom5 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0)]
    shapes = [(16, 48, 24, 4, mom3, 1), (18, 48, 32, 2, mom5, 2), (20, 64, 28, 2, mom3, 3)]
    stream = torch.cuda.Stream()
    data = []
    for L, n_ev, nd, n_t, mom, seed in shapes:
        inp, V, phis, B = _workload(torch, L, n_ev, nd, n_t, mom, 4000 + seed)
        ctx = bb.bblock_create(L, n_ev, nd, "bf16", bf16_products=6)
        bb.bblock_set_option(ctx, "graphs", 0)
        bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B,
                          stream=stream)      # warm caches before timing
        t0 = time.perf_counter()
        rep = bb.bblock_autotune(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B,
                                 stream=stream, repeats=3)
        wall = time.perf_counter() - t0
        assert len(rep) == 27 and all(r["ms"] > 0 for r in rep)
        data.append((ctx, inp, V, phis, B, rep, wall))
    X_train = np.concatenate([[r["features"] for r in d[5]] for d in data[:2]])
    y_train = np.log(np.concatenate([[r["ms"] for r in d[5]] for d in data[:2]]))
    cm = bb.CostModel(bb.bblock.TUNE_FEATURES, 32, seed=7)
    loss = cm.train(X_train, y_train, epochs=3000, lr=3e-3)
    ctx, inp, V, phis, B, rep_ex, wall_ex = data[2]
    best_ex = min(r["ms"] for r in rep_ex)
    t0 = time.perf_counter()
    rep_m = bb.bblock_autotune(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B,
                               stream=stream, model=cm, top_k=3, repeats=3)
    wall_m = time.perf_counter() - t0
    timed = [r for r in rep_m if r["ms"] > 0]
    best_m = min(r["ms"] for r in timed)
    default = [r["ms"] for r in rep_ex if (r["nc"], r["chunk"], r["slabs"]) == (48, 2, 0)]
    print(f"train loss {loss:.4f}; exhaustive best {best_ex:.3f} ms over 27 timed in "
          f"{wall_ex:.2f} s; model top-3 best {best_m:.3f} ms over {len(timed)} timed in "
          f"{wall_m:.2f} s; default tile {default[0] if default else float('nan'):.3f} ms")
    assert len(timed) == 3 and len(timed) < len(rep_ex)
    assert wall_m < wall_ex
    assert best_m <= 1.10 * best_ex
    # the tuned context still computes the same blocks
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B, stream=stream)
    bb.bblock_status(ctx)
    d1s, d2s, d3s = [0, 9, 27], [3, 27], [1, 26, 27]
    ref = oracle.bblock_sampled(inp.workload.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)],
                                inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
    got = B.cpu().numpy()[0][:, d1s][:, :, d2s][:, :, :, d3s]
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    for d in data:
        bb.bblock_destroy(d[0])


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_fp64_accurate_autotune_keeps_parity(env, precision):
    torch, bb = env
    inp, V, phis, B = _workload(torch, 6, 12, 10, 2, [(0, 0, 0), (1, 0, 0)], 4100)
    ctx = bb.bblock_create(6, 12, 10, precision)
    rep = bb.bblock_autotune(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B, repeats=2)
    assert len(rep) == 4 and all(r["ms"] > 0 for r in rep)
    bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, B_out=B)
    bb.bblock_status(ctx)
    for t in range(2):
        ref = oracle.bblock(6, inp.V[t], *[inp.phi[0][i][t] for i in range(3)], inp.momenta,
                            inp.spins, inp.coeffs)
        got = B.cpu().numpy()[t]
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    bb.bblock_destroy(ctx)
