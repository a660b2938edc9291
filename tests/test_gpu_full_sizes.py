"""Parity of the larger workloads at their full sizes, on sampled block entries.

Whole blocks of these workloads are too large for the oracle to finish in a test, so every
check takes a few dilution indices per quark line, always including the last index of the
line, which lies in the ragged edge of a tile. It then evaluates the definition on those
columns (``oracle.bblock_sampled``). The GPU computes the full blocks at the workload's sizes
in its default launch configuration: default tiles, CUDA graphs on a created stream.

* L = 32, N_ev = 128, N_dil = 64, 5 momenta, 4 spin triples, two of the 16 time slices:
  every form.
* L = 48, N_ev = 264, N_dil = 64, 7 momenta, 4 spin triples, one of the 4 time slices: the
  FP64 and double-float forms and the BF16 split with 6 products.
* L = 32, N_ev = 128, 9 momenta, 6 noise triples with N_dil drawn from {32, 48, 64}, two
  time slices per noise triple: 12 jobs of uneven size in one batched call, in the mixed
  forms and the double-float form. The call is repeated, so the second call is a
  CUDA-graph capture and the third a replay; every call is checked.
* The same workload at its full size, all 48 time slices: 288 jobs in one batched call, in
  the benchmark's headline form and launch configuration. The default workspace budget
  splits it into several waves; the second call is captured and the third replayed, and
  both are checked on jobs spread over every wave.

Tolerances are relative Frobenius errors over the sampled entries: 1e-12 for the FP64 and
double-float forms, 1e-6 for the split forms with 6 or 9 BF16 products and for TF32x3, and
1e-4 for the BF16 split with 3 products. The last form's dropped products are about
3 * 2^-16 relative, so it is reported rather than held to 1e-6.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

FORMS = {"fp64": ("fp64", 6, 1e-12), "df64": ("df64", 6, 1e-12),
         "bf16x6": ("bf16", 6, 1e-6), "bf16x9": ("bf16", 9, 1e-6),
         "tf32x3": ("tf32x3", 6, 1e-6), "bf16x3": ("bf16", 3, 1e-4),
         "fp16x3": ("fp16x3", 6, 1e-6)}


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


def samples(nd):
    """A few dilution indices of a line with nd columns: first, interior, last."""
    return sorted({0, nd // 3, (2 * nd) // 3 + 1, nd - 1})


def sampled(block, d1s, d2s, d3s):
    return block[:, d1s][:, :, d2s][:, :, :, d3s]


@pytest.fixture(scope="module")
def l32_inputs():
    return workloads.generate(workloads.WORKLOADS["l32_nev128_ndil64"], n_t=2)


@pytest.mark.parametrize("form", list(FORMS))
def test_l32_nev128_ndil64_sampled(env, l32_inputs, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    inp = l32_inputs
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    nd = inp.ndil[0]
    ctx = bb.bblock_create(w.L, w.n_ev, max(nd), precision, bf16_products=products)
    stream = torch.cuda.Stream()
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, stream=stream)
    bb.bblock_status(ctx)
    got = B.cpu().numpy()
    bb.bblock_destroy(ctx)
    d1s, d2s, d3s = samples(nd[0]), samples(nd[1]), samples(nd[2])
    for t in range(inp.V.shape[0]):
        ref = oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[0][i][t] for i in range(3)],
                                    inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
        err = rel(sampled(got[t], d1s, d2s, d3s), ref)
        print(f"{form} L=32 t={t}: sampled rel. error {err:.3e}")
        assert err <= tol


@pytest.mark.parametrize("form", ["fp64", "df64", "bf16x6", "fp16x3"])
def test_l48_nev264_ndil64_sampled(env, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    inp = workloads.generate(workloads.WORKLOADS["l48_nev264_ndil64"], n_t=1)
    w = inp.workload
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    phis = [torch.from_numpy(inp.phi[0][i]).to(dev) for i in range(3)]
    nd = inp.ndil[0]
    ctx = bb.bblock_create(w.L, w.n_ev, max(nd), precision, bf16_products=products)
    stream = torch.cuda.Stream()
    B = bb.bblock_compute(ctx, V, *phis, inp.momenta, inp.spins, inp.coeffs, stream=stream)
    bb.bblock_status(ctx)
    got = B.cpu().numpy()[0]
    bb.bblock_destroy(ctx)
    d1s, d2s, d3s = samples(nd[0]), samples(nd[1]), samples(nd[2])
    ref = oracle.bblock_sampled(w.L, inp.V[0], *[inp.phi[0][i][0] for i in range(3)],
                                inp.momenta, inp.spins, inp.coeffs, d1s, d2s, d3s)
    err = rel(sampled(got, d1s, d2s, d3s), ref)
    print(f"{form} L=48: sampled rel. error {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("form", ["bf16x6", "tf32x3", "df64", "fp16x3"])
def test_l32_batch_uneven_dilution_sampled(env, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    w = workloads.WORKLOADS["l32_batch_48t_6noise"]
    inp = workloads.generate(w, n_t=2)
    n_t = inp.V.shape[0]
    assert len({nd[0] for nd in inp.ndil}) > 1          # uneven dilution across the batch
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    jobs, outs = [], []
    for k in range(w.n_noise):
        phis = [torch.from_numpy(inp.phi[k][i]).to(dev) for i in range(3)]
        Bk = torch.empty((n_t, len(inp.momenta), *inp.ndil[k]), dtype=torch.complex128, device=dev)
        outs.append(Bk)
        for t in range(n_t):
            jobs.append((V[t], phis[0][t], phis[1][t], phis[2][t], Bk[t]))
    refs = {}
    for k in range(w.n_noise):
        nd = inp.ndil[k]
        ds = (samples(nd[0]), samples(nd[1]), samples(nd[2]))
        for t in range(n_t):
            refs[k, t] = (ds, oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[k][i][t] for i in range(3)],
                                                    inp.momenta, inp.spins, inp.coeffs, *ds))
    ctx = bb.bblock_create(w.L, w.n_ev, max(max(nd) for nd in inp.ndil), precision,
                           bf16_products=products)
    stream = torch.cuda.Stream()
    for call in range(3):           # plain launches, graph capture + replay, replay
        with torch.cuda.stream(stream):
            for Bk in outs:
                Bk.fill_(float("nan"))
        bb.bblock_compute_batch(ctx, jobs, inp.momenta, inp.spins, inp.coeffs, stream=stream)
        bb.bblock_status(ctx)
        stream.synchronize()
        got = [Bk.cpu().numpy() for Bk in outs]
        worst = 0.0
        for (k, t), (ds, ref) in refs.items():
            err = rel(sampled(got[k][t], *ds), ref)
            worst = max(worst, err)
            assert err <= tol, (call, k, t, err)
        print(f"{form} batch call {call}: worst sampled rel. error {worst:.3e}")
    bb.bblock_destroy(ctx)


@pytest.mark.parametrize("form", ["bf16x6", "fp16x3"])
def test_l32_full_batch_every_wave_sampled(env, form):
    torch, bb = env
    precision, products, tol = FORMS[form]
    w = workloads.WORKLOADS["l32_batch_48t_6noise"]
    inp = workloads.generate(w)
    n_t = inp.V.shape[0]
    assert n_t == 48 and len(inp.ndil) == 6
    dev = torch.device("cuda:0")
    V = torch.from_numpy(inp.V).to(dev)
    jobs, outs = [], []
    for k in range(w.n_noise):
        phis = [torch.from_numpy(inp.phi[k][i]).to(dev) for i in range(3)]
        Bk = torch.empty((n_t, len(inp.momenta), *inp.ndil[k]), dtype=torch.complex128, device=dev)
        outs.append(Bk)
        for t in range(n_t):
            jobs.append((V[t], phis[0][t], phis[1][t], phis[2][t], Bk[t]))
    n = len(jobs)
    # 16 jobs spread evenly over the job list (noise-major), first and last included
    picks = sorted({round(i * (n - 1) / 15) for i in range(16)})
    refs = {}
    for j in picks:
        k, t = divmod(j, n_t)
        nd = inp.ndil[k]
        ds = (samples(nd[0]), samples(nd[1]), samples(nd[2]))
        refs[k, t] = (ds, oracle.bblock_sampled(w.L, inp.V[t], *[inp.phi[k][i][t] for i in range(3)],
                                                inp.momenta, inp.spins, inp.coeffs, *ds))
    ctx = bb.bblock_create(w.L, w.n_ev, max(max(nd) for nd in inp.ndil), precision,
                           bf16_products=products)
    stream = torch.cuda.Stream()
    for call in range(3):           # plain launches, graph capture + replay, replay
        with torch.cuda.stream(stream):
            for Bk in outs:
                Bk.fill_(float("nan"))
        bb.bblock_compute_batch(ctx, jobs, inp.momenta, inp.spins, inp.coeffs, stream=stream)
        waves = bb.bblock_last_wave_count(ctx)
        bb.bblock_status(ctx)
        stream.synchronize()
        assert waves >= 3, waves
        worst = 0.0
        for (k, t), (ds, ref) in refs.items():
            got = outs[k][t].cpu().numpy()
            err = rel(sampled(got, *ds), ref)
            worst = max(worst, err)
            assert err <= tol, (call, k, t, err)
        print(f"{form} full batch call {call}: {waves} waves, worst sampled rel. error "
              f"{worst:.3e} over {len(refs)} jobs")
    bb.bblock_destroy(ctx)
