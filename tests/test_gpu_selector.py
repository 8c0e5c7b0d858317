"""The selector's kernels against the selector oracle (needs a GB300):
chunk statistics, MLP forward, loss gradient and SGD step, the selection
rule; then a small end-to-end training run showing what the trained network
gains over the fixed heuristic on held-out chunks."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import selector as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def zc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build()
    from paper_2308_05199_gb300 import zc as z
    z.zc_set_tile_chunks(8)
    return z


def np_of(t):
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def stats_chunks():
    r = np.random.default_rng(4)
    eb = 2.0 ** -10
    xs, ebs = [], []
    for n in (5, 100, 128, 129, 1000, 16384, 16384 + 77, 32768):
        xs.append(torch.from_numpy((r.standard_t(3, n) * 0.05).astype(np.float32)))
        ebs.append(1e-4)
    xs.append(torch.zeros(16384))
    ebs.append(1e-3)
    xs.append(torch.full((16384,), 0.3))
    ebs.append(1e-3)
    xs.append(torch.from_numpy((np.arange(16384) * 2 * eb).astype(np.float32)))
    ebs.append(eb)
    xs.append(torch.from_numpy(np.cumsum(r.normal(0, 0.01, 16384)).astype(np.float32)))
    ebs.append(1e-3)
    bf = torch.from_numpy((r.standard_t(3, 32768) * 0.05).astype(np.float32)).to(torch.bfloat16)
    xs.append(bf)
    ebs.append(1e-4)
    xs.append(bf[:20000])
    ebs.append(1e-2)
    bad = torch.zeros(16384)
    bad[1024 + 5] = float("inf")  # in sampled span 1
    xs.append(bad)
    ebs.append(1e-3)
    return xs, ebs


def test_chunk_stats_match_oracle(zc):
    xs, ebs = stats_chunks()
    b = zc.BatchCompress([x.cuda() for x in xs], [32] * len(xs), ebs)
    feat = torch.empty((len(xs), 16), device="cuda")
    assert zc.zc_batch_chunk_stats(b.plan, feat.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream) == 0
    got = feat.cpu().numpy().astype(np.float64)
    for i, (x, eb) in enumerate(zip(xs, ebs)):
        ref = OS.chunk_stats(np_of(x), eb)
        assert np.array_equal(np.isnan(got[i]), np.isnan(ref)), i
        ok = ~np.isnan(ref)
        # FP32 on the GPU: a few roundings (divisions, sums, log2f) on values the
        # oracle computes in FP64 from the same exact integer counts
        np.testing.assert_allclose(got[i][ok], ref[ok], rtol=1e-6, atol=2e-6, err_msg=str(i))


def _mlp_problem(B, seed):
    r = np.random.default_rng(seed)
    p = (OS.init_params(seed) + r.normal(0, 0.05, OS.N_PARAMS)).astype(np.float32)
    norm = np.concatenate([r.normal(0, 1, 16), r.uniform(0.5, 2, 16)]).astype(np.float32)
    X = r.normal(0, 1, (B, 16)).astype(np.float32)
    T = r.normal(0, 1, (B, 4)).astype(np.float32)
    return p, norm, X, T


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("B", [1, 63, 64, 200, 50001])  # 50001: CTAs loop over row tiles
def test_mlp_forward_matches_oracle(zc, B):
    p, norm, X, T = _mlp_problem(B, B)
    y = torch.empty((B, 4), device="cuda")
    dP, dN, dX = _dev(p), _dev(norm), _dev(X)  # alive until the kernel has run
    assert zc.zc_mlp_forward(dP.data_ptr(), dN.data_ptr(), dX.data_ptr(), B, y.data_ptr(),
                             torch.cuda.current_stream().cuda_stream) == 0
    ref = OS.forward(p.astype(np.float64), norm.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("B", [1, 64, 200, 1000])
def test_mlp_gradient_matches_oracle(zc, B):
    p, norm, X, T = _mlp_problem(2 * B + 3, B + 7)
    idx = np.random.default_rng(B).permutation(2 * B + 3)[:B].astype(np.int32)
    g = torch.empty(OS.N_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scratch = torch.empty(zc.zc_mlp_scratch_bytes(B) // 4, device="cuda")
    dX, dT, dI, dP, dN = _dev(X), _dev(T), _dev(idx), _dev(p), _dev(norm)
    st = zc.zc_mlp_grad(dP.data_ptr(), dN.data_ptr(), dX.data_ptr(), dT.data_ptr(),
                        dI.data_ptr(), B, g.data_ptr(), loss.data_ptr(), scratch.data_ptr(),
                        scratch.numel() * 4, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    ref_loss, ref_g = OS.loss_grad(p.astype(np.float64), norm.astype(np.float64),
                                   X[idx].astype(np.float64), T[idx].astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    # FP32 sums of at most 1000 terms: within 1e-4 of the largest gradient entry
    assert np.max(np.abs(gg - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    # same inputs, same bits: the summation order is fixed
    g2 = torch.empty_like(g)
    zc.zc_mlp_grad(dP.data_ptr(), dN.data_ptr(), dX.data_ptr(), dT.data_ptr(),
                   dI.data_ptr(), B, g2.data_ptr(), None, scratch.data_ptr(), scratch.numel() * 4,
                   torch.cuda.current_stream().cuda_stream)
    assert torch.equal(g, g2)


def test_sgd_step_matches_oracle(zc):
    r = np.random.default_rng(9)
    p = r.normal(0, 1, OS.N_PARAMS).astype(np.float32)
    v = r.normal(0, 1, OS.N_PARAMS).astype(np.float32)
    g = r.normal(0, 1, OS.N_PARAMS).astype(np.float32)
    dp, dv, dg = _dev(p), _dev(v), _dev(g)
    assert zc.zc_mlp_sgd(dp.data_ptr(), dv.data_ptr(), dg.data_ptr(), 0.05, 0.9,
                         torch.cuda.current_stream().cuda_stream) == 0
    rp, rv = OS.sgd_step(p, v, g, 0.05, 0.9)
    np.testing.assert_allclose(dv.cpu().numpy(), rv, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(dp.cpu().numpy(), rp, rtol=1e-6, atol=1e-6)


def test_selection_matches_oracle(zc):
    r = np.random.default_rng(3)
    M = 3000
    sizes = r.integers(1, 16385, M)
    xs = [torch.zeros(int(n), dtype=torch.float32 if i % 3 else torch.bfloat16, device="cuda")
          for i, n in enumerate(sizes)]
    b = zc.BatchCompress(xs, [32] * M, [1e-3] * M)
    f = np.abs(r.normal(8, 6, (M, 16))).astype(np.float32) + 0.5
    f[r.random(M) < 0.02, 1] = np.nan
    y = (np.log2(f[:, :4]) + r.normal(0, 0.6, (M, 4))).astype(np.float32)
    y[r.random(M) < 0.01, 2] = np.inf
    cfg = zc.ZcSelectCfg()
    cfg.link_gbs, cfg.raw_ns_per_byte, cfg.judge_log2 = 12.5, 0.004, 1.0
    for k, c in enumerate((0.03, 0.02, 0.018, 0.017)):
        cfg.ns_per_byte[k] = c
    ocfg = {"link_gbs": 12.5, "ns_per_byte": [0.03, 0.02, 0.018, 0.017], "raw_ns_per_byte": 0.004,
            "judge_log2": 1.0}
    dF, dY = _dev(f), _dev(y)
    choice = torch.zeros(M, dtype=torch.int32, device="cuda")
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    for use_mlp in (False, True):
        assert zc.zc_batch_select(b.plan, dF.data_ptr(), dY.data_ptr() if use_mlp else None, cfg,
                                  choice.data_ptr(), counts.data_ptr(), s) == 0
        got = choice.cpu().numpy()
        fb = 0
        for i in range(M):
            n, es = int(sizes[i]), (4 if i % 3 else 2)
            if use_mlp:
                want, fell = OS.mlp_choice(n, es, f[i].astype(np.float64), y[i].astype(np.float64),
                                           ocfg)
                fb += fell
            else:
                want = OS.heuristic_choice(n, es, f[i].astype(np.float64), ocfg)
            if got[i] != want:
                # only where FP32 and FP64 costs tie to within rounding
                coded, raw = OS.chunk_costs(n, es, [2.0 ** float(v) for v in y[i]] if use_mlp
                                            else [float(f[i, 1])] * 4, ocfg)
                allc = dict(zip((16, 32, 64, 128, 0), coded + [raw]))
                assert abs(allc[int(got[i])] - allc[want]) <= 1e-5 * allc[want], (i, got[i], want)
        if use_mlp:
            assert abs(int(counts[0].item()) - fb) <= 2
        assert int(counts[1].item()) == int((got == 0).sum())
    # the choices went into the plan: compressing now yields the chosen streams
    b.run()
    assert b.ws.status()[0] == 0
    for i, st in enumerate(b.streams()[:200]):
        h = oracle.header(st)
        if got[i] == 0:
            assert h["flags"] == 1
        else:
            assert h["flags"] == 0 and 1 << h["log2L"] == got[i]


def test_timed_selection_matches_oracle(zc):
    """zc_batch_select_timed against the oracle's choice with a time
    prediction: per-chunk rates judged against the batch-wide ones."""
    r = np.random.default_rng(13)
    M = 3000
    sizes = r.integers(1, 16385, M)
    xs = [torch.zeros(int(n), dtype=torch.float32 if i % 3 else torch.bfloat16, device="cuda")
          for i, n in enumerate(sizes)]
    b = zc.BatchCompress(xs, [32] * M, [1e-3] * M)
    f = np.abs(r.normal(8, 6, (M, 16))).astype(np.float32) + 0.5
    y = (np.log2(f[:, :4]) + r.normal(0, 0.3, (M, 4))).astype(np.float32)
    rates = [0.03, 0.02, 0.018, 0.017]
    judge_t = 1.5
    yt = (np.log2(rates)[None, :] + r.normal(0, 1.2, (M, 4))).astype(np.float32)
    # keep every time prediction clear of the judge's threshold (FP32 vs FP64)
    edge = np.abs(np.abs(yt.astype(np.float64) - np.log2(rates)[None, :]) - judge_t) < 1e-3
    yt[edge] += np.float32(0.01)
    yt[r.random(M) < 0.01, 1] = np.nan
    cfg = zc.ZcSelectCfg()
    cfg.link_gbs, cfg.raw_ns_per_byte, cfg.judge_log2, cfg.judge_time_log2 = 100.0, 0.004, 1.0, judge_t
    for k, c in enumerate(rates):
        cfg.ns_per_byte[k] = c
    ocfg = {"link_gbs": 100.0, "ns_per_byte": rates, "raw_ns_per_byte": 0.004,
            "judge_log2": 1.0, "judge_time_log2": judge_t}
    dF, dY, dT = _dev(f), _dev(y), _dev(yt)
    choice = torch.zeros(M, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert zc.zc_batch_select_timed(b.plan, dF.data_ptr(), dY.data_ptr(), dT.data_ptr(), cfg,
                                    choice.data_ptr(), None, s) == 0
    got = choice.cpu().numpy()
    changed = 0
    for i in range(M):
        n, es = int(sizes[i]), (4 if i % 3 else 2)
        want, _ = OS.mlp_choice(n, es, f[i].astype(np.float64), y[i].astype(np.float64), ocfg,
                                yt[i].astype(np.float64))
        plain, _ = OS.mlp_choice(n, es, f[i].astype(np.float64), y[i].astype(np.float64), ocfg)
        changed += want != plain
        if got[i] != want:
            coded, raw = OS.chunk_costs(n, es, [2.0 ** float(v) for v in y[i]], ocfg,
                                        OS.judged_rates(yt[i].astype(np.float64), ocfg))
            allc = dict(zip((16, 32, 64, 128, 0), coded + [raw]))
            assert abs(allc[int(got[i])] - allc[want]) <= 1e-5 * allc[want], (i, got[i], want)
    assert changed > M // 10  # the time prediction really moves choices
    # no time prediction: exactly zc_batch_select
    c2 = torch.zeros_like(choice)
    assert zc.zc_batch_select_timed(b.plan, dF.data_ptr(), dY.data_ptr(), None, cfg,
                                    c2.data_ptr(), None, s) == 0
    assert zc.zc_batch_select(b.plan, dF.data_ptr(), dY.data_ptr(), cfg, choice.data_ptr(),
                              None, s) == 0
    assert torch.equal(choice, c2)


def test_time_network_predicts_the_codec_rate_on_held_out_chunks(zc):
    """The time network, trained on rates the codec measured on groups of
    training chunks, predicts held-out groups' measured rates better than
    the batch-wide rate at each L does."""
    from paper_2308_05199_gb300 import selector as S
    train_v, train_e, _ = S.mixed_chunks(3000, seed=1, scale=64)
    test_v, test_e, _ = S.mixed_chunks(1600, seed=2, scale=64)
    tr = S.ChunkBatch(train_v, train_e)
    te = S.ChunkBatch(test_v, test_e)
    cfg = tr.cost_model(link_gbs=100.0)
    X, _, keep, bits = S.dataset(tr)
    rates, _ = S.time_labels(train_v, train_e, bits, groups=8)
    T = torch.from_numpy(np.log2(rates[keep]).astype(np.float32)).cuda()
    tm = S.Mlp(seed=1)
    tm.set_norm(X)
    hist = tm.fit(X, T, epochs=40, batch=256, lr=0.02, momentum=0.9, seed=0)
    assert hist[-1] < 0.5 * hist[0]
    feat = te.stats().clone()
    tbits = te.true_bits()
    trates, _ = S.time_labels(test_v, test_e, tbits, groups=8)
    ok = torch.isfinite(feat).all(1).cpu().numpy()
    pt = tm.forward(feat).cpu().numpy().astype(np.float64)
    want = np.log2(trates)
    uni = np.log2(np.array([cfg.ns_per_byte[k] for k in range(4)]))[None, :]
    err_net = np.sqrt(np.mean((pt[ok] - want[ok]) ** 2))
    err_uni = np.sqrt(np.mean((uni - want[ok]) ** 2))
    assert err_net < 0.7 * err_uni, (err_net, err_uni)


def test_training_beats_the_heuristic_on_held_out_chunks(zc):
    from paper_2308_05199_gb300 import selector as S
    train_v, train_e, _ = S.mixed_chunks(3000, seed=1, scale=64)
    test_v, test_e, _ = S.mixed_chunks(1600, seed=2, scale=64)
    tr = S.ChunkBatch(train_v, train_e)
    te = S.ChunkBatch(test_v, test_e)
    cfg = tr.cost_model(link_gbs=12.5)
    X, T, _, _ = S.dataset(tr)
    mlp = S.Mlp(seed=0)
    mlp.set_norm(X)
    hist = mlp.fit(X, T, epochs=40, batch=256, lr=0.02, momentum=0.9, seed=0)
    assert hist[-1] < 0.5 * hist[0]
    feat = te.stats()
    bits = te.true_bits()
    pred = mlp.forward(feat)
    heur = te.select(cfg, None).cpu().numpy().copy()
    learned = te.select(cfg, pred).cpu().numpy().copy()
    eh = S.evaluate(heur, te.n, te.es, bits, cfg)
    el = S.evaluate(learned, te.n, te.es, bits, cfg)
    assert el["cost_ns"] < eh["cost_ns"], (el, eh)
    assert el["mispredict"] < eh["mispredict"], (el, eh)
