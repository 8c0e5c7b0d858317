"""Host bookkeeping of the learned selector (CPU only): the vectorised cost
model and evaluation the bench reports agree with the oracle's per-chunk
cost model and best choice, and chunking covers every message exactly."""
import numpy as np
import torch

from oracle import selector as S
from paper_2308_05199_gb300 import selector as P
from paper_2308_05199_gb300 import zc


def _cfg():
    c = zc.ZcSelectCfg()
    c.link_gbs = 12.5
    for k, v in enumerate((0.017, 0.015, 0.016, 0.018)):
        c.ns_per_byte[k] = v
    c.raw_ns_per_byte = 0.002
    c.judge_log2 = 1.0
    return c, {"link_gbs": 12.5, "ns_per_byte": [float(c.ns_per_byte[k]) for k in range(4)],
               "raw_ns_per_byte": float(c.raw_ns_per_byte)}


def _chunks(M, seed):
    r = np.random.default_rng(seed)
    es = r.choice([4, 2], M)
    n = (65536 // es) - r.integers(0, 3000, M) * (r.random(M) < 0.2)
    bits = r.uniform(0.5, 36.0, (M, 4))
    return n.astype(np.int64), es.astype(np.int64), bits


def test_vectorised_costs_match_the_oracle_cost_model():
    cfg, ocfg = _cfg()
    n, es, bits = _chunks(300, 1)
    coded, raw = P.costs(n, es, bits, cfg)
    for i in range(len(n)):
        oc, oraw = S.chunk_costs(int(n[i]), int(es[i]), list(bits[i]), ocfg)
        np.testing.assert_allclose(coded[i], oc, rtol=1e-12)
        assert raw[i] == np.float64(oraw) or abs(raw[i] - oraw) <= 1e-12 * oraw


def test_evaluation_against_the_oracle_best_choice():
    cfg, ocfg = _cfg()
    n, es, bits = _chunks(400, 2)
    best = np.array([S.best_choice(int(n[i]), int(es[i]), list(bits[i]), ocfg)[0]
                     for i in range(len(n))])
    ev = P.evaluate(best, n, es, bits, cfg)
    assert ev["regret"] == 0.0 and ev["mispredict"] == 0.0
    assert ev["raw_frac"] == np.mean(best == 0)
    # always L = 32: regret and mispredicts are what the per-chunk costs say
    fixed = np.full(len(n), 32)
    ev32 = P.evaluate(fixed, n, es, bits, cfg)
    got, opt, worse = 0.0, 0.0, 0
    for i in range(len(n)):
        c, coded, raw = S.best_choice(int(n[i]), int(es[i]), list(bits[i]), ocfg)
        b = min(min(coded), raw)
        got += coded[1]
        opt += b
        worse += coded[1] > b * 1.001
    assert abs(ev32["regret"] - (got / opt - 1.0)) < 1e-9
    assert ev32["mispredict"] == worse / len(n)


def test_chunking_covers_every_message_once():
    xs = [torch.zeros(n, dtype=dt) for n, dt in ((0, torch.float32), (16384, torch.float32),
                                                  (16385, torch.float32), (40000, torch.bfloat16),
                                                  (5, torch.bfloat16))]
    views, ebs = P.split_chunks(xs, [1e-3, 2e-3, 3e-3, 4e-3, 5e-3])
    lens = [v.numel() for v in views]
    assert lens == [16384, 16384, 1, 32768, 7232, 5]
    assert all(v.numel() * v.element_size() <= 65536 for v in views)
    assert ebs == [2e-3, 3e-3, 3e-3, 4e-3, 4e-3, 5e-3]
