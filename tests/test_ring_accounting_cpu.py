"""Host-side accounting of the ring Allreduce (CPU only): the algorithmic
bytes the bench charges one ring (both arms use one formula), the oracle's
per-stage stream bookkeeping, and the ring's per-element error bounds."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2308_05199_gb300.collectives import (U32, chunk_bounds, ring_error_bounds,
                                                ring_target_bound)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_ring_bytes_hand_count_two_ranks():
    # n elements per rank, chunks of n/2.  First compression: each rank reads
    # its own chunk (4n/2 each, 4n in all) and writes S0.  The one step: every
    # rank reads S0's stream of its neighbour (S0 in all), a local chunk (4n
    # in all), writes its stream (S1) and its FP32 sum (4n in all).
    # Allgather: each rank decodes the other chunk's final stream (S1 in all)
    # into 4n/2 bytes (4n in all).
    n, S0, S1 = 1000, 700, 650
    want = (4 * n + S0) + (S0 + 4 * n + S1) + 4 * n + (S1 + 4 * n)
    assert _bench().ring_step_bytes(2, n, [S0, S1]) == want == 16 * n + 2 * S0 + 2 * S1


def test_ring_bytes_hand_count_three_ranks():
    # two steps; the Allgather decodes every final stream on the two other ranks
    n, S = 999, [600, 610, 620]
    want = (4 * n + S[0]) + (S[0] + 4 * n + S[1]) + (S[1] + 4 * n + S[2]) + 4 * n + \
        2 * (S[2] + 4 * n)
    assert _bench().ring_step_bytes(3, n, S) == want == 24 * n + 2 * S[0] + 2 * S[1] + 3 * S[2]


def test_oracle_stage_bytes_are_the_stream_lengths():
    r = np.random.default_rng(1)
    xs = [(r.standard_normal(3001) * 0.3).astype(np.float32) for _ in range(3)]
    stage = []
    _, final = oracle.ring_allreduce(xs, 1e-3, 5, stage_bytes=stage)
    assert len(stage) == 3
    B = chunk_bounds(3001, 3)
    first = sum(len(oracle.compress(xs[k][B[k]:B[k + 1]], 1e-3, 5)) for k in range(3))
    assert stage[0] == first
    assert stage[-1] == sum(map(len, final))
    # the bookkeeping changes nothing
    a, fa = oracle.ring_allreduce(xs, 1e-3, 5)
    b, fb = oracle.ring_allreduce(xs, 1e-3, 5, stage_bytes=[])
    assert fa == fb and all(np.array_equal(u, v) for u, v in zip(a, b))


def test_ring_error_bounds_closed_form():
    eb, A = 0.5, 3.0
    own, dec = ring_error_bounds(2, eb, A)
    # P = 2: one decode (eb + u |y|) and one addition (u |acc|), |y|, |acc| <= A + E
    assert own == pytest.approx((eb + 2 * U32 * A) / (1 - 2 * U32), rel=1e-15)
    assert own == pytest.approx(eb + 2 * U32 * (A + own), rel=1e-15)
    assert dec == pytest.approx(own + eb + U32 * (A + own + eb), rel=1e-15)
    own8, _ = ring_error_bounds(8, eb, 0.0)
    assert own8 == pytest.approx(7 * eb / (1 - 14 * U32), rel=1e-15)
    # arrays work elementwise
    o, d = ring_error_bounds(4, eb, np.array([0.0, A]))
    assert o[1] == pytest.approx(ring_error_bounds(4, eb, A)[0])


def test_target_covers_the_roundings_up_to_nine_ranks_only():
    eb = 1e-3
    for P in range(2, 10):
        for A in (0.0, 1.0, 1e6):
            own, _ = ring_error_bounds(P, eb, A)
            assert own <= ring_target_bound(P, eb, A) * (1 + 1e-5), (P, A)
    own, _ = ring_error_bounds(10, eb, 1e6)
    assert own > ring_target_bound(10, eb, 1e6)


@pytest.mark.parametrize("P", [2, 3, 5, 8])
def test_oracle_ring_within_its_bounds(P):
    r = np.random.default_rng(20 + P)
    n = 2048 * P + 7
    base = np.sin(np.arange(n) * 0.003)
    xs = [(base + r.normal(0, 0.01, n)).astype(np.float32) for _ in range(P)]
    eb = 1e-3
    out, _ = oracle.ring_allreduce(xs, eb, 5)
    exact = np.sum([x.astype(np.float64) for x in xs], 0)
    absum = np.sum([np.abs(x.astype(np.float64)) for x in xs], 0)
    eb_f = float(np.float32(eb))
    own, dec = ring_error_bounds(P, eb_f, absum)
    B = chunk_bounds(n, P)
    for k in range(P):
        err = np.abs(out[k].astype(np.float64) - exact)
        c = (k + 1) % P
        lim = dec.copy()
        lim[B[c]:B[c + 1]] = own[B[c]:B[c + 1]]
        assert np.all(err <= lim)
    # not vacuous: the errors reach a sizeable part of eb
    assert max(np.abs(out[k].astype(np.float64) - exact).max() for k in range(P)) > 0.3 * eb_f
