"""Pins of the simulated Allreduce algorithms of the oracle (ring with its
Allgather stage; recursive doubling with remainder ranks): closed forms for
small rank counts written from the codec's own compress / decompress calls,
consistency between ranks, and the error bounds against exact FP64 sums."""
import numpy as np
import pytest

import oracle

EB = 1e-3


def ranks_of(N, n, seed):
    r = np.random.default_rng(seed)
    return [(r.standard_normal(n) * 0.2).astype(np.float32) for _ in range(N)]


def d(s, n):
    return oracle.decompress(s, n)


def c(x):
    return oracle.compress(x, EB, 5)


def test_redoub_two_ranks_closed_form():
    x0, x1 = ranks_of(2, 3000, 1)
    out = oracle.redoub_allreduce([x0, x1], EB, 5)
    # each side adds the other's decoded buffer, decoded value first
    np.testing.assert_array_equal(out[0], (d(c(x1), 3000) + x0).astype(np.float32))
    np.testing.assert_array_equal(out[1], (d(c(x0), 3000) + x1).astype(np.float32))


def test_redoub_three_ranks_closed_form():
    x0, x1, x2 = ranks_of(3, 2000, 2)
    out = oracle.redoub_allreduce([x0, x1, x2], EB, 5)
    v1 = (d(c(x0), 2000) + x1).astype(np.float32)     # rank 1 absorbs rank 0
    o1 = (d(c(x2), 2000) + v1).astype(np.float32)     # new ranks 0 (=1) and 1 (=2) exchange
    o2 = (d(c(v1), 2000) + x2).astype(np.float32)
    np.testing.assert_array_equal(out[1], o1)
    np.testing.assert_array_equal(out[2], o2)
    np.testing.assert_array_equal(out[0], d(c(o1), 2000))  # sent back to rank 0


def test_redoub_schedule():
    assert oracle.redoub_plan(8) == (3, 0, list(range(8)))
    assert oracle.redoub_plan(6) == (2, 2, [1, 3, 4, 5])
    assert oracle.redoub_plan(7) == (2, 3, [1, 3, 5, 6])
    assert oracle.redoub_plan(2) == (1, 0, [0, 1])


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8, 9])
def test_redoub_error_bound(N):
    xs = ranks_of(N, 5000, 10 + N)
    out = oracle.redoub_allreduce(xs, EB, 5)
    exact = np.sum(np.array(xs, np.float64), 0)
    add = (N + 2) * np.finfo(np.float32).eps / 2 * np.sum(np.abs(np.array(xs, np.float64)), 0)
    for i in range(N):
        err = np.abs(out[i].astype(np.float64) - exact)
        assert np.all(err <= oracle.redoub_bound(N, i, EB) * 1.0000001 + 2 * add), (N, i)


def test_ring_two_ranks_closed_form():
    x0, x1 = ranks_of(2, 4001, 3)
    out, final = oracle.ring_allreduce([x0, x1], EB, 5)
    b = oracle.chunk_bounds(4001, 2)
    ch = lambda x, k: x[b[k]:b[k + 1]]
    # rank 1 owns chunk 0: decodes rank 0's chunk 0 and adds its own
    s0 = (d(c(ch(x0, 0)), b[1]) + ch(x1, 0)).astype(np.float32)
    s1 = (d(c(ch(x1, 1)), b[2] - b[1]) + ch(x0, 1)).astype(np.float32)
    np.testing.assert_array_equal(ch(out[1], 0), s0)
    np.testing.assert_array_equal(ch(out[0], 1), s1)
    assert final[0] == c(s0) and final[1] == c(s1)
    np.testing.assert_array_equal(ch(out[0], 0), d(c(s0), b[1]))
    np.testing.assert_array_equal(ch(out[1], 1), d(c(s1), b[2] - b[1]))


@pytest.mark.parametrize("P", [2, 3, 5, 8])
def test_ring_allreduce_bound_and_agreement(P):
    n = 6000 + P
    xs = ranks_of(P, n, 20 + P)
    out, final = oracle.ring_allreduce(xs, EB, 5)
    b = oracle.chunk_bounds(n, P)
    exact = np.sum(np.array(xs, np.float64), 0)
    add = P * np.finfo(np.float32).eps / 2 * np.sum(np.abs(np.array(xs, np.float64)), 0)
    rs, _ = oracle.ring_reduce_scatter(xs, EB, 5)
    for r in range(P):
        own = (r + 1) % P
        for k in range(P):
            sl = slice(b[k], b[k + 1])
            err = np.abs(out[r][sl].astype(np.float64) - exact[sl])
            bound = ((P - 1) if k == own else P) * EB
            assert np.all(err <= bound * 1.0000001 + add[sl]), (P, r, k)
        np.testing.assert_array_equal(out[r][b[own]:b[own + 1]], rs[r])
    # all ranks agree on every chunk they do not own
    for k in range(P):
        owner = (k - 1) % P
        vals = [out[r][b[k]:b[k + 1]] for r in range(P) if r != owner]
        for v in vals[1:]:
            np.testing.assert_array_equal(v, vals[0])


def test_redoub_bound_closed_form():
    """The recursive-doubling bound written out for small N (worst case of
    e_s = 2 e_(s-1) + eb over k steps, eb more for ranks that absorbed a
    neighbour first, one more for a folded rank's returned result)."""
    e = 1.0
    assert [oracle.redoub_bound(2, i, e) for i in range(2)] == [1, 1]
    assert [oracle.redoub_bound(4, i, e) for i in range(4)] == [3] * 4
    assert [oracle.redoub_bound(8, i, e) for i in range(8)] == [7] * 8
    assert [oracle.redoub_bound(3, i, e) for i in range(3)] == [4, 3, 3]
    assert [oracle.redoub_bound(6, i, e) for i in range(6)] == [8, 7, 8, 7, 7, 7]
