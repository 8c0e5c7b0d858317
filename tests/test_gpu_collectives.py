"""Simulated Allreduce algorithms on the GPU (ring with its Allgather stage,
recursive doubling with remainder ranks) against the oracle: every rank's
result bit-identical (needs a GB300)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
EB = 1e-3


@pytest.fixture(scope="session")
def zc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build()
    from paper_2308_05199_gb300 import zc as z
    z.zc_set_tile_chunks(8)
    return z


def ranks_of(N, n, seed):
    r = np.random.default_rng(seed)
    return [(r.standard_normal(n) * 0.2).astype(np.float32) for _ in range(N)]


@pytest.mark.parametrize("P", [2, 3, 5, 8])
def test_ring_allreduce_matches_oracle(zc, P):
    from paper_2308_05199_gb300.collectives import RingAllreduce
    n = 3 * 16384 + 77
    xs = ranks_of(P, n, P)
    ring = RingAllreduce([torch.from_numpy(x).cuda() for x in xs], EB, 32)
    out = ring.run()
    assert ring.ws.status()[0] == 0
    ref, final = oracle.ring_allreduce(xs, EB, 5)
    for r in range(P):
        np.testing.assert_array_equal(out[r].cpu().numpy(), ref[r], err_msg=str(r))


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_recursive_doubling_matches_oracle(zc, N):
    from paper_2308_05199_gb300.collectives import RecursiveDoublingAllreduce
    n = 2 * 16384 + 5
    xs = ranks_of(N, n, 40 + N)
    rd = RecursiveDoublingAllreduce([torch.from_numpy(x).cuda() for x in xs], EB, 32)
    out = rd.run()
    assert rd.ws.status()[0] == 0
    ref = oracle.redoub_allreduce(xs, EB, 5)
    for i in range(N):
        np.testing.assert_array_equal(out[i].cpu().numpy(), ref[i], err_msg=str(i))


def test_collectives_replay_from_a_graph(zc):
    from paper_2308_05199_gb300.collectives import RingAllreduce, RecursiveDoublingAllreduce
    n = 40000
    xs = ranks_of(5, n, 7)
    s = torch.cuda.Stream()
    dev = [torch.from_numpy(x).cuda() for x in xs]
    torch.cuda.synchronize()
    ring = RingAllreduce(dev, EB, 64, stream=s)
    rd = RecursiveDoublingAllreduce(dev, EB, 64, stream=s)
    ring.run()
    rd.run()
    s.synchronize()
    g = zc.Graph(s)
    with g.capture():
        ring.run()
        rd.run()
    for o in ring.out + [rd.val]:
        o.zero_()
    torch.cuda.synchronize()
    g.launch()
    s.synchronize()
    ref_ring, _ = oracle.ring_allreduce(xs, EB, 6)
    ref_rd = oracle.redoub_allreduce(xs, EB, 6)
    for r in range(5):
        np.testing.assert_array_equal(ring.out[r].cpu().numpy(), ref_ring[r])
        np.testing.assert_array_equal(rd.out[r].cpu().numpy(), ref_rd[r])
    m = ring.model(12.5, reps=2)
    assert m["per_rank_ms"] > m["link_ms"] > 0 and m["launches"] == 6
    m = rd.model(12.5, reps=2)
    assert m["launches"] == 7 and m["bytes_sent_per_rank"] > 0
