"""Parity at the full workload sizes the bench times (needs a GB300).

The oracle cannot redo a 512^3 field or a 6.85 GB batch in seconds, but the
format's blocks are independent: block j of a stream is exactly the only
block of the stream of x[jL, (j + 1)L) at the same bound.  So sampled blocks
of the full-size GPU streams are compared byte for byte with the oracle's
one-block streams, sampled decoded values with the oracle's decoding, and
every element against the error bound.  The ring Allreduce is checked the same
way: a sampled block of chunk c takes the same path through the ring when it
sits alone in chunk c of small rank buffers.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_05199_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SAMPLES = 400

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

def block_index(stream: np.ndarray, nb: int, L: int):
    """Payload start (absolute) and size of every block, from the width bytes."""
    w = stream[32:32 + nb].astype(np.int64)
    size = np.where(w > 0, (w + 1) * (L // 8), 0)
    off = np.concatenate([[0], np.cumsum(size)])
    return w, 32 + oracle.pad16(nb) + off, size

def check_sampled_blocks(x_np, stream, eb, lg, rng, samples=SAMPLES):
    """Compare sampled blocks of a GPU stream with the oracle's one-block streams."""
    L = 1 << lg
    n = x_np.size
    nb = (n + L - 1) // L
    w, start, size = block_index(stream, nb, L)
    picks = np.unique(np.concatenate([rng.integers(0, nb, samples), [0, nb - 1]]))
    for j in picks:
        ref = np.frombuffer(oracle.compress(x_np[j * L:(j + 1) * L], eb, lg), np.uint8)
        assert ref[32] == w[j], (j, ref[32], w[j])
        got = stream[start[j]:start[j] + size[j]]
        np.testing.assert_array_equal(got, ref[48:48 + size[j]], err_msg="block %d" % j)
    return picks

def test_grf512_relative_bound_full_size(zc):
    """The bench's 512^3 field at REL 1e-3, L = 32: header, sampled blocks,
    sampled decoded values, the bound on every element."""
    x = W.grf_3d(side=512, seed=2000, device="cuda")
    n = x.numel()
    ws = zc.Workspace(n, 1)
    out, ob = zc.compress(x, 1e-3, 32, mode=zc.EB_REL, ws=ws)
    assert ws.status()[0] == 0
    stream = out[:int(ob.item())].cpu().numpy()
    hdr = oracle.header(stream.tobytes())
    mn, mx = float(x.min()), float(x.max())
    eb = oracle.eb_from_rel(1e-3, mn, mx)
    assert hdr["eb"] == np.float32(eb) and hdr["n"] == n and hdr["log2L"] == 5
    x_np = np_of(x)
    rng = np.random.default_rng(1)
    picks = check_sampled_blocks(x_np, stream, hdr["eb"], 5, rng)
    y = zc.decompress(out, n, ws=ws)
    assert ws.status()[0] == 0
    for j in picks[:100]:
        blk = x_np[j * 32:(j + 1) * 32]
        ref = oracle.decompress(oracle.compress(blk, hdr["eb"], 5), blk.size)
        np.testing.assert_array_equal(y[j * 32:j * 32 + blk.size].cpu().numpy(), ref)
    err = (y.double() - x.double()).abs()
    half_ulp = torch.finfo(torch.float32).eps / 2 * y.double().abs()
    assert bool((err <= float(np.float32(hdr["eb"])) + half_ulp).all())

def test_batch_1000_messages_full_size(zc):
    """The bench's 1000-message batch (6.85 GB): sampled messages, whole
    streams for the small ones, sampled blocks for the large ones."""
    specs = W.message_specs(1000)
    xs = [W.message(sp, device="cuda") for sp in specs]
    ebs = [sp["eb"] for sp in specs]
    b = zc.BatchCompress(xs, [32] * len(xs), ebs, grid=608)
    b.run()
    assert b.ws.status()[0] == 0
    off = b.msg_off.cpu().numpy()
    rng = np.random.default_rng(2)
    for i in rng.choice(len(xs), 24, replace=False):
        s = b.packed[int(off[i]):int(off[i + 1])].cpu().numpy()
        x_np = np_of(xs[i])
        if x_np.size <= 1 << 20:
            ref = oracle.compress(x_np, ebs[i], 5)
            assert s.tobytes() == ref, i
        else:
            hdr = oracle.header(s.tobytes())
            assert hdr["n"] == x_np.size and hdr["log2L"] == 5
            check_sampled_blocks(x_np, s, ebs[i], 5, rng, samples=60)

def test_ring_allreduce_8x8192sq_full_size(zc):
    """The bench's ring (8 ranks of 8192^2): every element within its bound,
    sampled blocks identical to the oracle's ring on one-block chunks."""
    from paper_2308_05199_gb300.collectives import RingAllreduce, chunk_bounds
    P, side = 8, 8192
    base = W.stacking_base(side=side, seed=3000, device="cuda")
    ranks = [W.stacking_rank(base, r, seed=3000) for r in range(P)]
    del base
    eb = 1e-3 * max(float(x.max() - x.min()) for x in ranks)
    ring = RingAllreduce(ranks, eb, 32)
    out = ring.run()
    assert ring.ws.status()[0] == 0
    n = ranks[0].numel()
    exact = torch.zeros(n, dtype=torch.float64, device="cuda")
    absum = torch.zeros_like(exact)
    for x in ranks:
        exact += x.double()
        absum += x.double().abs()
    eb32 = float(np.float32(eb))
    for r in range(P):
        slack = P * 2.0 ** -24 * absum
        assert bool(((out[r].double() - exact).abs() <= P * eb32 + slack).all()), r
    B = chunk_bounds(n, P)
    rng = np.random.default_rng(3)
    for _ in range(40):
        c = int(rng.integers(P))
        o = 32 * int(rng.integers((B[c + 1] - B[c]) // 32))
        small = []
        for r in range(P):
            a = np.zeros(P * 32, np.float32)
            a[c * 32:(c + 1) * 32] = ranks[r][B[c] + o:B[c] + o + 32].cpu().numpy()
            small.append(a)
        ref, _ = oracle.ring_allreduce(small, eb, 5)
        for r in range(P):
            np.testing.assert_array_equal(out[r][B[c] + o:B[c] + o + 32].cpu().numpy(),
                                          ref[r][c * 32:(c + 1) * 32], err_msg=str((c, o, r)))
