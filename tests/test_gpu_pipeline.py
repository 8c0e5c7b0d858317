"""The encoder's tile pipeline at its limits (needs a GB300).

Every encoder CTA stages its tiles in a ring of its own inside the workspace
and stores each tile one or two tiles after encoding it, once its resolver
warp has placed it in the chain.  The grid is bounded by the rings the
workspace holds, so a small workspace runs few CTAs, each through many tiles:
every stream must still be byte-identical to the oracle's.  The same holds for
one CTA, for batched launches whose grid is 1, and for the fused ring step."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_05199_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def zc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build()
    from paper_2308_05199_gb300 import zc as z
    z.zc_set_tile_chunks(8)
    yield z
    z.zc_set_tile_chunks(8)


def np_of(t):
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def small_workspace(zc, n_small):
    """A workspace sized for n_small elements: few rings, few encoder CTAs."""
    return zc.Workspace(n_small, 1)


@pytest.mark.parametrize("chunks,n_small,n", [(8, 40000, 600001), (16, 1, 300001),
                                              (4, 1, 140001)])
def test_ring_limited_grid_streams_match_oracle(zc, chunks, n_small, n):
    """Workspaces whose rings allow 2 to 5 CTAs: 10 to 37 tiles per launch go
    through the same few CTAs."""
    zc.zc_set_tile_chunks(chunks)
    try:
        for dt, seed in ((torch.float32, 1), (torch.bfloat16, 2)):
            x = W.student_t3(n, 0.05, seed, dtype=dt).cuda()
            ws = small_workspace(zc, n_small)
            out, ob = zc.compress(x, 5e-5, 32, ws=ws)
            assert ws.status()[0] == 0, ws.status()
            assert zc.stream_bytes(out, ob) == oracle.compress(np_of(x), 5e-5, 5)
    finally:
        zc.zc_set_tile_chunks(8)


def test_ring_limited_relative_bound(zc):
    """Relative bound (range kernel first) with two encoder CTAs."""
    x = W.grf_3d(side=64, seed=5, device="cuda")
    ws = small_workspace(zc, 1)
    out, ob = zc.compress(x, 1e-3, 64, mode=zc.EB_REL, ws=ws)
    assert ws.status()[0] == 0
    s = zc.stream_bytes(out, ob)
    eb = oracle.header(s)["eb"]
    assert s == oracle.compress(np_of(x), eb, 6)


@pytest.mark.parametrize("chunks", [4, 8, 16])
def test_batch_with_one_cta(zc, chunks):
    """grid = 1: every tile of every message through one CTA's pipeline."""
    rng = np.random.default_rng(chunks)
    sizes = [0, 1, 17, 2048, 16385, 70001, 5, 40000, 131075]
    xs, blocks, ebs = [], [], []
    for i, n in enumerate(sizes):
        dt = torch.float32 if i % 2 == 0 else torch.bfloat16
        xs.append(W.student_t3(n, 0.01, 100 + i, dtype=dt).cuda())
        blocks.append(int((16, 32, 64, 128, 0)[rng.integers(5)]))
        ebs.append(1e-5)
    b = zc.BatchCompress(xs, blocks, ebs, tile_chunks=chunks, grid=1)
    b.run()
    assert b.ws.status()[0] == 0
    streams = b.streams()
    for i, (x, blk, eb) in enumerate(zip(xs, blocks, ebs)):
        a = np_of(x)
        ref = oracle.compress_raw(a) if blk == 0 else oracle.compress(a, eb, int(math.log2(blk)))
        assert streams[i] == ref, (i, x.numel(), blk)


def test_ring_step_with_few_ctas(zc):
    """The fused decode + add + encode step with 16-chunk tiles on a workspace
    that holds the input's decode slots but rings for only 16 CTAs (31 tiles):
    stream and FP32 sum equal the oracle's step."""
    n = 1000001
    a = W.student_t3(n, 0.02, 7).cuda()
    b = W.student_t3(n, 0.02, 8).cuda()
    eb = 2e-5
    cin, cb = zc.compress(a, eb, 32)
    s_in = zc.stream_bytes(cin, cb)
    zc.zc_set_tile_chunks(16)
    try:
        ws = zc.Workspace(235520, 1)  # 248 decode slots, 16 rings
        out, ob, total = zc.reduce_step(cin, b, eb, 32, want_sum=True, ws=ws)
        assert ws.status()[0] == 0, ws.status()
    finally:
        zc.zc_set_tile_chunks(8)
    ref_stream, ref_sum = oracle.reduce_step(np.frombuffer(s_in, np.uint8), np_of(b), eb, 5,
                                             want_sum=True)
    assert zc.stream_bytes(out, ob) == ref_stream
    np.testing.assert_array_equal(total.cpu().numpy(), ref_sum)
