"""Batched compression and decompression (many messages, one launch each)
against the CPU oracle, through the C ABI (needs a GB300).

Every message's stream inside the packed buffer must be byte-identical to the
oracle's stream of that message alone; decoded values must be bit-identical
to the oracle's decoding.  Messages mix FP32 and BF16, all block sizes and raw
storage, sizes from empty to several tiles with ragged tails."""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2308_05199_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES_MIX = [0, 1, 17, 1000, 2048, 16383, 16384, 16385, 70001, 300001, 5, 65536,
             131072 + 3, 40000]


@pytest.fixture(scope="session")
def zc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build()
    from paper_2308_05199_gb300 import zc as z
    z.zc_set_tile_chunks(8)
    return z


def np_of(t: torch.Tensor) -> np.ndarray:
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def mixed_messages(seed, sizes, blocks_from=(16, 32, 64, 128, 0)):
    """Student-t(3) messages with sigma log-uniform in [1e-4, 1e-1], eb = 1e-3 sigma,
    alternating FP32 / BF16, block sizes drawn from blocks_from (0 = raw)."""
    rng = np.random.default_rng(seed)
    xs, blocks, ebs = [], [], []
    for i, n in enumerate(sizes):
        sigma = float(10 ** rng.uniform(-4, -1))
        dt = torch.float32 if i % 2 == 0 else torch.bfloat16
        xs.append(W.student_t3(n, sigma, seed * 1000 + i, dtype=dt))
        blocks.append(int(blocks_from[rng.integers(len(blocks_from))]))
        ebs.append(1e-3 * sigma)
    return xs, blocks, ebs


def oracle_stream(x, blk, eb):
    a = np_of(x)
    return oracle.compress_raw(a) if blk == 0 else oracle.compress(a, eb, int(math.log2(blk)))


def check_against_oracle(b, xs, blocks, ebs):
    assert b.ws.status()[0] == 0, b.ws.status()
    streams = b.streams()
    off = b.msg_off.cpu().tolist()
    assert off[0] == 0
    for i, (x, blk, eb) in enumerate(zip(xs, blocks, ebs)):
        ref = oracle_stream(x, blk, eb)
        assert off[i + 1] - off[i] == len(ref), (i, x.numel(), blk)
        assert streams[i] == ref, (i, x.numel(), blk)


@pytest.mark.parametrize("chunks", [4, 8, 16])
@pytest.mark.parametrize("grid", [0, 152, 304])
def test_batch_streams_match_oracle(zc, chunks, grid):
    xs, blocks, ebs = mixed_messages(chunks * 7 + grid, SIZES_MIX)
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs, tile_chunks=chunks, grid=grid)
    b.run()
    check_against_oracle(b, xs, blocks, ebs)


@pytest.mark.parametrize("sizes", [[1 << 20] * 36 + [70001, 3],  # mean >= 2^15: 16-chunk tiles
                                   SIZES_MIX[:8] * 60])             # mean 6527: 4-chunk tiles
def test_batch_automatic_tile_size(zc, sizes):
    """With no tile size set, a batch plan takes the largest tile no larger
    than its mean message that keeps about 5/3 tiles per resident CTA: every
    stream still byte-equal to the oracle's."""
    try:
        assert zc.zc_set_tile_chunks(0) == 0
        xs, blocks, ebs = mixed_messages(77, sizes)
        b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs)
        b.run()
        check_against_oracle(b, xs, blocks, ebs)
    finally:
        zc.zc_set_tile_chunks(8)


def test_batch_single_message_equals_plain_compress(zc):
    x = W.student_t3(250001, 0.01, 7).cuda()
    b = zc.BatchCompress([x], [32], [1e-5])
    b.run()
    out, ob = zc.compress(x, 1e-5, 32)
    assert b.streams()[0] == zc.stream_bytes(out, ob)


def test_many_small_messages(zc):
    rng = np.random.default_rng(11)
    sizes = [int(v) for v in rng.integers(0, 5000, 1000)]
    xs, blocks, ebs = mixed_messages(12, sizes)
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs, grid=152)
    b.run()
    check_against_oracle(b, xs, blocks, ebs)


def test_raw_messages_from_unaligned_inputs(zc):
    big32 = W.student_t3(100003, 1.0, 3).cuda()
    big16 = W.student_t3(100003, 1.0, 4, dtype=torch.bfloat16).cuda()
    xs = [big32[1:], big16[1:], big16[3:50000], big32[2:7]]
    b = zc.BatchCompress(xs, [0, 0, 0, 0], [0.0] * 4)
    b.run()
    check_against_oracle(b, [x.cpu() for x in xs], [0] * 4, [0.0] * 4)


@pytest.mark.parametrize("chunks", [4, 16])
def test_coded_messages_from_unaligned_inputs(zc, chunks):
    """Coded messages whose data start off a 16-byte boundary beside 16-byte
    aligned ones, every block size, FP32 and BF16, in one launch: byte-exact
    streams."""
    big32 = W.student_t3(300007, 0.05, 13).cuda()
    big16 = W.student_t3(300007, 0.05, 14, dtype=torch.bfloat16).cuda()
    xs = [big32[1:], big16[1:], big32[4:], big16[8:200000], big32[2:], big16[3:], big32,
          big16[16:250001]]
    blocks = [32, 32, 16, 64, 128, 16, 64, 128]
    ebs = [1e-5] * len(xs)
    b = zc.BatchCompress(xs, blocks, ebs, tile_chunks=chunks)
    b.run()
    check_against_oracle(b, [x.cpu() for x in xs], blocks, ebs)


def test_batch_decompress_matches_oracle(zc):
    xs, blocks, ebs = mixed_messages(5, SIZES_MIX)
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs)
    b.run()
    outs = [torch.empty(x.numel(), dtype=(torch.float32, torch.bfloat16)[(i // 2) % 2],
                        device="cuda") for i, x in enumerate(xs)]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs)
    d.run()
    assert d.ws.status()[0] == 0, d.ws.status()
    for i, (x, blk, eb) in enumerate(zip(xs, blocks, ebs)):
        s = oracle_stream(x, blk, eb)
        code = 0 if outs[i].dtype == torch.float32 else 1
        np.testing.assert_array_equal(np_of(outs[i]), oracle.decompress(s, x.numel(), code))


def test_batch_decompress_wrong_count_is_a_format_error(zc):
    xs, blocks, ebs = mixed_messages(6, [1000, 5000])
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs)
    b.run()
    outs = [torch.empty(1000, device="cuda"), torch.empty(4999, device="cuda")]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs)
    d.run()
    assert d.ws.status()[0] == zc.ERR_FORMAT


def test_batch_capacity_error_never_writes_past_capacity(zc):
    xs = [W.student_t3(50000, 0.01, 20 + i) for i in range(3)]
    blocks, ebs = [32] * 3, [1e-6] * 3
    need = sum(len(oracle_stream(x, 32, 1e-6)) for x in xs)
    cap = need - 8192
    buf = torch.full((need,), 0xA5, dtype=torch.uint8, device="cuda")
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs, cap=cap, packed=buf)
    b.run()
    assert b.ws.status()[0] == zc.ERR_CAPACITY
    assert bool((buf[cap:] == 0xA5).all())


def test_batch_and_decompress_in_a_cuda_graph(zc):
    xs, blocks, ebs = mixed_messages(9, SIZES_MIX)
    gx = [x.cuda() for x in xs]
    s = torch.cuda.Stream()
    b = zc.BatchCompress(gx, blocks, ebs, grid=304)
    outs = [torch.empty(x.numel(), dtype=x.dtype, device="cuda") for x in xs]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs)
    torch.cuda.synchronize()
    b.run(s)  # ordinary calls first: they set the kernels' attributes
    d.run(s)
    s.synchronize()
    b.packed.zero_()
    b.msg_off.zero_()
    for o in outs:
        o.zero_()
    torch.cuda.synchronize()
    g = zc.Graph(s)
    with g.capture():
        b.run(s)
        d.run(s)
    for rep in range(3):
        if rep == 2:  # new values in the same buffers: the graph compresses them
            gx[9].mul_(-1.5)
            xs[9] = gx[9].cpu()
            torch.cuda.synchronize()
        g.launch()
        s.synchronize()
        check_against_oracle(b, xs, blocks, ebs)
        for i, (x, blk, eb) in enumerate(zip(xs, blocks, ebs)):
            code = 0 if x.dtype == torch.float32 else 1
            np.testing.assert_array_equal(
                np_of(outs[i]), oracle.decompress(oracle_stream(x, blk, eb), x.numel(), code))


def test_autotuner_picks_the_best_valid_candidate(zc):
    xs, blocks, ebs = mixed_messages(13, [300000, 120000, 5000, 70000, 1 << 18, 33333],
                                     blocks_from=(32, 32, 0))
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs)
    best, pts = b.autotune(tune_block=True, link_gbs=12.5, reps=2)
    assert best["status"] == 0 and best["block"] in (16, 32, 64, 128)
    ok = [p for p in pts if p["status"] == 0]
    assert len(ok) >= 12
    assert best["score_ms"] == min(p["score_ms"] for p in ok)
    for p in ok:
        assert p["score_ms"] == pytest.approx(p["ms"] + p["packed_bytes"] / 12.5e6, rel=1e-6)
    # the plan is left at the winner; its streams are the oracle's at the chosen block size
    b.run()
    tuned = [best["block"] if blk else 0 for blk in blocks]
    check_against_oracle(b, xs, tuned, ebs)


@pytest.mark.parametrize("chunks", [4, 8])
def test_grouped_batch_streams_and_layout(zc, chunks):
    """A grouped plan packs the streams by block size (raw, 16, 32, 64, 128;
    message order within a size): every message's stream, found at
    msg_off[i] with its header's length, is the oracle's; msg_off[M] is the
    packed total; decoding from the grouped buffer matches the oracle."""
    sizes = SIZES_MIX * 3
    xs, blocks, ebs = mixed_messages(40 + chunks, sizes)
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs, tile_chunks=chunks, grouped=True)
    for _ in range(2):  # the device rewrite of the tile starts repeats identically
        b.packed.zero_()
        b.run()
        assert b.ws.status()[0] == 0, b.ws.status()
        streams = b.streams()
        off = b.msg_off.cpu().tolist()
        refs = [oracle_stream(x, blk, eb) for x, blk, eb in zip(xs, blocks, ebs)]
        for i in range(len(xs)):
            assert streams[i] == refs[i], (i, xs[i].numel(), blocks[i])
        assert off[-1] == sum(len(r) for r in refs)
        cls = {0: 0, 16: 1, 32: 2, 64: 3, 128: 4}
        order = sorted(range(len(xs)), key=lambda i: off[i])
        keys = [(cls[blocks[i]], i) for i in order]
        assert keys == sorted(keys)  # grouped by size, message order within a size
    outs = [torch.empty(x.numel(), dtype=x.dtype, device="cuda") for x in xs]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs, grouped=True)
    d.run()
    assert d.ws.status()[0] == 0, d.ws.status()
    for i, x in enumerate(xs):
        code = 0 if x.dtype == torch.float32 else 1
        np.testing.assert_array_equal(np_of(outs[i]), oracle.decompress(refs[i], x.numel(), code))


def test_grouped_batch_follows_block_sizes_changed_on_the_device(zc):
    """The grouping is derived on the device at every launch, so block sizes
    written into the table after planning (as the selector does, here by a
    plain copy) take effect, also when the launch is replayed from a graph."""
    xs, blocks, ebs = mixed_messages(77, [3000, 20000, 70001, 5, 16384, 40000],
                                     blocks_from=(32,))
    dev = [x.cuda() for x in xs]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    b = zc.BatchCompress(dev, blocks, ebs, grouped=True, stream=s)
    b.run(s)
    s.synchronize()
    g = zc.Graph(s)
    with g.capture():
        b.run(s)
    # the same plan (same output buffer) with other block sizes, planned
    # elsewhere: copy its table over
    new_blocks = [128, 16, 0, 64, 16, 128]
    b2 = zc.BatchCompress(dev, new_blocks, ebs, cap=b.cap, packed=b.packed)
    torch.cuda.synchronize()
    b.table.copy_(b2.table)
    torch.cuda.synchronize()
    g.launch()
    s.synchronize()
    assert b.ws.status()[0] == 0
    off = b.msg_off.cpu().tolist()
    buf = b.packed[:off[-1]].cpu().numpy().tobytes()
    for i, (x, blk, eb) in enumerate(zip(xs, new_blocks, ebs)):
        ref = oracle_stream(x, blk, eb)
        assert buf[off[i]:off[i] + len(ref)] == ref, i
    assert off[-1] == sum(len(oracle_stream(x, blk, eb)) for x, blk, eb in zip(xs, new_blocks, ebs))


@pytest.mark.parametrize("block", [16, 32, 64, 128])
def test_batch_decompress_small_and_large_items(zc, block):
    """Items of up to four decode tiles (16384 elements each) are decoded
    without the width scan, larger ones with it: both sides of that boundary,
    every block size, FP32 and BF16, bit-identical to the oracle."""
    sizes = [1, 31, 16383, 16384, 16385, 32768 + 7, 49152, 65535, 65536, 65537, 81920, 81921,
             3, 40000]
    xs, _, ebs = mixed_messages(7, sizes)
    blocks = [block] * len(sizes)
    b = zc.BatchCompress([x.cuda() for x in xs], blocks, ebs)
    b.run()
    check_against_oracle(b, xs, blocks, ebs)
    outs = [torch.empty(x.numel(), dtype=x.dtype, device="cuda") for x in xs]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs)
    for _ in range(2):  # the second run reuses the workspace
        d.run()
        assert d.ws.status()[0] == 0, d.ws.status()
        for i, (x, eb) in enumerate(zip(xs, ebs)):
            s = oracle_stream(x, block, eb)
            code = 0 if x.dtype == torch.float32 else 1
            np.testing.assert_array_equal(np_of(outs[i]), oracle.decompress(s, x.numel(), code))


@pytest.mark.parametrize("n", [5000, 60000, 100000])
def test_batch_decompress_payload_size_mismatch_is_a_format_error(zc, n):
    """A header whose payload size disagrees with the width bytes is caught
    whether the item's offsets come from the width scan (100000 elements) or
    from its decoder CTAs (5000, 60000)."""
    xs, _, ebs = mixed_messages(8, [3000, n])
    b = zc.BatchCompress([x.cuda() for x in xs], [32, 32], ebs)
    b.run()
    off = b.msg_off.cpu().tolist()
    hdr = b.packed[off[1]:off[1] + 32].cpu().numpy().copy()
    pl = int(hdr[24:32].view(np.uint64)[0])
    assert pl >= 32
    hdr[24:32] = np.array([pl - 16], dtype=np.uint64).view(np.uint8)
    b.packed[off[1]:off[1] + 32] = torch.from_numpy(hdr).cuda()
    outs = [torch.empty(x.numel(), dtype=x.dtype, device="cuda") for x in xs]
    d = zc.BatchDecompress(b.packed, b.msg_off, outs)
    d.run()
    assert d.ws.status()[0] == zc.ERR_FORMAT
