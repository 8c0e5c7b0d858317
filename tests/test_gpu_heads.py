"""Heads-apart stream format on the GPU against the oracle (needs a GB300):
byte-identical streams from zc_compress_heads, bit-identical decoding by
zc_decompress of the oracle's heads-apart streams."""
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

SIZES = [1, 31, 32, 33, 1000, 2048 + 17, 16384 * 3 + 5, 100003]


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


def signal(kind, n, seed):
    r = np.random.default_rng(seed)
    if kind == "offset_walk":
        x = 37.0 + np.cumsum(r.normal(0, 0.01, n))
    elif kind == "negative_offset":
        x = -1200.0 + r.normal(0, 0.05, n)
    elif kind == "tdist":
        x = r.standard_t(3, n) * 0.01
    elif kind == "zeros":
        x = np.zeros(n)
    else:
        x = np.full(n, 3.25)
    return torch.from_numpy(x.astype(np.float32))


@pytest.mark.parametrize("block", [16, 32, 64, 128])
@pytest.mark.parametrize("kind", ["offset_walk", "negative_offset", "tdist", "zeros", "const"])
def test_heads_streams_match_oracle(zc, block, kind):
    for n in SIZES:
        x = signal(kind, n, n)
        out, ob = zc.compress(x.cuda(), 1e-3, block, heads=True)
        s = zc.stream_bytes(out, ob)
        assert s == oracle.compress_heads(np_of(x), 1e-3, int(math.log2(block))), (n, block, kind)


@pytest.mark.parametrize("block", [16, 32, 64, 128])
def test_heads_bf16_and_relative_bound(zc, block):
    x = signal("offset_walk", 50001, 3).to(torch.bfloat16)
    ws = zc.Workspace(x.numel(), 1)
    out, ob = zc.compress(x.cuda(), 1e-3, block, mode=zc.EB_REL, ws=ws, heads=True)
    assert ws.status()[0] == 0
    a = np_of(x)
    eb = oracle.resolve_eb(a, "rel", 1e-3)
    assert zc.stream_bytes(out, ob) == oracle.compress_heads(a, eb, int(math.log2(block)))


@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_decompress_heads_streams(zc, out_dtype):
    code = 0 if out_dtype == torch.float32 else 1
    for block in (16, 32, 64, 128):
        for n in (1, 1000, 3 * 16384 + 5, 100003):
            x = signal("negative_offset", n, n + block)
            s = oracle.compress_heads(np_of(x), 1e-3, int(math.log2(block)))
            cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
            ws = zc.Workspace(n, 1)
            y = zc.decompress(cmp, n, out_dtype, ws=ws)
            assert ws.status()[0] == 0
            np.testing.assert_array_equal(np_of(y), oracle.decompress(s, n, code))


def test_heads_save_on_offset_data(zc):
    x = signal("offset_walk", 1 << 20, 9).cuda()
    a, na = zc.compress(x, 1e-3, 32)
    b, nb = zc.compress(x, 1e-3, 32, heads=True)
    assert nb.item() < 0.6 * na.item()


def test_fused_step_rejects_heads_streams(zc):
    x = signal("offset_walk", 5000, 4)
    s = oracle.compress_heads(np_of(x), 1e-3, 5)
    cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
    ws = zc.Workspace(5000, 1)
    zc.reduce_step(cmp, x.cuda(), 1e-3, 32, ws=ws)
    assert ws.status()[0] == zc.ERR_FORMAT


def test_heads_capacity_covers_heads_area(zc):
    x = signal("tdist", 4096, 2).cuda()
    out = torch.empty(32 + 128 + 16, dtype=torch.uint8, device="cuda")  # no room for the heads
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = zc.Workspace(4096, 1)
    st = zc.zc_compress_heads(x.data_ptr(), 4096, 0, 0, 1e-3, 32, out.data_ptr(), out.numel(),
                              ob.data_ptr(), ws.ptr, ws.nbytes,
                              torch.cuda.current_stream().cuda_stream)
    assert st == zc.ERR_CAPACITY


@pytest.mark.parametrize("block", [16, 32, 64, 128])
@pytest.mark.parametrize("kind", ["offset_walk", "tdist", "tdist_wide"])
def test_decompress_heads_narrow_and_wide_units(zc, block, kind):
    """Heads-apart streams whose units have at most 11 planes per block
    (decoded two rows per integer scan, the heads added after it) and wider
    ones (one row per scan), and streams that mix both, decode bit for bit
    as the oracle does."""
    for n in (2048 * 8 + 3, 100003):
        x = signal("tdist" if kind == "tdist_wide" else kind, n, n + block)
        if kind == "tdist_wide":
            x = x * 300.0  # deltas beyond 1023 levels in most units
        a = np_of(x)
        s = oracle.compress_heads(a, 1e-3, int(math.log2(block)))
        cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
        for out_dtype, code in ((torch.float32, 0), (torch.bfloat16, 1)):
            ws = zc.Workspace(n, 1)
            y = zc.decompress(cmp, n, out_dtype, ws=ws)
            assert ws.status()[0] == 0
            np.testing.assert_array_equal(np_of(y), oracle.decompress(s, n, code))
