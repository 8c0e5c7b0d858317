"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Streams must be byte-identical to the oracle's (one correct stream exists for
given input, bound and block size); decompressed values and FP32 sums must be
bit-identical.  Sizes span several tiles with ragged tails; edge cases cover
empty input, single elements, constant and zero data, exact ties of the
quantizer, and every error status.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

SIZES = [1, 31, 32, 33, 127, 1000, 1024, 2048 + 17, 3 * 4096 + 5, 100003]
BLOCKS = [16, 32, 64, 128]


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


def signal(kind, n, seed=0):
    g = np.random.default_rng(seed)
    i = np.arange(n)
    if kind == "sin":
        x = np.sin(2 * np.pi * 5.3 * i / max(n, 1)) + g.normal(0, 1e-3, n)
    elif kind == "walk":
        x = np.cumsum(g.normal(0, 0.01, n))
    elif kind == "tdist":
        x = g.standard_t(3, n) * 0.01
    elif kind == "zeros":
        x = np.zeros(n)
    elif kind == "const":
        x = np.full(n, -0.3333)
    else:
        x = i * 0.002
    return torch.from_numpy(x.astype(np.float32))


def gpu_compress(zc, x, eb, block, mode=0):
    ws = zc.Workspace(x.numel(), 1)
    out, ob = zc.compress(x.cuda(), eb, block, mode=mode, ws=ws)
    st = ws.status()
    return zc.stream_bytes(out, ob), st


@pytest.mark.parametrize("block", BLOCKS)
@pytest.mark.parametrize("kind", ["sin", "walk", "tdist", "zeros", "const", "ramp"])
def test_compress_stream_bytes_match_oracle(zc, block, kind):
    for n in SIZES:
        x = signal(kind, n, seed=n)
        s_gpu, st = gpu_compress(zc, x, 1e-3, block)
        assert st[0] == 0, st
        s_ref = oracle.compress(np_of(x), 1e-3, int(math.log2(block)))
        assert s_gpu == s_ref, (n, block, kind)


@pytest.mark.parametrize("chunks", [4, 8, 16])
def test_tile_size_does_not_change_the_stream(zc, chunks):
    x = signal("walk", 150000, 3)
    ref = oracle.compress(np_of(x), 1e-4, 5)
    try:
        assert zc.zc_set_tile_chunks(chunks) == 0
        for block in BLOCKS:
            s, st = gpu_compress(zc, x, 1e-4, block)
            assert st[0] == 0 and s == oracle.compress(np_of(x), 1e-4, int(math.log2(block)))
        assert gpu_compress(zc, x, 1e-4, 32)[0] == ref
        # decode and the ring step at this tile size too, every block size
        for block in BLOCKS:
            lg = int(math.log2(block))
            rb = oracle.compress(np_of(x), 1e-4, lg)
            cmp = torch.frombuffer(bytearray(rb), dtype=torch.uint8).cuda()
            np.testing.assert_array_equal(np_of(zc.decompress(cmp, x.numel())),
                                          oracle.decompress(rb, x.numel()))
            out, ob, sm = zc.reduce_step(cmp, x.cuda(), 1e-4, block, want_sum=True)
            r_s, r_sum = oracle.reduce_step(rb, np_of(x), 1e-4, lg, want_sum=True)
            assert zc.stream_bytes(out, ob) == r_s
            np.testing.assert_array_equal(np_of(sm), r_sum)
    finally:
        zc.zc_set_tile_chunks(8)


def test_automatic_tile_size_streams(zc):
    """With no tile size set the library picks one per launch (4 chunks for
    2^20 elements, 8 for 2^24, 16 for 2^25 on 152 SMs): whole streams still
    byte-equal to the oracle's, and the ring step and scatter pack at the
    same sizes."""
    try:
        assert zc.zc_set_tile_chunks(0) == 0
        for n in ((1 << 20) + 3, (1 << 24) + 5, (1 << 25) + 7):
            x = signal("walk", n, n)
            s, st = gpu_compress(zc, x, 1e-3, 32)
            assert st[0] == 0 and s == oracle.compress(np_of(x), 1e-3, 5), n
        n = (1 << 25) + 7
        x = signal("walk", n, 5)
        rb = oracle.compress(np_of(x), 1e-3, 5)
        cmp = torch.frombuffer(bytearray(rb), dtype=torch.uint8).cuda()
        out, ob, sm = zc.reduce_step(cmp, x.cuda(), 1e-3, 32, want_sum=True)
        r_s, r_sum = oracle.reduce_step(rb, np_of(x), 1e-3, 5, want_sum=True)
        assert zc.stream_bytes(out, ob) == r_s
        np.testing.assert_array_equal(np_of(sm), r_sum)
        # scatter pack: 8 segments of about 2^22 elements (16-chunk tiles)
        counts = [(1 << 22) - 3 * k for k in range(8)]
        displs = list(np.cumsum([0] + counts[:-1]))
        packed, seg = zc.scatter_pack(x.cuda(), counts, displs, 1e-3, 32)
        ref, ref_seg = oracle.scatter_pack(np_of(x), counts, displs, 1e-3, 5)
        seg_h = seg.cpu().numpy().astype(np.uint64)
        np.testing.assert_array_equal(seg_h, ref_seg)
        assert packed[: int(seg_h[-1])].cpu().numpy().tobytes() == ref
    finally:
        zc.zc_set_tile_chunks(8)


@pytest.mark.parametrize("block", BLOCKS)
def test_wide_and_narrow_blocks_mixed(zc, block):
    """Heavy-tailed data at a tight bound: blocks above 16 planes (one row per
    transpose) next to narrow ones (two rows per transpose), through
    compress, decompress and the ring step."""
    lg = int(math.log2(block))
    g = np.random.default_rng(17)
    scale = np.where(np.arange(70000) < 35000, 0.002, 100.0)  # narrow half, wide half
    x = np.clip(g.standard_t(2, 70000) * scale, -3000, 3000).astype(np.float32)
    xt = torch.from_numpy(x)
    s, st = gpu_compress(zc, xt, 1e-3, block)
    ref = oracle.compress(x, 1e-3, lg)
    assert st[0] == 0 and s == ref
    widths = np.frombuffer(ref[32:32 + (70000 + block - 1) // block], np.uint8)
    assert widths.max() > 16 and widths.min() < 15
    cmp = torch.frombuffer(bytearray(ref), dtype=torch.uint8).cuda()
    np.testing.assert_array_equal(np_of(zc.decompress(cmp, 70000)), oracle.decompress(ref, 70000))
    out, ob, sm = zc.reduce_step(cmp, xt.cuda(), 1e-3, block, want_sum=True)
    r_s, r_sum = oracle.reduce_step(ref, x, 1e-3, lg, want_sum=True)
    assert zc.stream_bytes(out, ob) == r_s
    np.testing.assert_array_equal(np_of(sm), r_sum)


def eight_plane_boundary_input(block=32, n_groups=400, tail=77, seed=23):
    """Quantized values built group by group (8 rows of 32): every group's
    largest sign-magnitude delta is drawn from one class: none, below 2^8
    (at most 8 planes), exactly 2^8 - 1 or 2^8 (either side of the 8-plane
    boundary), below 2^16, or wide.  Returns FP32 data whose quantization at
    eb = 1e-3 gives exactly these values, and the class of every group."""
    g = np.random.default_rng(seed)
    eb_f, two = oracle.qparams(1e-3)
    n = 256 * n_groups + tail
    cls = g.integers(0, 6, n_groups + 1)
    q = np.zeros(n, np.int64)
    for k in range(n_groups + 1):
        lo, hi = 256 * k, min(256 * (k + 1), n)
        if lo >= n:
            break
        c = cls[k]
        dmax = [0, 60, 127, 128, 30000, 100000][c]
        d = g.integers(-dmax, dmax + 1, hi - lo) if dmax else np.zeros(hi - lo, np.int64)
        if c in (2, 3):
            d[g.integers(0, hi - lo)] = dmax * (1 if g.random() < 0.5 else -1)
        # within every block the first value is a delta from 0
        for b in range(lo, hi, block):
            e = min(b + block, hi)
            q[b:e] = np.cumsum(d[b - lo:e - lo])
    x = (q.astype(np.float64) * np.float64(two)).astype(np.float32)
    return x, cls[: (n + 255) // 256]


@pytest.mark.parametrize("block", [32, 64, 128])
def test_eight_plane_groups(zc, block):
    """At L >= 32 a group whose values all fit 8 planes is encoded with four
    rows per transpose, otherwise two rows (16 planes) or one: groups on both
    sides of each boundary, a ragged tail, plain and heads-apart streams,
    decoding."""
    lg = int(math.log2(block))
    x, cls = eight_plane_boundary_input(block)
    n = x.size
    s, st = gpu_compress(zc, torch.from_numpy(x), 1e-3, block)
    ref = oracle.compress(x, 1e-3, lg)
    assert st[0] == 0 and s == ref
    widths = np.frombuffer(ref[32:32 + (n + block - 1) // block], np.uint8)
    per = 256 // block  # blocks of a group of 8 rows
    gmax = np.array([widths[i:i + per].max() for i in range(0, widths.size, per)])
    assert (gmax <= 7).mean() > 0.2 and (gmax == 8).any() and (gmax > 16).any()
    cmp = torch.frombuffer(bytearray(ref), dtype=torch.uint8).cuda()
    np.testing.assert_array_equal(np_of(zc.decompress(cmp, n)), oracle.decompress(ref, n))
    out, ob = zc.compress(torch.from_numpy(x).cuda(), 1e-3, block, heads=True)
    assert zc.stream_bytes(out, ob) == oracle.compress_heads(x, 1e-3, lg)
    out, ob, sm = zc.reduce_step(cmp, torch.from_numpy(x).cuda(), 1e-3, block, want_sum=True)
    r_s, r_sum = oracle.reduce_step(ref, x, 1e-3, lg, want_sum=True)
    assert zc.stream_bytes(out, ob) == r_s
    np.testing.assert_array_equal(np_of(sm), r_sum)


@pytest.mark.parametrize("block", BLOCKS)
def test_bf16_input(zc, block):
    x = (signal("tdist", 20011, 5) * 3).to(torch.bfloat16)
    s, st = gpu_compress(zc, x, 1e-3, block)
    assert st[0] == 0
    assert s == oracle.compress(np_of(x), 1e-3, int(math.log2(block)))


def test_quantizer_ties_and_near_ties(zc):
    """Values planted exactly on, and one ulp beside, half-integer multiples of
    2eb, at every magnitude up to |q| = 2^22: the GPU's fast/slow quantizer
    must agree with the exact rounding everywhere."""
    eb = 1e-3
    eb_f, two = oracle.qparams(eb)
    g = np.random.default_rng(1)
    k = np.concatenate([g.integers(-2000, 2000, 3000), g.integers(-(1 << 21), 1 << 21, 3000),
                        np.array([(1 << 22) - 1, -(1 << 22) + 1, 0, -1])])
    ties = ((k + 0.5) * np.float64(two)).astype(np.float32)
    x = np.concatenate([ties, np.nextafter(ties, np.float32(np.inf)),
                        np.nextafter(ties, np.float32(-np.inf)),
                        (k * np.float64(two)).astype(np.float32)])
    x = x[np.abs(x.astype(np.float64) / np.float64(two)) < (1 << 22) - 1]
    for block in BLOCKS:
        s, st = gpu_compress(zc, torch.from_numpy(x), eb, block)
        assert st[0] == 0
        assert s == oracle.compress(x, eb, int(math.log2(block)))


def test_quantizer_fast_path_edge(zc):
    """The fast rounding is trusted only where v = x * inv lies farther than
    |v| 2^-22 from a half-integer: that is about 2 ulp of v.  Values 1 to 8
    ulp on both sides of ties, at magnitudes from 1/8 to 2^21 (where the fast
    test switches off), under three bounds: the GPU must round every one of
    them exactly like the oracle."""
    g = np.random.default_rng(7)
    for eb in (1e-3, 3.7e-5, 0.25):
        eb_f, two = oracle.qparams(eb)
        k = np.concatenate([g.integers(-8, 8, 200), g.integers(-4096, 4096, 1500),
                            g.integers(-(1 << 21), 1 << 21, 1500),
                            np.array([(1 << 21) - 1, (1 << 21), -(1 << 21), (1 << 20) + 7])])
        ties = ((k + 0.5) * np.float64(two)).astype(np.float32)
        parts = [ties]
        for direction in (np.float32(np.inf), np.float32(-np.inf)):
            y = ties.copy()
            for _ in range(8):
                y = np.nextafter(y, direction)
                parts.append(y.copy())
        x = np.concatenate(parts)
        x = x[np.abs(x.astype(np.float64) / np.float64(two)) < (1 << 22) - 1]
        for block in (16, 32):
            s, st = gpu_compress(zc, torch.from_numpy(x), eb, block)
            assert st[0] == 0
            assert s == oracle.compress(x, eb, int(math.log2(block))), (eb, block)


def test_relative_bound(zc):
    from paper_2308_05199_gb300 import workloads
    x = workloads.grf_3d(side=48, seed=2000, device="cuda")
    xn = np_of(x)
    for rel in (1e-2, 1e-3, 1e-4):
        s, st = gpu_compress(zc, x, rel, 32, mode=1)
        assert st[0] == 0
        eb_abs = oracle.resolve_eb(xn, "rel", rel)
        assert s == oracle.compress(xn, eb_abs, 5)


def test_minmax(zc):
    x = signal("tdist", 77777, 9).cuda()
    ws = zc.Workspace(x.numel(), 1)
    mm = torch.zeros(2, dtype=torch.float32, device="cuda")
    assert zc.zc_minmax(x.data_ptr(), x.numel(), 0, mm.data_ptr(), ws.ptr, ws.nbytes,
                        torch.cuda.current_stream().cuda_stream) == 0
    lo, hi = oracle.minmax(np_of(x))
    assert mm[0].item() == lo and mm[1].item() == hi


@pytest.mark.parametrize("out_dtype", [torch.float32, torch.bfloat16])
def test_decompress_matches_oracle(zc, out_dtype):
    code = 0 if out_dtype == torch.float32 else 1
    for block in BLOCKS:
        for n in (1, 1000, 3 * 4096 + 5, 100003):
            x = signal("sin", n, n)
            s = oracle.compress(np_of(x), 1e-4, int(math.log2(block)))
            cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
            ws = zc.Workspace(n, 1)
            y = zc.decompress(cmp, n, out_dtype, ws=ws)
            assert ws.status()[0] == 0
            np.testing.assert_array_equal(np_of(y), oracle.decompress(s, n, code))


def test_decompress_raw_streams(zc):
    x = signal("tdist", 999, 1)
    for src in (np_of(x), np_of(x.to(torch.bfloat16))):
        s = oracle.compress_raw(src)
        cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
        for out_dtype, code in ((torch.float32, 0), (torch.bfloat16, 1)):
            y = zc.decompress(cmp, 999, out_dtype)
            np.testing.assert_array_equal(np_of(y), oracle.decompress(s, 999, code))


def test_round_trip_error_bound(zc):
    x = signal("tdist", 300000, 4).cuda()
    for block in BLOCKS:
        out, ob = zc.compress(x, 1e-4, block)
        y = zc.decompress(out, x.numel())
        err = (x.double() - y.double()).abs()
        lim = np.float32(1e-4).astype(np.float64) + y.abs().double() * 2.0 ** -24
        assert bool((err <= lim).all())


def test_empty_input(zc):
    x = torch.zeros(0, dtype=torch.float32)
    s, st = gpu_compress(zc, x, 1e-3, 32)
    assert st[0] == 0 and s == oracle.compress(np_of(x), 1e-3, 5)
    cmp = torch.frombuffer(bytearray(s), dtype=torch.uint8).cuda()
    assert zc.decompress(cmp, 0).numel() == 0


@pytest.mark.parametrize("block", BLOCKS)
def test_reduce_step_matches_oracle(zc, block):
    lg = int(math.log2(block))
    for n in (1, 1000, 3 * 4096 + 5, 65536 + 77):
        a, b = signal("walk", n, 1), signal("sin", n, 2)
        cin = oracle.compress(np_of(a), 1e-3, lg)
        ref_s, ref_sum = oracle.reduce_step(cin, np_of(b), 1e-3, lg, want_stream=True,
                                            want_sum=True)
        cin_t = torch.frombuffer(bytearray(cin), dtype=torch.uint8).cuda()
        ws = zc.Workspace(n, 1)
        out, ob, sm = zc.reduce_step(cin_t, b.cuda(), 1e-3, block, want_stream=True,
                                     want_sum=True, ws=ws)
        assert ws.status()[0] == 0
        assert zc.stream_bytes(out, ob) == ref_s
        np.testing.assert_array_equal(np_of(sm), ref_sum)
        # initial step (nothing received) and last step (sum only)
        out0, ob0, _ = zc.reduce_step(None, b.cuda(), 1e-3, block, ws=ws)
        assert zc.stream_bytes(out0, ob0) == oracle.reduce_step(None, np_of(b), 1e-3, lg)[0]
        _, _, last = zc.reduce_step(cin_t, b.cuda(), 1e-3, block, want_stream=False,
                                    want_sum=True, ws=ws)
        np.testing.assert_array_equal(np_of(last), ref_sum)


def run_ring_gpu(zc, ranks, eb_abs, block):
    """Simulated ring reduce-scatter: one batched launch per step over all ranks."""
    P = len(ranks)
    n = ranks[0].numel()
    bounds = oracle.chunk_bounds(n, P)
    dev = [r.cuda() for r in ranks]
    m_max = max(bounds[c + 1] - bounds[c] for c in range(P))
    cap = zc.zc_max_compressed_bytes(m_max, block)
    bufs = [[torch.empty(cap, dtype=torch.uint8, device="cuda") for _ in range(P)] for _ in range(2)]
    nbytes = torch.zeros(2, P, dtype=torch.int64, device="cuda")
    sums = [torch.empty(bounds[(r + 1) % P + 1] - bounds[(r + 1) % P], device="cuda")
            for r in range(P)]
    ws = zc.Workspace(n, P)
    tables = []
    history = []

    def chunk(r, c):
        return dev[r][bounds[c]:bounds[c + 1]]

    steps = []
    # step -1: initial compress of own chunk into buffer set 0
    items = (zc.ZcReduceItem * P)()
    for r in range(P):
        c = chunk(r, r)
        items[r] = zc.ZcReduceItem(None, c.data_ptr(), bufs[0][r].data_ptr(), None,
                                   nbytes[0, r].data_ptr(), c.numel(), 0, cap)
    steps.append(items)
    for t in range(P - 1):
        last = t == P - 2
        src, dst = t % 2, (t + 1) % 2
        items = (zc.ZcReduceItem * P)()
        for r in range(P):
            cidx = (r - 1 - t) % P
            c = chunk(r, cidx)
            items[r] = zc.ZcReduceItem(bufs[src][(r - 1) % P].data_ptr(), c.data_ptr(),
                                       None if last else bufs[dst][r].data_ptr(),
                                       sums[r].data_ptr() if last else None,
                                       None if last else nbytes[dst, r].data_ptr(), c.numel(),
                                       cap, cap)
        steps.append(items)
    stream = torch.cuda.current_stream().cuda_stream
    for k, items in enumerate(steps):
        plan = zc.ZcPlan()
        table = torch.empty(max(zc.zc_plan_table_bytes(P), 16), dtype=torch.uint8, device="cuda")
        tables.append(table)
        assert zc.zc_plan_reduce(plan, P, items, eb_abs, block, table.data_ptr(),
                                 table.numel()) == 0
        assert zc.zc_reduce_step_batch(plan, ws.ptr, ws.nbytes, stream) == 0
        if k < P - 1:
            buf = k % 2
            history.append([zc.stream_bytes(bufs[buf][r], nbytes[buf, r]) for r in range(P)])
    assert ws.status()[0] == 0
    return [np_of(s) for s in sums], history


@pytest.mark.parametrize("P", [2, 3, 5, 8])
def test_ring_reduce_scatter_matches_oracle(zc, P):
    g = np.random.default_rng(P)
    n = 4096 * P + 3 * P + 1
    base = np.sin(np.arange(n) * 0.001).astype(np.float32)
    ranks = [torch.from_numpy((base + g.normal(0, 0.01, n)).astype(np.float32)) for _ in range(P)]
    eb = 1e-3
    ref_sum, ref_hist = oracle.ring_reduce_scatter([np_of(r) for r in ranks], eb, 5)
    got_sum, got_hist = run_ring_gpu(zc, ranks, eb, 32)
    assert len(got_hist) == len(ref_hist)
    for t in range(len(ref_hist)):
        for r in range(P):
            assert got_hist[t][r] == ref_hist[t][r], (t, r)
    for r in range(P):
        np.testing.assert_array_equal(got_sum[r], ref_sum[r])


@pytest.mark.parametrize("block", [16, 32, 128])
def test_scatter_pack_matches_oracle(zc, block):
    x = signal("walk", 40000, 8)
    counts = [1000, 0, 12345, 33, 4096, 22526]
    displs = list(np.cumsum([0] + counts[:-1]))
    for xt in (x, x.to(torch.bfloat16)):
        packed, seg = zc.scatter_pack(xt.cuda(), counts, displs, 1e-3, block)
        ref, ref_seg = oracle.scatter_pack(np_of(xt), counts, displs, 1e-3, int(math.log2(block)))
        seg_h = seg.cpu().numpy().astype(np.uint64)
        np.testing.assert_array_equal(seg_h, ref_seg)
        assert packed[: int(seg_h[-1])].cpu().numpy().tobytes() == ref


def test_scatter_pack_relative_bound(zc):
    x = signal("tdist", 30000, 2)
    counts = [10000, 5000, 15000]
    displs = [0, 12000, 15000]  # overlapping / gapped segments: bound over their union
    packed, seg = zc.scatter_pack(x.cuda(), counts, displs, 1e-3, 32, mode=1)
    xs = np.concatenate([np_of(x)[d:d + c] for c, d in zip(counts, displs)])
    eb = oracle.resolve_eb(xs, "rel", 1e-3)
    ref, ref_seg = oracle.scatter_pack(np_of(x), counts, displs, eb, 5)
    assert packed[: int(seg[-1].item())].cpu().numpy().tobytes() == ref


# ---- error statuses -------------------------------------------------------

def test_nonfinite_and_range_errors(zc):
    x = signal("sin", 10000, 1)
    x[777] = float("nan")
    assert gpu_compress(zc, x, 1e-3, 32)[1][0] == zc.ERR_NONFINITE
    x[777] = float("inf")
    assert gpu_compress(zc, x, 1e-3, 32)[1][0] == zc.ERR_NONFINITE
    x[777] = 9e3  # 9e3 / 2e-3 > 2^22
    assert gpu_compress(zc, x, 1e-3, 32)[1][0] == zc.ERR_RANGE
    x[777] = 8e3
    assert gpu_compress(zc, x, 1e-3, 32)[1][0] == 0


def test_capacity_error_never_writes_past_capacity(zc):
    n = 50000
    x = signal("tdist", n, 3).cuda()
    need = len(oracle.compress(np_of(x), 1e-5, 5))
    cap = need - 4096
    buf = torch.full((cap + 4096,), 0xA5, dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws = zc.Workspace(n, 1)
    st = zc.zc_compress(x.data_ptr(), n, 0, 0, 1e-5, 32, buf.data_ptr(), cap, ob.data_ptr(),
                        ws.ptr, ws.nbytes, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert ws.status()[0] == zc.ERR_CAPACITY
    assert bool((buf[cap:] == 0xA5).all())
    assert ob.item() == need  # the length needed is still reported


def test_format_errors(zc):
    x = signal("sin", 5000, 1)
    good = bytearray(oracle.compress(np_of(x), 1e-3, 5))
    for pos, val in ((0, ord("X")), (5, 9), (32, 25), (20, 9)):
        b = bytearray(good)
        b[pos] = val
        cmp = torch.frombuffer(b, dtype=torch.uint8).cuda()
        ws = zc.Workspace(5000, 1)
        zc.decompress(cmp, 5000, ws=ws)
        assert ws.status()[0] == zc.ERR_FORMAT, pos
    # width bytes that disagree with the header's payload size, while every
    # plane still lies inside the buffer: the width scan's total decides
    short = bytearray(good)
    short[24:32] = (oracle.header(good)["payload"] - 16).to_bytes(8, "little")
    wider = bytearray(good)
    wider[32] = wider[32] + 1 if wider[32] < 24 else 23
    for b in (short, wider):
        cmp = torch.frombuffer(b, dtype=torch.uint8).cuda()
        ws = zc.Workspace(5000, 1)
        zc.decompress(cmp, 5000, ws=ws)
        assert ws.status()[0] == zc.ERR_FORMAT
    cmp = torch.frombuffer(bytearray(good), dtype=torch.uint8).cuda()
    ws = zc.Workspace(5000, 1)
    zc.decompress(cmp, 4999, ws=ws)  # wrong n
    assert ws.status()[0] == zc.ERR_FORMAT
    ws = zc.Workspace(5000, 1)
    zc.decompress(cmp, 5000, ws=ws, cmp_cap=len(good) - 32)  # truncated
    assert ws.status()[0] == zc.ERR_FORMAT


def test_uninitialised_workspace_is_refused(zc):
    x = signal("sin", 5000, 1).cuda()
    nbytes = zc.zc_workspace_bytes(5000, 1)
    ws = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")  # zeroed but not stamped
    out = torch.empty(zc.zc_max_compressed_bytes(5000, 32), dtype=torch.uint8, device="cuda")
    ob = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert zc.zc_compress(x.data_ptr(), 5000, 0, 0, 1e-3, 32, out.data_ptr(), out.numel(),
                          ob.data_ptr(), ws.data_ptr(), nbytes, s) == 0
    assert zc.zc_get_device_status(ws.data_ptr(), s)[0] == zc.ERR_WORKSPACE


def test_lookback_wait_times_out_and_recovers(zc):
    """A tile that never publishes its offset: its successors' bounded waits
    run out, ZC_ERR_TIMEOUT is recorded, the kernel returns, and the same
    workspace works normally afterwards."""
    n = 16384 * 12  # 12 encoder tiles of 8 chunks
    x = signal("walk", n, 2)
    ws = zc.Workspace(n, 1)
    try:
        zc.zc_set_wait_limit_ns(2_000_000)  # 2 ms
        zc.zc_debug_withhold_tile(3)
        zc.compress(x.cuda(), 1e-3, 32, ws=ws)
        st, detail = ws.status()
        assert st == zc.ERR_TIMEOUT and detail > 3
    finally:
        zc.zc_debug_withhold_tile(-1)
        zc.zc_set_wait_limit_ns(1_000_000_000)
    ws.clear()
    out, ob = zc.compress(x.cuda(), 1e-3, 32, ws=ws)
    assert ws.status()[0] == 0
    assert zc.stream_bytes(out, ob) == oracle.compress(np_of(x), 1e-3, 5)


def test_repeated_calls_reuse_workspace(zc):
    """The look-back flags carry a launch generation: hundreds of calls of
    different sizes on one workspace never see a stale flag."""
    ws = zc.Workspace(200000, 1)
    g = np.random.default_rng(0)
    for i in range(200):
        n = int(g.integers(1, 200000))
        x = signal("walk", n, i)
        out, ob = zc.compress(x.cuda(), 1e-3, 32, ws=ws)
        if i % 25 == 0:
            assert zc.stream_bytes(out, ob) == oracle.compress(np_of(x), 1e-3, 5)
    assert ws.status()[0] == 0
