"""Argument checks of every C-ABI entry point (CPU only).

Each call below fails a check that the library makes on the host before any
CUDA call, so it returns its status synchronously and never dereferences the
placeholder device addresses it is given."""
import ctypes

import numpy as np
import pytest

import oracle

FAKE = 1 << 20          # a 16-byte aligned placeholder address, never dereferenced
BIG_WS = 1 << 30        # workspace size that passes the size check


@pytest.fixture(scope="module")
def zc():
    from paper_2308_05199_gb300 import build as zbuild
    zbuild.build()
    from paper_2308_05199_gb300 import zc as z
    return z


def test_decompress_arguments(zc):
    d = zc.zc_decompress
    assert d(None, 4096, FAKE, 10, 0, FAKE, BIG_WS, None) == zc.ERR_ARG       # no stream
    assert d(FAKE + 8, 4096, FAKE, 10, 0, FAKE, BIG_WS, None) == zc.ERR_ARG   # stream not 16-aligned
    assert d(FAKE, 16, FAKE, 10, 0, FAKE, BIG_WS, None) == zc.ERR_ARG         # shorter than a header
    assert d(FAKE, 4096, None, 10, 0, FAKE, BIG_WS, None) == zc.ERR_ARG       # no output
    assert d(FAKE, 4096, FAKE, 10, 3, FAKE, BIG_WS, None) == zc.ERR_ARG       # unknown dtype
    assert d(FAKE, 4096, FAKE + 2, 10, 0, FAKE, BIG_WS, None) == zc.ERR_ARG   # FP32 out not 4-aligned
    assert d(FAKE, 4096, FAKE + 1, 10, 1, FAKE, BIG_WS, None) == zc.ERR_ARG   # BF16 out not 2-aligned
    assert d(FAKE, 4096, FAKE, 10, 0, None, BIG_WS, None) == zc.ERR_ARG       # no workspace
    assert d(FAKE, 4096, FAKE, 10, 0, FAKE + 4, BIG_WS, None) == zc.ERR_ARG   # workspace not aligned
    assert d(FAKE, 4096, FAKE, 10, 0, FAKE, 64, None) == zc.ERR_WORKSPACE     # workspace too small
    ws_small = zc.zc_workspace_bytes(1 << 16, 1)
    assert d(FAKE, 1 << 30, FAKE, 1 << 30, 0, FAKE, ws_small, None) == zc.ERR_WORKSPACE


def test_reduce_step_arguments(zc):
    def r(cin=FAKE, cin_cap=4096, local=FAKE, n=1000, eb=1e-3, block=32, out=FAKE, cap=1 << 16,
          ob=FAKE, sum_out=None, ws=FAKE, ws_bytes=BIG_WS):
        return zc.zc_reduce_step(cin, cin_cap, local, n, eb, block, out, cap, ob, sum_out, ws,
                                 ws_bytes, None)

    assert r(block=48) == zc.ERR_ARG
    assert r(local=None) == zc.ERR_ARG
    assert r(local=FAKE + 2) == zc.ERR_ARG                 # FP32 local chunk not 4-aligned
    assert r(out=None, sum_out=None) == zc.ERR_ARG         # nothing to produce
    assert r(cin=FAKE + 8) == zc.ERR_ARG
    assert r(cin_cap=31) == zc.ERR_ARG
    assert r(out=FAKE + 8) == zc.ERR_ARG
    assert r(ob=None) == zc.ERR_ARG                        # a stream needs its length word
    assert r(sum_out=FAKE + 2) == zc.ERR_ARG
    assert r(cap=32 + 16) == zc.ERR_CAPACITY               # below header + width bytes
    assert r(ws=None) == zc.ERR_ARG
    assert r(ws_bytes=64) == zc.ERR_WORKSPACE
    assert r(eb=0.0) == zc.ERR_ARG
    assert r(eb=float("inf")) == zc.ERR_ARG
    assert r(eb=1e-45) == zc.ERR_ARG                       # subnormal in FP32
    assert r(eb=3e38) == zc.ERR_ARG                        # 2 eb overflows FP32


def test_plan_reduce_arguments(zc):
    P = 3
    items = (zc.ZcReduceItem * P)()
    for it in items:
        it.cmp_in, it.local, it.cmp_out, it.sum_out, it.out_bytes = FAKE, FAKE, FAKE, None, FAKE
        it.n, it.cmp_in_cap, it.out_cap = 1000, 4096, 1 << 16
    plan = zc.ZcPlan()
    tb = zc.zc_plan_table_bytes(P)
    assert tb > 0 and zc.zc_plan_table_bytes(0) == 0

    def rc(p=P, eb=1e-3, block=32, table=FAKE, table_bytes=tb):
        return zc.zc_plan_reduce(plan, p, items, eb, block, table, table_bytes)

    assert rc(p=0) == zc.ERR_ARG
    assert rc(block=100) == zc.ERR_ARG
    assert rc(table=None) == zc.ERR_ARG
    assert rc(table=FAKE + 8) == zc.ERR_ARG
    assert rc(table_bytes=tb - 1) == zc.ERR_ARG
    assert rc(eb=-1.0) == zc.ERR_ARG
    items[1].cmp_out, items[1].sum_out = None, None
    assert rc() == zc.ERR_ARG
    items[1].cmp_out = FAKE
    items[2].out_cap = 40
    assert rc() == zc.ERR_CAPACITY
    items[2].out_cap = 1 << 16
    items[0].local = FAKE + 1
    assert rc() == zc.ERR_ARG
    items[0].local = FAKE
    items[0].cmp_in_cap = 8
    assert rc() == zc.ERR_ARG
    # a plan that was never filled in does not launch
    assert zc.zc_reduce_step_batch(zc.ZcPlan(), FAKE, BIG_WS, None) == zc.ERR_ARG


def test_scatter_pack_arguments(zc):
    P = 4
    counts = (ctypes.c_uint64 * P)(1000, 2000, 0, 3000)
    displs = (ctypes.c_uint64 * P)(0, 1000, 3000, 3000)
    cap = sum(zc.zc_max_compressed_bytes(int(c), 32) for c in counts)

    def sp(d_in=FAKE, dtype=0, p=P, mode=zc.EB_ABS, eb=1e-3, block=32, out=FAKE, out_cap=cap,
           seg=FAKE, ws=FAKE, ws_bytes=BIG_WS):
        return zc.zc_scatter_pack(d_in, dtype, p, counts, displs, mode, eb, block, out, out_cap,
                                  seg, ws, ws_bytes, None)

    assert sp(p=0) == zc.ERR_ARG
    assert sp(p=100000) == zc.ERR_ARG                      # more segments than a launch carries
    assert sp(block=8) == zc.ERR_ARG
    assert sp(dtype=2) == zc.ERR_ARG
    assert sp(mode=5) == zc.ERR_ARG
    assert sp(eb=float("nan")) == zc.ERR_ARG
    assert sp(out=None) == zc.ERR_ARG
    assert sp(out=FAKE + 4) == zc.ERR_ARG
    assert sp(seg=None) == zc.ERR_ARG
    assert sp(d_in=FAKE + 2) == zc.ERR_ARG                 # FP32 input not 4-aligned
    assert sp(d_in=None) == zc.ERR_ARG                     # counts > 0 with no input
    assert sp(out_cap=4 * 48 - 1) == zc.ERR_CAPACITY       # below every segment's header + widths
    assert sp(ws_bytes=64) == zc.ERR_WORKSPACE


def test_compress_variants_arguments(zc):
    h = zc.zc_compress_heads
    assert h(FAKE, 10, 0, 0, 1e-3, 24, FAKE, 4096, FAKE, FAKE, BIG_WS, None) == zc.ERR_ARG
    assert h(FAKE, 10, 0, 7, 1e-3, 32, FAKE, 4096, FAKE, FAKE, BIG_WS, None) == zc.ERR_ARG
    na = zc.zc_compress_noalloc
    assert na(FAKE, zc.NOALLOC_MAX_N + 1, 0, 0, 1e-3, 32, FAKE, 1 << 30, FAKE, FAKE, None) == zc.ERR_ARG
    assert na(FAKE, 1000, 0, 0, 1e-3, 32, FAKE, 1 << 20, FAKE, None, None) == zc.ERR_ARG
    mm = zc.zc_minmax
    assert mm(FAKE, 10, 5, FAKE, FAKE, BIG_WS, None) == zc.ERR_ARG


def test_selector_and_status_arguments(zc):
    assert zc.zc_mlp_forward(None, FAKE, FAKE, 4, FAKE, None) == zc.ERR_ARG
    assert zc.zc_mlp_forward(FAKE, FAKE, FAKE, -1, FAKE, None) == zc.ERR_ARG
    assert zc.zc_mlp_forward(FAKE, FAKE, None, 4, FAKE, None) == zc.ERR_ARG
    assert zc.zc_mlp_forward(FAKE, FAKE, None, 0, None, None) == zc.OK  # nothing to do
    assert zc.zc_mlp_scratch_bytes(0) == 0
    assert zc.zc_mlp_scratch_bytes(1) > 0
    sb = zc.zc_mlp_scratch_bytes(100)
    g = zc.zc_mlp_grad
    assert g(FAKE, FAKE, FAKE, FAKE, None, 0, FAKE, FAKE, FAKE, sb, None) == zc.ERR_ARG
    assert g(FAKE, FAKE, FAKE, FAKE, None, 100, FAKE, FAKE, FAKE, sb - 4, None) == zc.ERR_ARG
    assert g(FAKE, FAKE, FAKE, FAKE, None, 100, FAKE, FAKE, FAKE + 2, sb, None) == zc.ERR_ARG
    assert zc.zc_mlp_sgd(FAKE, None, FAKE, 0.1, 0.9, None) == zc.ERR_ARG
    empty = zc.ZcBatch()
    assert zc.zc_batch_chunk_stats(empty, FAKE, None) == zc.ERR_ARG
    cfg = zc.ZcSelectCfg()
    cfg.link_gbs, cfg.judge_log2 = 12.5, 1.0
    assert zc.zc_batch_select(empty, FAKE, FAKE, cfg, FAKE, None, None) == zc.ERR_ARG
    assert zc.zc_batch_select_timed(empty, FAKE, FAKE, FAKE, cfg, FAKE, None, None) == zc.ERR_ARG
    fake_plan = zc.ZcBatch()
    fake_plan.n_msgs, fake_plan.d_table = 1, FAKE
    # a time prediction needs a bits prediction and a judge of its own
    assert zc.zc_batch_select_timed(fake_plan, FAKE, None, FAKE, cfg, FAKE, None,
                                    None) == zc.ERR_ARG
    cfg.judge_time_log2 = -1.0
    assert zc.zc_batch_select_timed(fake_plan, FAKE, FAKE, FAKE, cfg, FAKE, None,
                                    None) == zc.ERR_ARG
    assert zc.zc_decompress_batch(empty, FAKE, BIG_WS, None) == zc.ERR_ARG
    assert zc.zc_compress_batch(empty, FAKE, BIG_WS, None) == zc.ERR_ARG
    assert zc.zc_graph_launch(None, None) == zc.ERR_ARG
    assert zc.zc_clear_device_status(None, None) == zc.ERR_ARG
    with pytest.raises(zc.ZcError):
        zc.zc_get_device_status(None, None)


def test_heads_bound_holds_on_extreme_data(zc):
    """zc_max_compressed_bytes_heads bounds every heads-apart stream the oracle
    writes: widest deltas (alternating extremes) and widest heads."""
    rng = np.random.default_rng(5)
    eb = 1.0
    for n in (1, 15, 16, 17, 1000, 4099):
        hi = float(2 ** 22 - 2)
        x = np.where(np.arange(n) % 2 == 0, hi, -hi).astype(np.float32) * (2 * eb)
        y = (rng.uniform(-1, 1, n) * hi * 2 * eb).astype(np.float32)
        for log2L in (4, 5, 6, 7):
            bound = zc.zc_max_compressed_bytes_heads(n, 1 << log2L)
            nb = (n + (1 << log2L) - 1) >> log2L
            assert bound == oracle.max_stream_bytes(n, log2L) + oracle.pad16(3 * nb)
            for v in (x, y):
                assert len(oracle.compress_heads(v, eb, log2L)) <= bound
    assert zc.zc_max_compressed_bytes_heads(10, 3) == 0
    assert zc.zc_max_compressed_bytes_heads(0, 32) == oracle.max_stream_bytes(0, 5)


def test_batch_set_grouped_arguments(zc):
    p = zc.ZcBatch()
    assert zc.zc_batch_set_grouped(None, 1) == zc.ERR_ARG
    assert zc.zc_batch_set_grouped(p, 2) == zc.ERR_ARG
    assert zc.zc_batch_set_grouped(p, -1) == zc.ERR_ARG
    p.decompress = 1                      # a decompression plan without stream offsets
    assert zc.zc_batch_set_grouped(p, 1) == zc.ERR_ARG
    p.d_msg_off = FAKE
    assert zc.zc_batch_set_grouped(p, 1) == zc.OK and p.grouped == 1
    assert zc.zc_batch_set_grouped(p, 0) == zc.OK and p.grouped == 0
