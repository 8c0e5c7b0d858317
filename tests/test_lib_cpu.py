"""The C-ABI library on the CPU: it builds for sm_103a, loads, exports every
function include/zc.h declares, and its host-side sizing rules agree with
the stream format.  No compute call (there is no GPU here)."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2308_05199_gb300 import build as zbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = zbuild.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "zc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(zc_[a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("zc_compress", "zc_decompress", "zc_reduce_step", "zc_scatter_pack",
                 "zc_reduce_step_batch", "zc_minmax", "zc_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2308_05199_gb300 import zc
    assert set(declared_functions()) <= set(zc.exported_names())


def test_sizing_matches_format(lib):
    lib.zc_max_compressed_bytes.restype = ctypes.c_size_t
    lib.zc_max_compressed_bytes.argtypes = [ctypes.c_uint64, ctypes.c_int]
    lib.zc_raw_stream_bytes.restype = ctypes.c_size_t
    lib.zc_raw_stream_bytes.argtypes = [ctypes.c_uint64, ctypes.c_int]
    lib.zc_workspace_bytes.restype = ctypes.c_size_t
    lib.zc_workspace_bytes.argtypes = [ctypes.c_uint64, ctypes.c_int]
    for n in (0, 1, 15, 16, 17, 1 << 20, (1 << 27) + 3):
        for log2L in (4, 5, 6, 7):
            assert lib.zc_max_compressed_bytes(n, 1 << log2L) == oracle.max_stream_bytes(n, log2L)
        assert lib.zc_raw_stream_bytes(n, 0) == 32 + (4 * n + 15) // 16 * 16
        assert lib.zc_raw_stream_bytes(n, 1) == 32 + (2 * n + 15) // 16 * 16
    assert lib.zc_max_compressed_bytes(100, 48) == 0
    a = lib.zc_workspace_bytes(1 << 20, 1)
    b = lib.zc_workspace_bytes(1 << 27, 1)
    c = lib.zc_workspace_bytes(1 << 27, 64)
    assert 0 < a < b < c and a % 256 == 0
    # one record set (8 u64) per 2048-element decode tile
    assert b >= 8 * 8 * ((1 << 27) // 2048)
    # the encoder CTAs' tile rings: 200 KB per 16 entries of a small
    # workspace, at most 608 CTAs' worth (124.5 MB) in a large one
    ring = 2 * 8 * 100 * 128
    assert a >= 8 * 8 * ((1 << 20) // 2048) + ring
    assert lib.zc_workspace_bytes(1 << 34, 1) - lib.zc_workspace_bytes(1 << 33, 1) < 9 * 8 * (1 << 24)
    assert b >= 608 * ring


def test_argument_errors_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    lib.zc_compress.restype = ctypes.c_int
    lib.zc_compress.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p]
    fake = 1 << 20  # never dereferenced: every call below fails its argument check
    # block size 48
    assert lib.zc_compress(fake, 10, 0, 0, 1e-3, 48, fake, 4096, fake, fake, 1 << 20, None) == 1
    # eb <= 0, NaN
    assert lib.zc_compress(fake, 10, 0, 0, 0.0, 32, fake, 4096, fake, fake, 1 << 20, None) == 1
    assert lib.zc_compress(fake, 10, 0, 0, float("nan"), 32, fake, 4096, fake, fake, 1 << 20,
                           None) == 1
    # misaligned output
    assert lib.zc_compress(fake, 10, 0, 0, 1e-3, 32, fake + 4, 4096, fake, fake, 1 << 20,
                           None) == 1
    # output too small for header + widths
    assert lib.zc_compress(fake, 1 << 20, 0, 0, 1e-3, 32, fake, 64, fake, fake, 1 << 24,
                           None) == 4
    # workspace too small
    assert lib.zc_compress(fake, 1 << 20, 0, 0, 1e-3, 32, fake, 1 << 23, fake, fake, 4096,
                           None) == 8
    lib.zc_set_tile_chunks.restype = ctypes.c_int
    assert lib.zc_set_tile_chunks(5) == 1
    assert lib.zc_set_tile_chunks(8) == 0
    assert lib.zc_set_tile_chunks(0) == 0  # chosen per launch (the default)


def test_batch_plan_argument_errors_without_gpu():
    """Batch planning validates every message before touching the GPU."""
    from paper_2308_05199_gb300 import zc as z
    fake = 1 << 20  # never dereferenced
    msgs = (z.ZcMessage * 2)()
    for m in msgs:
        m.in_, m.n, m.dtype, m.block, m.eb_abs = fake, 1000, 0, 32, 1e-3
    msgs[1].block = z.RAW
    plan = z.ZcBatch()
    tb = z.zc_batch_table_bytes(2)
    assert tb >= 2 * 64
    assert z.zc_batch_max_bytes(2, msgs) == (z.zc_max_compressed_bytes(1000, 32) +
                                             z.zc_raw_stream_bytes(1000, 0))

    def plan_rc(chunks=8, grid=0, cap=1 << 20, table=tb):
        return z.zc_plan_compress_batch(plan, 2, msgs, chunks, grid, fake, cap, fake, fake, table)

    assert plan_rc(chunks=5) == z.ERR_ARG
    assert plan_rc(grid=-1) == z.ERR_ARG
    assert plan_rc(table=tb - 1) == z.ERR_ARG
    assert plan_rc(cap=64) == z.ERR_CAPACITY  # below the headers, widths and raw payload
    msgs[0].block = 48
    assert plan_rc() == z.ERR_ARG
    msgs[0].block = 32
    msgs[0].eb_abs = 0.0
    assert plan_rc() == z.ERR_ARG
    msgs[0].eb_abs = 1e-3
    msgs[0].dtype = 7
    assert plan_rc() == z.ERR_ARG
    msgs[0].dtype = 1
    msgs[0].in_ = fake + 1  # BF16 input must be 2-byte aligned
    assert plan_rc() == z.ERR_ARG
    assert z.zc_plan_decompress_batch(plan, 2, msgs, fake + 8, 4096, fake, fake, tb) == z.ERR_ARG
    assert z.zc_graph_begin(None) == z.ERR_ARG
