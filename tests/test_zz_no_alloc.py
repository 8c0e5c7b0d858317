"""zc_compress_noalloc: compression for callers that may not allocate device
memory (a collective's progress path, where cudaMalloc would synchronise the
device; a plugin whose host framework owns all device memory).  Its scratch
is a fixed array inside the library, so it must give the same stream as
zc_compress with a caller-supplied workspace -- on consecutive calls too,
since every call reuses what the previous one left in that array.

This file is collected last on purpose: a failure here leaves every other
test already run.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_05199_gb300 import build
    build.build()
    from paper_2308_05199_gb300 import zc as z
    return z


def _input(n, seed, dtype):
    g = np.random.default_rng(seed)
    x = np.cumsum(g.normal(0, 0.01, n)).astype(np.float32)
    return torch.from_numpy(x).to(dtype).cuda()


def _noalloc(zc, x, eb, block, mode):
    n = x.numel()
    cap = zc.zc_max_compressed_bytes(n, block)
    out = torch.empty(cap, dtype=torch.uint8, device="cuda")
    nbytes = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    st = zc.zc_compress_noalloc(x.data_ptr(), n, zc.dtype_code(x), mode, eb, block,
                                out.data_ptr(), cap, nbytes.data_ptr(), status.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == zc.OK
    torch.cuda.synchronize()
    assert int(status.item()) == zc.OK
    return zc.stream_bytes(out, nbytes)


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(zc):
    cases = [(300001, 1, torch.float32, 1e-3, 32, zc.EB_ABS),
             (123457, 2, torch.bfloat16, 1e-2, 64, zc.EB_REL),
             (zc.NOALLOC_MAX_N, 3, torch.float32, 1e-4, 16, zc.EB_ABS)]
    for n, seed, dtype, eb, block, mode in cases:
        x = _input(n, seed, dtype)
        ref_out, ref_n = zc.compress(x, eb, block, mode=mode)
        ref = zc.stream_bytes(ref_out, ref_n)
        assert _noalloc(zc, x, eb, block, mode) == ref
        assert _noalloc(zc, x, eb, block, mode) == ref


def test_noalloc_matches_the_oracle_on_the_smallest_case(zc):
    """Independently of zc_compress: the stream of a small ragged input is
    the oracle's byte for byte, on two calls in a row."""
    import oracle
    x = _input(5000 + 17, 4, torch.float32)
    ref = oracle.compress(x.cpu().numpy(), 1e-3, 5)
    assert _noalloc(zc, x, 1e-3, 32, zc.EB_ABS) == ref
    assert _noalloc(zc, x, 1e-3, 32, zc.EB_ABS) == ref


def test_noalloc_rejects_sizes_beyond_its_limit(zc):
    n = zc.NOALLOC_MAX_N + 1
    st = zc.zc_compress_noalloc(1 << 20, n, zc.F32, zc.EB_ABS, 1e-3, 32, 1 << 20, 1 << 30,
                                1 << 20, 1 << 20, torch.cuda.current_stream().cuda_stream)
    assert st == zc.ERR_ARG
