"""ctypes binding of libzc.so (include/zc.h): argument marshalling only.

Every function named ``zc_*`` here calls the C entry point of the same name
with raw device pointers; all work runs in the library's CUDA kernels.  PyTorch
supplies device memory and streams.  The library must have been built
(``paper_2308_05199_gb300.build``); if it is missing, the first call raises --
there is no fallback.

The helpers below the raw bindings (``Workspace``, ``compress``, ...) only
allocate torch tensors and forward to the raw calls.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

OK, ERR_ARG, ERR_RANGE, ERR_NONFINITE, ERR_CAPACITY, ERR_FORMAT, ERR_TIMEOUT, ERR_CUDA, \
    ERR_WORKSPACE, ERR_BOUNDS = range(10)
F32, BF16 = 0, 1
EB_ABS, EB_REL = 0, 1
HEADER = 32

_lock = threading.Lock()
_lib = None


class ZcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s returned zc status %d" % (where, status))
        self.status = status


class ZcReduceItem(ctypes.Structure):
    _fields_ = [("cmp_in", ctypes.c_void_p), ("local", ctypes.c_void_p),
                ("cmp_out", ctypes.c_void_p), ("sum_out", ctypes.c_void_p),
                ("out_bytes", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("cmp_in_cap", ctypes.c_uint64), ("out_cap", ctypes.c_uint64)]


class ZcPlan(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int), ("tile_chunks", ctypes.c_int), ("block", ctypes.c_int),
                ("has_input", ctypes.c_int), ("total_tiles", ctypes.c_uint64),
                ("total_chunks", ctypes.c_uint64), ("d_table", ctypes.c_void_p)]


RAW = 0  # zc_message.block: store the message verbatim


class ZcMessage(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("dtype", ctypes.c_int), ("block", ctypes.c_int), ("eb_abs", ctypes.c_double)]


class ZcBatch(ctypes.Structure):
    _fields_ = [("n_msgs", ctypes.c_int), ("tile_chunks", ctypes.c_int), ("grid", ctypes.c_int),
                ("decompress", ctypes.c_int), ("grouped", ctypes.c_int),
                ("total_tiles", ctypes.c_uint64),
                ("total_chunks", ctypes.c_uint64), ("d_table", ctypes.c_void_p),
                ("d_packed", ctypes.c_void_p), ("packed_cap", ctypes.c_size_t),
                ("d_msg_off", ctypes.c_void_p)]


class ZcTunePoint(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("tile_chunks", ctypes.c_int), ("grid", ctypes.c_int),
                ("status", ctypes.c_int), ("ms", ctypes.c_float),
                ("packed_bytes", ctypes.c_uint64), ("score_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ZcSelectCfg(ctypes.Structure):
    _fields_ = [("link_gbs", ctypes.c_float), ("ns_per_byte", ctypes.c_float * 4),
                ("raw_ns_per_byte", ctypes.c_float), ("judge_log2", ctypes.c_float),
                ("judge_time_log2", ctypes.c_float)]


N_STATS = 16
MLP_PARAMS = 5508


def lib_path() -> str:
    """The library this process loads: the release build, or the
    bounds-checked one when the environment sets ZC_LIBRARY=debug."""
    return _build.DEBUG_LIB if os.environ.get("ZC_LIBRARY") == "debug" else _build.LIB


def lib():
    """Load libzc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError("libzc.so is not built (%s); run "
                                   "paper_2308_05199_gb300.build.build()" % path)
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    c = ctypes
    vp, u64, sz, i32, dbl = c.c_void_p, c.c_uint64, c.c_size_t, c.c_int, c.c_double
    sig = {
        "zc_max_compressed_bytes": (sz, [u64, i32]),
        "zc_raw_stream_bytes": (sz, [u64, i32]),
        "zc_workspace_bytes": (sz, [u64, i32]),
        "zc_workspace_init": (i32, [vp, sz, vp]),
        "zc_minmax": (i32, [vp, u64, i32, vp, vp, sz, vp]),
        "zc_compress": (i32, [vp, u64, i32, i32, dbl, i32, vp, sz, vp, vp, sz, vp]),
        "zc_compress_heads": (i32, [vp, u64, i32, i32, dbl, i32, vp, sz, vp, vp, sz, vp]),
        "zc_max_compressed_bytes_heads": (sz, [u64, i32]),
        "zc_decompress": (i32, [vp, sz, vp, u64, i32, vp, sz, vp]),
        "zc_reduce_step": (i32, [vp, sz, vp, u64, dbl, i32, vp, sz, vp, vp, vp, sz, vp]),
        "zc_plan_table_bytes": (sz, [i32]),
        "zc_plan_reduce": (i32, [c.POINTER(ZcPlan), i32, c.POINTER(ZcReduceItem), dbl, i32, vp,
                                 sz]),
        "zc_reduce_step_batch": (i32, [c.POINTER(ZcPlan), vp, sz, vp]),
        "zc_scatter_pack": (i32, [vp, i32, i32, vp, vp, i32, dbl, i32, vp, sz, vp, vp, sz, vp]),
        "zc_compress_noalloc": (i32, [vp, u64, i32, i32, dbl, i32, vp, sz, vp, vp, vp]),
        "zc_batch_table_bytes": (sz, [i32]),
        "zc_batch_max_bytes": (sz, [i32, c.POINTER(ZcMessage)]),
        "zc_plan_compress_batch": (i32, [c.POINTER(ZcBatch), i32, c.POINTER(ZcMessage), i32, i32,
                                         vp, sz, vp, vp, sz]),
        "zc_compress_batch": (i32, [c.POINTER(ZcBatch), vp, sz, vp]),
        "zc_plan_decompress_batch": (i32, [c.POINTER(ZcBatch), i32, c.POINTER(ZcMessage), vp, sz,
                                           vp, vp, sz]),
        "zc_decompress_batch": (i32, [c.POINTER(ZcBatch), vp, sz, vp]),
        "zc_batch_set_grouped": (i32, [c.POINTER(ZcBatch), i32]),
        "zc_plan_decompress_streams": (i32, [c.POINTER(ZcBatch), i32, vp, vp,
                                             c.POINTER(ZcMessage), vp, sz]),
        "zc_autotune_batch": (i32, [i32, c.POINTER(ZcMessage), i32, dbl, i32, vp, sz, vp, vp, sz,
                                    vp, sz, vp, c.POINTER(ZcTunePoint), i32, c.POINTER(i32),
                                    c.POINTER(ZcTunePoint)]),
        "zc_batch_chunk_stats": (i32, [c.POINTER(ZcBatch), vp, vp]),
        "zc_mlp_forward": (i32, [vp, vp, vp, i32, vp, vp]),
        "zc_mlp_scratch_bytes": (sz, [i32]),
        "zc_mlp_grad": (i32, [vp, vp, vp, vp, vp, i32, vp, vp, vp, sz, vp]),
        "zc_mlp_sgd": (i32, [vp, vp, vp, c.c_float, c.c_float, vp]),
        "zc_batch_select": (i32, [c.POINTER(ZcBatch), vp, vp, c.POINTER(ZcSelectCfg), vp, vp,
                                  vp]),
        "zc_batch_select_timed": (i32, [c.POINTER(ZcBatch), vp, vp, vp, c.POINTER(ZcSelectCfg),
                                        vp, vp, vp]),
        "zc_graph_begin": (i32, [vp]),
        "zc_graph_end": (i32, [vp, c.POINTER(vp)]),
        "zc_graph_launch": (i32, [vp, vp]),
        "zc_graph_destroy": (None, [vp]),
        "zc_get_device_status": (i32, [vp, vp, c.POINTER(c.c_int), c.POINTER(u64)]),
        "zc_clear_device_status": (i32, [vp, vp]),
        "zc_set_wait_limit_ns": (None, [u64]),
        "zc_debug_withhold_tile": (None, [c.c_int64]),
        "zc_set_tile_chunks": (i32, [i32]),
        "zc_version": (c.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def exported_names():
    return ["zc_max_compressed_bytes", "zc_raw_stream_bytes", "zc_workspace_bytes",
            "zc_workspace_init", "zc_minmax", "zc_compress", "zc_compress_heads",
            "zc_max_compressed_bytes_heads", "zc_decompress", "zc_reduce_step",
            "zc_plan_table_bytes", "zc_plan_reduce", "zc_reduce_step_batch", "zc_scatter_pack",
            "zc_compress_noalloc", "zc_batch_table_bytes", "zc_batch_max_bytes",
            "zc_plan_compress_batch", "zc_compress_batch", "zc_plan_decompress_batch",
            "zc_decompress_batch", "zc_batch_set_grouped", "zc_plan_decompress_streams",
            "zc_autotune_batch", "zc_batch_chunk_stats", "zc_mlp_forward",
            "zc_mlp_scratch_bytes", "zc_mlp_grad", "zc_mlp_sgd", "zc_batch_select",
            "zc_batch_select_timed",
            "zc_graph_begin", "zc_graph_end",
            "zc_graph_launch", "zc_graph_destroy",
            "zc_get_device_status", "zc_clear_device_status", "zc_set_wait_limit_ns",
            "zc_debug_withhold_tile", "zc_set_tile_chunks", "zc_version"]


def _check(st: int, where: str):
    if st != OK:
        raise ZcError(st, where)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


def dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError("zc takes float32 or bfloat16 tensors, got %s" % t.dtype)


# ---- raw bindings (same names as the C ABI) --------------------------------

def zc_max_compressed_bytes(n: int, block: int) -> int:
    return lib().zc_max_compressed_bytes(n, block)


def zc_raw_stream_bytes(n: int, dtype: int) -> int:
    return lib().zc_raw_stream_bytes(n, dtype)


def zc_workspace_bytes(n_total: int, n_items: int = 1) -> int:
    return lib().zc_workspace_bytes(n_total, n_items)


def zc_workspace_init(d_ws: int, ws_bytes: int, stream: int) -> int:
    return lib().zc_workspace_init(d_ws, ws_bytes, stream)


def zc_minmax(d_in, n, dtype, d_minmax, d_ws, ws_bytes, stream) -> int:
    return lib().zc_minmax(d_in, n, dtype, d_minmax, d_ws, ws_bytes, stream)


def zc_compress(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes, d_ws,
                ws_bytes, stream) -> int:
    return lib().zc_compress(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap,
                             d_out_bytes, d_ws, ws_bytes, stream)


def zc_compress_heads(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes,
                      d_ws, ws_bytes, stream) -> int:
    return lib().zc_compress_heads(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap,
                                   d_out_bytes, d_ws, ws_bytes, stream)


def zc_max_compressed_bytes_heads(n: int, block: int) -> int:
    return lib().zc_max_compressed_bytes_heads(n, block)


def zc_decompress(d_cmp, cmp_cap, d_out, n, out_dtype, d_ws, ws_bytes, stream) -> int:
    return lib().zc_decompress(d_cmp, cmp_cap, d_out, n, out_dtype, d_ws, ws_bytes, stream)


def zc_reduce_step(d_cmp_in, cmp_in_cap, d_local, n, eb_abs, block, d_cmp_out, out_cap,
                   d_out_bytes, d_sum_out, d_ws, ws_bytes, stream) -> int:
    return lib().zc_reduce_step(d_cmp_in, cmp_in_cap, d_local, n, eb_abs, block, d_cmp_out,
                                out_cap, d_out_bytes, d_sum_out, d_ws, ws_bytes, stream)


def zc_plan_table_bytes(n_items: int) -> int:
    return lib().zc_plan_table_bytes(n_items)


def zc_plan_reduce(plan, P, h_items, eb_abs, block, d_table, table_bytes) -> int:
    return lib().zc_plan_reduce(ctypes.byref(plan), P, h_items, eb_abs, block, d_table,
                                table_bytes)


def zc_reduce_step_batch(plan, d_ws, ws_bytes, stream) -> int:
    return lib().zc_reduce_step_batch(ctypes.byref(plan), d_ws, ws_bytes, stream)


def zc_scatter_pack(d_in, dtype, P, h_counts, h_displs, eb_mode, eb_value, block, d_out,
                    out_cap, d_seg_off, d_ws, ws_bytes, stream) -> int:
    return lib().zc_scatter_pack(d_in, dtype, P, h_counts, h_displs, eb_mode, eb_value, block,
                                 d_out, out_cap, d_seg_off, d_ws, ws_bytes, stream)


def zc_compress_noalloc(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes,
                        d_status, stream) -> int:
    return lib().zc_compress_noalloc(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap,
                                     d_out_bytes, d_status, stream)


NOALLOC_MAX_N = 1 << 24


def zc_batch_table_bytes(n_msgs: int) -> int:
    return lib().zc_batch_table_bytes(n_msgs)


def zc_batch_max_bytes(n_msgs: int, h_msgs) -> int:
    return lib().zc_batch_max_bytes(n_msgs, h_msgs)


def zc_plan_compress_batch(plan, n_msgs, h_msgs, tile_chunks, grid, d_packed, packed_cap,
                           d_msg_off, d_table, table_bytes) -> int:
    return lib().zc_plan_compress_batch(ctypes.byref(plan), n_msgs, h_msgs, tile_chunks, grid,
                                        d_packed, packed_cap, d_msg_off, d_table, table_bytes)


def zc_compress_batch(plan, d_ws, ws_bytes, stream) -> int:
    return lib().zc_compress_batch(ctypes.byref(plan), d_ws, ws_bytes, stream)


def zc_plan_decompress_batch(plan, n_msgs, h_msgs, d_packed, packed_cap, d_msg_off, d_table,
                             table_bytes) -> int:
    return lib().zc_plan_decompress_batch(ctypes.byref(plan), n_msgs, h_msgs, d_packed,
                                          packed_cap, d_msg_off, d_table, table_bytes)


def zc_plan_decompress_streams(plan, n_msgs, h_streams, h_caps, h_msgs, d_table,
                               table_bytes) -> int:
    return lib().zc_plan_decompress_streams(ctypes.byref(plan), n_msgs, h_streams, h_caps,
                                            h_msgs, d_table, table_bytes)


def zc_batch_set_grouped(plan, grouped: int) -> int:
    return lib().zc_batch_set_grouped(plan, grouped)


def zc_decompress_batch(plan, d_ws, ws_bytes, stream) -> int:
    return lib().zc_decompress_batch(ctypes.byref(plan), d_ws, ws_bytes, stream)


def zc_autotune_batch(n_msgs, h_msgs, tune_block, link_gbs, reps, d_packed, packed_cap,
                      d_msg_off, d_table, table_bytes, d_ws, ws_bytes, stream, h_points,
                      max_points, n_points, best) -> int:
    return lib().zc_autotune_batch(n_msgs, h_msgs, tune_block, link_gbs, reps, d_packed,
                                   packed_cap, d_msg_off, d_table, table_bytes, d_ws, ws_bytes,
                                   stream, h_points, max_points, n_points, best)


def zc_batch_chunk_stats(plan, d_feat, stream) -> int:
    return lib().zc_batch_chunk_stats(ctypes.byref(plan), d_feat, stream)


def zc_mlp_forward(d_params, d_norm, d_x, B, d_y, stream) -> int:
    return lib().zc_mlp_forward(d_params, d_norm, d_x, B, d_y, stream)


def zc_mlp_scratch_bytes(B: int) -> int:
    return lib().zc_mlp_scratch_bytes(B)


def zc_mlp_grad(d_params, d_norm, d_x, d_t, d_idx, B, d_grad, d_loss, d_scratch, scratch_bytes,
                stream) -> int:
    return lib().zc_mlp_grad(d_params, d_norm, d_x, d_t, d_idx, B, d_grad, d_loss, d_scratch,
                             scratch_bytes, stream)


def zc_mlp_sgd(d_params, d_vel, d_grad, lr, momentum, stream) -> int:
    return lib().zc_mlp_sgd(d_params, d_vel, d_grad, lr, momentum, stream)


def zc_batch_select(plan, d_feat, d_pred, cfg, d_choice, d_counts, stream) -> int:
    return lib().zc_batch_select(ctypes.byref(plan), d_feat, d_pred, ctypes.byref(cfg), d_choice,
                                 d_counts, stream)


def zc_batch_select_timed(plan, d_feat, d_pred, d_pred_time, cfg, d_choice, d_counts,
                          stream) -> int:
    return lib().zc_batch_select_timed(ctypes.byref(plan), d_feat, d_pred, d_pred_time,
                                       ctypes.byref(cfg), d_choice, d_counts, stream)


def zc_graph_begin(stream) -> int:
    return lib().zc_graph_begin(stream)


def zc_graph_end(stream, graph_out) -> int:
    return lib().zc_graph_end(stream, graph_out)


def zc_graph_launch(graph, stream) -> int:
    return lib().zc_graph_launch(graph, stream)


def zc_graph_destroy(graph):
    lib().zc_graph_destroy(graph)


def zc_get_device_status(d_ws, stream):
    st, detail = ctypes.c_int(0), ctypes.c_uint64(0)
    r = lib().zc_get_device_status(d_ws, stream, ctypes.byref(st), ctypes.byref(detail))
    _check(r, "zc_get_device_status")
    return st.value, detail.value


def zc_clear_device_status(d_ws, stream) -> int:
    return lib().zc_clear_device_status(d_ws, stream)


def zc_set_wait_limit_ns(ns: int):
    lib().zc_set_wait_limit_ns(int(ns))


def zc_debug_withhold_tile(tile: int):
    lib().zc_debug_withhold_tile(int(tile))


def zc_set_tile_chunks(chunks: int) -> int:
    return lib().zc_set_tile_chunks(chunks)


def zc_version() -> str:
    return lib().zc_version().decode()


# ---- tensor helpers ----------------------------------------------------------

class Workspace:
    """Device workspace sized for ``n_total`` elements over ``n_items`` items."""

    def __init__(self, n_total: int, n_items: int = 1, device="cuda", stream=None):
        self.nbytes = zc_workspace_bytes(n_total, n_items)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        _check(zc_workspace_init(self.buf.data_ptr(), self.nbytes, _stream(stream)),
               "zc_workspace_init")

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def status(self, stream=None):
        return zc_get_device_status(self.ptr, _stream(stream))

    def clear(self, stream=None):
        _check(zc_clear_device_status(self.ptr, _stream(stream)), "zc_clear_device_status")


def empty_stream_buffer(n: int, block: int, device="cuda") -> torch.Tensor:
    return torch.empty(zc_max_compressed_bytes(n, block), dtype=torch.uint8, device=device)


def compress(x: torch.Tensor, eb: float, block: int = 32, mode: int = EB_ABS,
             ws: Workspace | None = None, out: torch.Tensor | None = None,
             out_bytes: torch.Tensor | None = None, stream=None, heads: bool = False):
    """Compress a contiguous FP32/BF16 tensor; returns (stream buffer, u64 length
    tensor).  heads: the heads-apart format (zc_compress_heads)."""
    x = x.contiguous()
    n = x.numel()
    ws = ws or Workspace(n, 1, x.device, stream)
    if out is None:
        cap = zc_max_compressed_bytes_heads(n, block) if heads else zc_max_compressed_bytes(n, block)
        out = torch.empty(cap, dtype=torch.uint8, device=x.device)
    out_bytes = out_bytes if out_bytes is not None else torch.zeros(1, dtype=torch.int64,
                                                                    device=x.device)
    fn, name = (zc_compress_heads, "zc_compress_heads") if heads else (zc_compress, "zc_compress")
    _check(fn(x.data_ptr(), n, dtype_code(x), mode, float(eb), block, out.data_ptr(), out.numel(),
              out_bytes.data_ptr(), ws.ptr, ws.nbytes, _stream(stream)), name)
    return out, out_bytes


def decompress(cmp: torch.Tensor, n: int, out_dtype=torch.float32, ws: Workspace | None = None,
               out: torch.Tensor | None = None, cmp_cap: int | None = None, stream=None):
    ws = ws or Workspace(n, 1, cmp.device, stream)
    out = out if out is not None else torch.empty(n, dtype=out_dtype, device=cmp.device)
    _check(zc_decompress(cmp.data_ptr(), cmp_cap if cmp_cap is not None else cmp.numel(),
                         out.data_ptr(), n, dtype_code(out), ws.ptr, ws.nbytes, _stream(stream)),
           "zc_decompress")
    return out


def reduce_step(cmp_in, local: torch.Tensor, eb_abs: float, block: int = 32, want_stream=True,
                want_sum=False, ws: Workspace | None = None, out=None, out_bytes=None,
                sum_out=None, stream=None):
    n = local.numel()
    ws = ws or Workspace(n, 1, local.device, stream)
    if want_stream:
        out = out if out is not None else empty_stream_buffer(n, block, local.device)
        out_bytes = out_bytes if out_bytes is not None else torch.zeros(1, dtype=torch.int64,
                                                                        device=local.device)
    if want_sum:
        sum_out = sum_out if sum_out is not None else torch.empty(n, dtype=torch.float32,
                                                                  device=local.device)
    _check(zc_reduce_step(_ptr(cmp_in), cmp_in.numel() if cmp_in is not None else 0,
                          local.data_ptr(), n, float(eb_abs), block,
                          _ptr(out) if want_stream else None, out.numel() if want_stream else 0,
                          _ptr(out_bytes) if want_stream else None,
                          _ptr(sum_out) if want_sum else None, ws.ptr, ws.nbytes,
                          _stream(stream)), "zc_reduce_step")
    return (out if want_stream else None), (out_bytes if want_stream else None), \
        (sum_out if want_sum else None)


def scatter_pack(x: torch.Tensor, counts, displs, eb: float, block: int = 32, mode: int = EB_ABS,
                 ws: Workspace | None = None, out=None, seg_off=None, stream=None):
    x = x.contiguous()
    P = len(counts)
    ws = ws or Workspace(int(sum(counts)), P, x.device, stream)
    cap = sum(zc_max_compressed_bytes(int(c), block) for c in counts)
    out = out if out is not None else torch.empty(cap, dtype=torch.uint8, device=x.device)
    seg_off = seg_off if seg_off is not None else torch.zeros(P + 1, dtype=torch.int64,
                                                              device=x.device)
    hc = (ctypes.c_uint64 * P)(*[int(c) for c in counts])
    hd = (ctypes.c_uint64 * P)(*[int(d) for d in displs])
    _check(zc_scatter_pack(x.data_ptr(), dtype_code(x), P, ctypes.addressof(hc),
                           ctypes.addressof(hd), mode, float(eb), block, out.data_ptr(),
                           out.numel(), seg_off.data_ptr(), ws.ptr, ws.nbytes, _stream(stream)),
           "zc_scatter_pack")
    return out, seg_off


def stream_bytes(out: torch.Tensor, out_bytes: torch.Tensor) -> bytes:
    """Copy a finished stream to the host (synchronises)."""
    n = int(out_bytes.item())
    return out[:n].cpu().numpy().tobytes()


# ---- batched compression -------------------------------------------------------

def _messages(n_msgs):
    return (ZcMessage * n_msgs)()


class BatchCompress:
    """Plan for compressing a list of FP32/BF16 tensors in one launch.

    ``blocks`` and ``ebs`` give each message's block size (RAW = verbatim) and
    absolute bound.  ``run()`` launches the plan; the streams are packed in
    ``self.packed`` at offsets ``self.msg_off`` (device, M + 1 entries)."""

    def __init__(self, xs, blocks, ebs, tile_chunks: int = 0, grid: int = 0,
                 ws: Workspace | None = None, cap: int | None = None, packed=None,
                 stream=None, grouped: bool = False):
        self.grouped = bool(grouped)
        self.xs = [x.contiguous() for x in xs]
        M = len(self.xs)
        dev = self.xs[0].device
        self.msgs = _messages(M)
        for i, x in enumerate(self.xs):
            m = self.msgs[i]
            m.in_ = x.data_ptr() if x.numel() else None
            m.out = None
            m.n = x.numel()
            m.dtype = dtype_code(x)
            m.block = int(blocks[i])
            m.eb_abs = float(ebs[i])
        self.n_total = sum(x.numel() for x in self.xs)
        self.ws = ws or Workspace(self.n_total, M, dev, stream)
        self.cap = cap if cap is not None else self.max_bytes(max_width=True)
        self.packed = packed if packed is not None else \
            torch.empty(max(self.cap, 16), dtype=torch.uint8, device=dev)
        self.msg_off = torch.zeros(M + 1, dtype=torch.int64, device=dev)
        self.table = torch.empty(zc_batch_table_bytes(M), dtype=torch.uint8, device=dev)
        self.plan = ZcBatch()
        self.replan(tile_chunks, grid)

    def max_bytes(self, max_width: bool = False) -> int:
        """Worst-case packed length; with max_width, at the block size whose
        worst case is largest (what an autotuner over block sizes needs)."""
        M = len(self.xs)
        if not max_width:
            return zc_batch_max_bytes(M, self.msgs)
        tmp = _messages(M)
        ctypes.memmove(tmp, self.msgs, ctypes.sizeof(tmp))
        best = 0
        for b in (16, 32, 64, 128):
            for i in range(M):
                tmp[i].block = self.msgs[i].block if self.msgs[i].block == RAW else b
            best = max(best, zc_batch_max_bytes(M, tmp))
        return best

    def replan(self, tile_chunks: int = 0, grid: int = 0, block: int = 0):
        if block:
            for i in range(len(self.xs)):
                if self.msgs[i].block != RAW:
                    self.msgs[i].block = block
        _check(zc_plan_compress_batch(self.plan, len(self.xs), self.msgs, tile_chunks, grid,
                                      self.packed.data_ptr(), self.cap, self.msg_off.data_ptr(),
                                      self.table.data_ptr(), self.table.numel()),
               "zc_plan_compress_batch")
        if self.grouped:
            _check(zc_batch_set_grouped(self.plan, 1), "zc_batch_set_grouped")

    def run(self, stream=None):
        _check(zc_compress_batch(self.plan, self.ws.ptr, self.ws.nbytes, _stream(stream)),
               "zc_compress_batch")
        return self.packed, self.msg_off

    def autotune(self, tune_block: bool = False, link_gbs: float = 0.0, reps: int = 3,
                 stream=None):
        """Run the library's autotuner; the plan is left at the best candidate.
        Returns (best, [all measured candidates]) as dicts."""
        pts = (ZcTunePoint * 64)()
        npts = ctypes.c_int(0)
        best = ZcTunePoint()
        _check(zc_autotune_batch(len(self.xs), self.msgs, int(tune_block), float(link_gbs), reps,
                                 self.packed.data_ptr(), self.cap, self.msg_off.data_ptr(),
                                 self.table.data_ptr(), self.table.numel(), self.ws.ptr,
                                 self.ws.nbytes, _stream(stream), pts, 64, ctypes.byref(npts),
                                 ctypes.byref(best)), "zc_autotune_batch")
        self.replan(best.tile_chunks, best.grid, best.block)
        return best.as_dict(), [pts[i].as_dict() for i in range(min(npts.value, 64))]

    def streams(self):
        """Host copies of every message's stream (synchronises)."""
        off = self.msg_off.cpu().tolist()
        buf = self.packed[:off[-1]].cpu().numpy().tobytes()
        M = len(self.xs)
        if not self.grouped:
            return [buf[off[i]:off[i + 1]] for i in range(M)]
        return [buf[off[i]:off[i] + stream_length(buf[off[i]:off[i] + 32])] for i in range(M)]


def stream_length(header: bytes) -> int:
    """Length of a stream from its 32-byte header (host bookkeeping): header,
    padded width bytes (and block heads when stored apart), padded payload."""
    h = bytes(header[:32])
    flags = h[6]
    nb = int.from_bytes(h[20:24], "little")
    payload = int.from_bytes(h[24:32], "little")
    pad = lambda v: (v + 15) // 16 * 16
    if flags & 1:
        return 32 + pad(payload)
    return 32 + pad(nb) + (pad(3 * nb) if flags & 2 else 0) + pad(payload)


class BatchDecompress:
    """Plan for decoding a packed buffer of M streams into ``outs`` (grouped:
    the streams were packed by a grouped compression plan)."""

    def __init__(self, packed: torch.Tensor, msg_off: torch.Tensor, outs,
                 ws: Workspace | None = None, stream=None, grouped: bool = False):
        self.outs = outs
        M = len(outs)
        self.msgs = _messages(M)
        for i, o in enumerate(outs):
            m = self.msgs[i]
            m.in_ = None
            m.out = o.data_ptr() if o.numel() else None
            m.n = o.numel()
            m.dtype = dtype_code(o)
            m.block = 0
            m.eb_abs = 0.0
        dev = packed.device
        self.packed, self.msg_off = packed, msg_off
        self.ws = ws or Workspace(sum(o.numel() for o in outs), M, dev, stream)
        self.table = torch.empty(zc_batch_table_bytes(M), dtype=torch.uint8, device=dev)
        self.plan = ZcBatch()
        _check(zc_plan_decompress_batch(self.plan, M, self.msgs, packed.data_ptr(), packed.numel(),
                                        msg_off.data_ptr(), self.table.data_ptr(),
                                        self.table.numel()), "zc_plan_decompress_batch")
        if grouped:
            _check(zc_batch_set_grouped(self.plan, 1), "zc_batch_set_grouped")

    def run(self, stream=None):
        _check(zc_decompress_batch(self.plan, self.ws.ptr, self.ws.nbytes, _stream(stream)),
               "zc_decompress_batch")
        return self.outs


class Graph:
    """A CUDA graph of zc calls recorded on a (non-default) torch stream:

        g = Graph(stream)
        with g.capture():
            batch.run(stream)
        g.launch()
    """

    def __init__(self, stream: torch.cuda.Stream):
        self.stream = stream
        self.handle = ctypes.c_void_p(None)

    def capture(self):
        g = self

        class _Ctx:
            def __enter__(self_inner):
                _check(zc_graph_begin(g.stream.cuda_stream), "zc_graph_begin")
                return g

            def __exit__(self_inner, et, ev, tb):
                st = zc_graph_end(g.stream.cuda_stream, ctypes.byref(g.handle))
                if et is None:
                    _check(st, "zc_graph_end")
                return False

        return _Ctx()

    def launch(self):
        _check(zc_graph_launch(self.handle, self.stream.cuda_stream), "zc_graph_launch")

    def __del__(self):
        try:
            if self.handle.value:
                zc_graph_destroy(self.handle)
                self.handle = ctypes.c_void_p(None)
        except Exception:
            pass
