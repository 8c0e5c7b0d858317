"""CPU oracle for the error-bounded codec and its collective steps.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports it, and it shares no code with the
CUDA path: ``zc_oracle.c`` is plain C compiled with ``-O2 -ffp-contract=off``
so its FP32 quantization performs exactly the operations the method states,
one rounding each.

Functions follow gZCCL (arXiv 2308.05199): the codec of Sec. 3.3.2 (an
error-bounded compressor), the ring reduce-scatter step of
Sec. 3.2.3 / 3.3.3 (decompress, add, recompress) and the per-destination
scatter pack of Sec. 3.3.4.  The codec internals the paper leaves open are
fixed in ``zc_oracle.c``'s header comment.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_RANGE, ERR_NONFINITE, ERR_CAPACITY, ERR_FORMAT = 0, 1, 2, 3, 4, 5
F32, BF16 = 0, 1
HEADER = 32


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no SIMD flags, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    c = ctypes
    u64p = c.POINTER(c.c_uint64)
    L.zco_qparams.argtypes = [c.c_double, c.POINTER(c.c_float), c.POINTER(c.c_float)]
    L.zco_minmax.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.POINTER(c.c_float),
                             c.POINTER(c.c_float)]
    L.zco_eb_from_rel.argtypes = [c.c_double, c.c_float, c.c_float]
    L.zco_eb_from_rel.restype = c.c_double
    L.zco_quantize.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_double, c.c_void_p, u64p]
    L.zco_encode_q.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_float, c.c_int, c.c_void_p,
                               c.c_uint64, u64p]
    L.zco_compress.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_double, c.c_int, c.c_void_p,
                               c.c_uint64, u64p, u64p]
    L.zco_compress_raw.argtypes = [c.c_void_p, c.c_uint64, c.c_int, c.c_void_p, c.c_uint64, u64p]
    L.zco_encode_q_heads.argtypes = L.zco_encode_q.argtypes
    L.zco_compress_heads.argtypes = L.zco_compress.argtypes
    L.zco_decode_q.argtypes = [c.c_void_p, c.c_uint64, c.c_void_p, c.c_uint64]
    L.zco_decompress.argtypes = [c.c_void_p, c.c_uint64, c.c_void_p, c.c_uint64, c.c_int]
    L.zco_parse_header.argtypes = [c.c_void_p, c.c_uint64, c.POINTER(c.c_int),
                                   c.POINTER(c.c_int), c.POINTER(c.c_int), u64p,
                                   c.POINTER(c.c_float), c.POINTER(c.c_uint32), u64p]
    L.zco_reduce_step.argtypes = [c.c_void_p, c.c_uint64, c.c_void_p, c.c_uint64, c.c_double,
                                  c.c_int, c.c_void_p, c.c_uint64, u64p, c.c_void_p, u64p]
    L.zco_scatter_pack.argtypes = [c.c_void_p, c.c_int, c.c_int, c.c_void_p, c.c_void_p,
                                   c.c_double, c.c_int, c.c_void_p, c.c_uint64, c.c_void_p]


class OracleError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        super().__init__("oracle status %d %s" % (status, where))
        self.status = status


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _dtype_code(x: np.ndarray) -> int:
    """f32 arrays are FP32; uint16 arrays carry BF16 bit patterns."""
    if x.dtype == np.float32:
        return F32
    if x.dtype == np.uint16:
        return BF16
    raise TypeError("oracle takes float32 or uint16 (bf16 bits), got %s" % x.dtype)


def pad16(v: int) -> int:
    return (v + 15) & ~15


def max_stream_bytes(n: int, log2L: int) -> int:
    """Largest stream the encoder can emit: every block at width 24."""
    L = 1 << log2L
    nb = (n + L - 1) // L
    return HEADER + pad16(nb) + pad16(nb * 25 * L // 8)


def qparams(eb_abs: float):
    """(eb, 2 eb) as FP32 values."""
    e, t = ctypes.c_float(), ctypes.c_float()
    st = lib().zco_qparams(float(eb_abs), ctypes.byref(e), ctypes.byref(t))
    if st:
        raise OracleError(st, "qparams")
    return e.value, t.value


def minmax(x: np.ndarray):
    x = np.ascontiguousarray(x)
    lo, hi = ctypes.c_float(), ctypes.c_float()
    st = lib().zco_minmax(_ptr(x), x.size, _dtype_code(x), ctypes.byref(lo), ctypes.byref(hi))
    if st:
        raise OracleError(st, "minmax")
    return lo.value, hi.value


def eb_from_rel(rel: float, mn: float, mx: float) -> float:
    return lib().zco_eb_from_rel(float(rel), float(mn), float(mx))


def resolve_eb(x: np.ndarray, mode: str, value: float) -> float:
    """Absolute bound for ``mode`` 'abs' or 'rel' (relative to max - min)."""
    if mode == "abs":
        return float(value)
    mn, mx = minmax(x) if x.size else (0.0, 0.0)
    return eb_from_rel(value, mn, mx)


def quantize(x: np.ndarray, eb_abs: float) -> np.ndarray:
    x = np.ascontiguousarray(x)
    q = np.empty(max(x.size, 1), np.int32)
    bad = ctypes.c_uint64(0)
    st = lib().zco_quantize(_ptr(x), x.size, _dtype_code(x), float(eb_abs), _ptr(q),
                            ctypes.byref(bad))
    if st:
        raise OracleError(st, "quantize at %d" % bad.value)
    return q[: x.size]


def encode_q(q: np.ndarray, eb_f32: float, log2L: int, dtype: int = F32) -> bytes:
    q = np.ascontiguousarray(q, dtype=np.int32)
    cap = max_stream_bytes(q.size, log2L) + 64
    out = np.zeros(cap, np.uint8)
    n_out = ctypes.c_uint64(0)
    st = lib().zco_encode_q(_ptr(q), q.size, dtype, float(eb_f32), log2L, _ptr(out), cap,
                            ctypes.byref(n_out))
    if st:
        raise OracleError(st, "encode_q")
    return out[: n_out.value].tobytes()


def compress(x: np.ndarray, eb_abs: float, log2L: int = 5) -> bytes:
    x = np.ascontiguousarray(x)
    cap = max_stream_bytes(x.size, log2L) + 64
    out = np.zeros(cap, np.uint8)
    n_out, bad = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib().zco_compress(_ptr(x), x.size, _dtype_code(x), float(eb_abs), log2L, _ptr(out),
                            cap, ctypes.byref(n_out), ctypes.byref(bad))
    if st:
        raise OracleError(st, "compress at %d" % bad.value)
    return out[: n_out.value].tobytes()


def compress_heads(x: np.ndarray, eb_abs: float, log2L: int = 5) -> bytes:
    """Stream with the block heads stored apart (flag bit 1): a 24-bit field
    per block head, widths over the in-block deltas only."""
    x = np.ascontiguousarray(x)
    L = 1 << log2L
    nb = (x.size + L - 1) // L
    cap = max_stream_bytes(x.size, log2L) + pad16(3 * nb) + 64
    out = np.zeros(cap, np.uint8)
    n_out, bad = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib().zco_compress_heads(_ptr(x), x.size, _dtype_code(x), float(eb_abs), log2L,
                                  _ptr(out), cap, ctypes.byref(n_out), ctypes.byref(bad))
    if st:
        raise OracleError(st, "compress_heads at %d" % bad.value)
    return out[: n_out.value].tobytes()


def encode_q_heads(q: np.ndarray, eb_f32: float, log2L: int, dtype: int = F32) -> bytes:
    q = np.ascontiguousarray(q, dtype=np.int32)
    L = 1 << log2L
    cap = max_stream_bytes(q.size, log2L) + pad16(3 * ((q.size + L - 1) // L)) + 64
    out = np.zeros(cap, np.uint8)
    n_out = ctypes.c_uint64(0)
    st = lib().zco_encode_q_heads(_ptr(q), q.size, dtype, float(eb_f32), log2L, _ptr(out), cap,
                                  ctypes.byref(n_out))
    if st:
        raise OracleError(st, "encode_q_heads")
    return out[: n_out.value].tobytes()


def compress_raw(x: np.ndarray) -> bytes:
    x = np.ascontiguousarray(x)
    cap = HEADER + pad16(x.nbytes) + 16
    out = np.zeros(cap, np.uint8)
    n_out = ctypes.c_uint64(0)
    st = lib().zco_compress_raw(_ptr(x), x.size, _dtype_code(x), _ptr(out), cap,
                                ctypes.byref(n_out))
    if st:
        raise OracleError(st, "compress_raw")
    return out[: n_out.value].tobytes()


def _as_u8(stream) -> np.ndarray:
    return np.frombuffer(bytes(stream), np.uint8).copy()


def header(stream) -> dict:
    s = _as_u8(stream)
    dt, lg, fl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n, eb, nb, pl = ctypes.c_uint64(), ctypes.c_float(), ctypes.c_uint32(), ctypes.c_uint64()
    st = lib().zco_parse_header(_ptr(s), s.size, ctypes.byref(dt), ctypes.byref(lg),
                                ctypes.byref(fl), ctypes.byref(n), ctypes.byref(eb),
                                ctypes.byref(nb), ctypes.byref(pl))
    if st:
        raise OracleError(st, "header")
    return dict(dtype=dt.value, log2L=lg.value, flags=fl.value, n=n.value, eb=eb.value,
                nb=nb.value, payload=pl.value)


def decode_q(stream, n: int) -> np.ndarray:
    s = _as_u8(stream)
    q = np.empty(max(n, 1), np.int32)
    st = lib().zco_decode_q(_ptr(s), s.size, _ptr(q), n)
    if st:
        raise OracleError(st, "decode_q")
    return q[:n]


def decompress(stream, n: int, out_dtype: int = F32) -> np.ndarray:
    s = _as_u8(stream)
    out = np.empty(max(n, 1), np.float32 if out_dtype == F32 else np.uint16)
    st = lib().zco_decompress(_ptr(s), s.size, _ptr(out), n, out_dtype)
    if st:
        raise OracleError(st, "decompress")
    return out[:n]


def reduce_step(cin, local: np.ndarray, eb_abs: float, log2L: int = 5, want_stream=True,
                want_sum=False):
    """One ring step: decode ``cin`` (None = nothing received yet), add
    ``local`` in FP32, re-encode with the fixed bound."""
    local = np.ascontiguousarray(local, dtype=np.float32)
    n = local.size
    if cin is not None:
        s = _as_u8(cin)
        s_ptr, s_len = _ptr(s), s.size
    else:
        s, s_ptr, s_len = None, None, 0
    cap = max_stream_bytes(n, log2L) + 64
    out = np.zeros(cap, np.uint8) if want_stream else None
    sm = np.empty(max(n, 1), np.float32) if want_sum else None
    n_out, bad = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib().zco_reduce_step(s_ptr, s_len, _ptr(local), n, float(eb_abs), log2L,
                               _ptr(out) if want_stream else None, cap, ctypes.byref(n_out),
                               _ptr(sm) if want_sum else None, ctypes.byref(bad))
    if st:
        raise OracleError(st, "reduce_step at %d" % bad.value)
    stream = out[: n_out.value].tobytes() if want_stream else None
    return stream, (sm[:n] if want_sum else None)


def scatter_pack(x: np.ndarray, counts, displs, eb_abs: float, log2L: int = 5):
    x = np.ascontiguousarray(x)
    P = len(counts)
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    d = np.ascontiguousarray(displs, dtype=np.uint64)
    cap = sum(max_stream_bytes(int(k), log2L) for k in counts) + 64
    out = np.zeros(cap, np.uint8)
    seg = np.zeros(P + 1, np.uint64)
    st = lib().zco_scatter_pack(_ptr(x), _dtype_code(x), P, _ptr(c), _ptr(d), float(eb_abs),
                                log2L, _ptr(out), cap, _ptr(seg))
    if st:
        raise OracleError(st, "scatter_pack")
    return out[: int(seg[P])].tobytes(), seg


def ring_reduce_scatter(ranks, eb_abs: float, log2L: int = 5):
    """Simulated ring reduce-scatter over P rank buffers (Sec. 3.2.3): the
    buffer is cut into P chunks; at step t rank r decodes what rank r-1 sent
    for chunk (r-1-t) mod P, adds its own copy of that chunk and re-encodes,
    except at the last step, which keeps the FP32 sum.  Returns, per rank r,
    the reduced chunk (r+1) mod P and the streams sent at every step."""
    P = len(ranks)
    n = ranks[0].size
    bounds = chunk_bounds(n, P)
    chunk = lambda r, c: ranks[r][bounds[c]:bounds[c + 1]]
    # initial compress: rank r encodes its own chunk r
    sent = [reduce_step(None, chunk(r, r), eb_abs, log2L)[0] for r in range(P)]
    history = [list(sent)]
    result = [None] * P
    for t in range(P - 1):
        last = t == P - 2
        new = [None] * P
        for r in range(P):
            c = (r - 1 - t) % P
            src = sent[(r - 1) % P]
            s, sm = reduce_step(src, chunk(r, c), eb_abs, log2L, want_stream=not last,
                                want_sum=last)
            if last:
                result[r] = sm
            else:
                new[r] = s
        if not last:
            sent = new
            history.append(list(sent))
    return result, history


def chunk_bounds(n: int, P: int):
    """Chunk c of a rank buffer is [bounds[c], bounds[c+1]): equal parts, the
    remainder spread over the first chunks."""
    base, rem = divmod(n, P)
    b = [0]
    for c in range(P):
        b.append(b[-1] + base + (1 if c < rem else 0))
    return b


def ring_allreduce(ranks, eb_abs: float, log2L: int = 5, stage_bytes=None):
    """Simulated ring Allreduce (Sec. 3.3.3): the reduce-scatter of
    ``ring_reduce_scatter`` whose last step also re-encodes the full sum (the
    Allgather stage's one compression), then the Allgather stage: every rank
    decodes the P - 1 chunks it does not own; it keeps its own chunk as the
    FP32 sum.  Returns the P result buffers and the P final chunk streams
    (stream c encodes chunk c).  If ``stage_bytes`` is a list, the total
    length of the P streams written at every stage (the first compression,
    then each step) is appended to it (bookkeeping only)."""
    P = len(ranks)
    n = ranks[0].size
    bounds = chunk_bounds(n, P)
    chunk = lambda r, c: ranks[r][bounds[c]:bounds[c + 1]]
    sent = [reduce_step(None, chunk(r, r), eb_abs, log2L)[0] for r in range(P)]
    if stage_bytes is not None:
        stage_bytes.append(sum(map(len, sent)))
    own = [None] * P
    final = [None] * P
    for t in range(P - 1):
        last = t == P - 2
        new = [None] * P
        for r in range(P):
            c = (r - 1 - t) % P
            s, sm = reduce_step(sent[(r - 1) % P], chunk(r, c), eb_abs, log2L, want_stream=True,
                                want_sum=last)
            new[r] = s
            if last:
                own[r] = sm
                final[c] = s
        sent = new
        if stage_bytes is not None:
            stage_bytes.append(sum(map(len, sent)))
    if P == 1:
        own[0] = np.asarray(ranks[0], np.float32).copy()
        final[0] = sent[0]
    out = []
    for r in range(P):
        mine = (r + 1) % P if P > 1 else 0
        buf = np.empty(n, np.float32)
        for c in range(P):
            m = bounds[c + 1] - bounds[c]
            buf[bounds[c]:bounds[c + 1]] = own[r] if c == mine else decompress(final[c], m)
        out.append(buf)
    return out, final


def redoub_plan(N: int):
    """The recursive-doubling schedule of Sec. 3.3.4 for N ranks: k = floor(log2
    N), r = N - 2^k.  Returns (k, r, active) where active[j] is the original
    rank playing new rank j in the 2^k-rank stage: the odd ranks below 2r
    (which absorbed their even neighbour) and the ranks from 2r on."""
    k = N.bit_length() - 1
    r = N - (1 << k)
    active = [i for i in range(2 * r) if i % 2 == 1] + list(range(2 * r, N))
    return k, r, active


def redoub_allreduce(ranks, eb_abs: float, log2L: int = 5):
    """Simulated recursive-doubling Allreduce (Sec. 3.3.4, gZ-Allreduce
    ReDoub).  Stage 1: each even rank i < 2r compresses its whole buffer and
    sends it to rank i + 1, which decodes it and adds it to its own.  Stage
    2, among the 2^k remaining ranks, log2(2^k) steps: every rank compresses
    its whole current buffer and sends it to its partner (new rank xor 2^s),
    then decodes the partner's and adds it to its own (one fused ring-style
    step: decode, add, re-encode for the next send).  Final stage: rank i + 1
    sends its result, compressed, back to rank i < 2r (even), which decodes
    it.  Returns the N result buffers."""
    N = len(ranks)
    k, r, active = redoub_plan(N)
    cur = [np.asarray(x, np.float32).copy() for x in ranks]
    n = cur[0].size
    for i in range(0, 2 * r, 2):  # stage 1
        s = compress(cur[i], eb_abs, log2L)
        cur[i + 1] = reduce_step(s, cur[i + 1], eb_abs, log2L, want_stream=False,
                                 want_sum=True)[1]
    sent = {j: compress(cur[active[j]], eb_abs, log2L) for j in range(1 << k)}
    for step in range(k):
        last = step == k - 1
        new = {}
        for j in range(1 << k):
            p = j ^ (1 << step)
            s, sm = reduce_step(sent[p], cur[active[j]], eb_abs, log2L, want_stream=not last,
                                want_sum=True)
            cur[active[j]] = sm
            new[j] = s
        sent = new
    for i in range(0, 2 * r, 2):  # final stage: results back to the folded even ranks
        cur[i] = decompress(compress(cur[i + 1], eb_abs, log2L), n)
    return cur


def redoub_bound(N: int, rank: int, eb: float) -> float:
    """Worst-case quantization error of rank's recursive-doubling result (FP32
    add roundings excluded): a step adds the partner's error and one fresh
    quantization to its own, e_s = 2 e_(s-1) + eb over k steps; ranks that
    absorbed a neighbour start at eb; a folded rank adds one more eb."""
    k, r, active = redoub_plan(N)
    e0 = eb if r > 0 else 0.0
    e = (1 << k) * e0 + ((1 << k) - 1) * eb
    if rank < 2 * r and rank % 2 == 0:
        e += eb
    return e
