"""CPU oracle of the per-chunk codec selector: chunk statistics, the MLP
(forward, loss gradient, SGD step) and the selection rule.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: tests/,
``__graft_entry__.smoke()`` and ``bench.py``'s reference leg may use it; the
CUDA library shares no code with it.  Everything is plain numpy in FP64
(written for reading, not speed), except the quantizer, which is the codec
oracle's exact one (``oracle.quantize``).

The paper fixes one codec configuration per run; Sec. 3.2.2 shows that what a
compression step costs depends on the message, and Sec. 3.3.3 weighs the
compression cost of a collective against what it saves on the link.  The
selector makes that trade per 64 KiB chunk: 16 cheap statistics of a sample
of the chunk feed a 16-64-64-4 MLP that predicts, for each block size
L in {16, 32, 64, 128}, the log2 of the stream's bits per element, and a
second network of the same shape (a time network) may predict the log2 of
the codec's ns per input byte at each L; a cost model turns predictions into
a choice of L or of sending the chunk raw.  The
fixed heuristic (L = 32, raw when the sampled estimate does not pay) is the
fallback, and it judges the network: a prediction too far from the sampled
estimate of the chosen L is discarded in favour of the heuristic.  The
measured batch-wide codec rate judges the time network the same way: a
predicted rate too far from it is replaced by it.

Definitions (the CUDA kernels implement the same ones):

Sample.  A chunk of n_c elements has m = n_c // 128 full spans of 128
elements; the sample is S = min(16, m) of them, span j starting at element
128 * floor(j (m - 1) / (S - 1)) (span 0 alone when S = 1).  A chunk with
m = 0 is sampled as one partial span of n_c elements.

Per span, with q the exactly quantized values (Sec. 3.3.2's prequantization,
as in the codec):
  - for every L, the blocks of L elements (the last may be partial): the
    codec's block bits, (w + 1) L for width w > 0 (else 0), where w is the
    bit length of the largest |d| of the block, d the Lorenzo deltas with the
    block head predicted from 0;
  - the first differences d_i = q_i - q_{i-1} (i >= 1), the second
    differences d_i - d_{i-1} (i >= 2), the sign changes d_i d_{i-1} < 0.

Features (f[k], FP32 on the GPU):
  f0..f3  sampled bits per element at L = 16, 32, 64, 128, plus the width
          bytes (8 / L) and the header (256 / n_c);
  f4      log2(1 + max q - min q);
  f5      log2(1 + mean |d|);     f6  log2(1 + max |d|);
  f7      fraction of d == 0;     f8  fraction of q == 0;
  f9      log2(1 + mean |q|);     f10 log2(1 + mean |second difference|);
  f11     fraction of sign changes among consecutive d;
  f12     mean bit length of |q| at the heads of the L = 32 blocks, / 24;
  f13     population standard deviation over the spans of the span's L = 32
          bits per element;
  f14     raw bits per element / 32 (1 for FP32, 0.5 for BF16);
  f15     log2(n_c) / 16.
Means over empty sets are 0.  A chunk whose sample holds a value the codec
cannot quantize (non-finite, or |q| > 2^22), or an empty chunk, gets a row of
NaN (the selection then sends it raw).
"""
from __future__ import annotations

import math

import numpy as np

from . import quantize as _quantize, OracleError

N_STATS = 16
SPANS = 16
SPAN = 128
BLOCKS = (16, 32, 64, 128)
N_IN, N_HID, N_OUT = 16, 64, 4
# parameter vector layout: W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]
_SHAPES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
           ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in _SHAPES)


def bitlen(v: int) -> int:
    return int(v).bit_length()


def span_starts(n_c: int):
    """(start, count) of the sampled spans of an n_c-element chunk."""
    m = n_c // SPAN
    if m == 0:
        return [(0, n_c)] if n_c > 0 else []
    S = min(SPANS, m)
    if S == 1:
        return [(0, SPAN)]
    return [(SPAN * ((j * (m - 1)) // (S - 1)), SPAN) for j in range(S)]


def block_bits(q: np.ndarray, L: int) -> int:
    """The codec's payload bits for the values q split into blocks of L."""
    bits = 0
    for b0 in range(0, len(q), L):
        blk = [int(v) for v in q[b0:b0 + L]]
        d = [blk[0]] + [blk[i] - blk[i - 1] for i in range(1, len(blk))]
        w = bitlen(max(abs(v) for v in d))
        if w > 0:
            bits += (w + 1) * L
    return bits


def chunk_stats(x: np.ndarray, eb_abs: float) -> np.ndarray:
    """The 16 features of one chunk (x: float32, or uint16 BF16 bits)."""
    n_c = x.size
    spans = span_starts(n_c)
    f = np.full(N_STATS, np.nan)
    if not spans:
        return f
    raw_bits = 32 if x.dtype == np.float32 else 16
    qs = []
    for s0, cnt in spans:
        try:
            qs.append(_quantize(x[s0:s0 + cnt], eb_abs).astype(np.int64))
        except OracleError:
            return f
    tot = sum(len(q) for q in qs)
    for k, L in enumerate(BLOCKS):
        f[k] = sum(block_bits(q, L) for q in qs) / tot + 8.0 / L + 256.0 / n_c
    allq = np.concatenate(qs)
    f[4] = math.log2(1 + int(allq.max()) - int(allq.min()))
    d = [np.diff(q) for q in qs]
    d2 = [np.diff(v) for v in d]
    nd = sum(len(v) for v in d)
    nd2 = sum(len(v) for v in d2)
    if nd:
        f[5] = math.log2(1 + sum(int(np.abs(v).sum()) for v in d) / nd)
        f[6] = math.log2(1 + max(int(np.abs(v).max()) if len(v) else 0 for v in d))
        f[7] = sum(int((v == 0).sum()) for v in d) / nd
    else:
        f[5] = f[6] = f[7] = 0.0
    f[8] = int((allq == 0).sum()) / tot
    f[9] = math.log2(1 + int(np.abs(allq).sum()) / tot)
    if nd2:
        f[10] = math.log2(1 + sum(int(np.abs(v).sum()) for v in d2) / nd2)
        f[11] = sum(int((v[1:] * v[:-1] < 0).sum()) for v in d) / nd2
    else:
        f[10] = f[11] = 0.0
    heads = [bitlen(abs(int(q[b0]))) for q in qs for b0 in range(0, len(q), 32)]
    f[12] = sum(heads) / len(heads) / 24.0
    per_span = np.array([block_bits(q, 32) / len(q) for q in qs])
    f[13] = float(np.sqrt(np.mean((per_span - per_span.mean()) ** 2)))
    f[14] = raw_bits / 32.0
    f[15] = math.log2(n_c) / 16.0
    return f


def chunk_bits_per_element(x: np.ndarray, eb_abs: float, log2L: int, codec_compress) -> float:
    """Label: bits per element of the whole chunk's stream at block 2^log2L
    (codec_compress: the codec oracle's compress)."""
    return 8.0 * len(codec_compress(x, eb_abs, log2L)) / x.size


# ---- the MLP ---------------------------------------------------------------------

def unpack(p: np.ndarray):
    out, o = {}, 0
    for name, shape in _SHAPES:
        k = int(np.prod(shape))
        out[name] = p[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], np.float64).reshape(-1) for name, _ in _SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    r = np.random.Generator(np.random.PCG64(seed))
    parts = {}
    for name, shape in _SHAPES:
        if name.startswith("W"):
            bound = math.sqrt(6.0 / shape[1])
            parts[name] = r.uniform(-bound, bound, shape)
        else:
            parts[name] = np.zeros(shape)
    return pack(parts).astype(np.float32)


def normalize(X: np.ndarray, norm: np.ndarray) -> np.ndarray:
    """norm = [mu(16), inv_sd(16)]: x' = (x - mu) * inv_sd."""
    return (np.asarray(X, np.float64) - norm[:N_IN]) * norm[N_IN:]


def forward(p: np.ndarray, norm: np.ndarray, X: np.ndarray, keep=False):
    P = unpack(np.asarray(p, np.float64))
    Xn = normalize(X, np.asarray(norm, np.float64))
    A1 = Xn @ P["W1"].T + P["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ P["W3"].T + P["b3"]
    if keep:
        return Y, (P, Xn, A1, H1, A2, H2)
    return Y


def loss_grad(p: np.ndarray, norm: np.ndarray, X: np.ndarray, T: np.ndarray):
    """Mean squared error over the B x 4 outputs and its gradient (backprop
    through the two ReLU layers; the ReLU derivative is 0 at 0)."""
    B = X.shape[0]
    Y, (P, Xn, A1, H1, A2, H2) = forward(p, norm, X, keep=True)
    R = Y - np.asarray(T, np.float64)
    loss = float((R * R).sum() / (B * N_OUT))
    dY = 2.0 * R / (B * N_OUT)
    g = {"W3": dY.T @ H2, "b3": dY.sum(0)}
    dA2 = (dY @ P["W3"]) * (A2 > 0)
    g["W2"] = dA2.T @ H1
    g["b2"] = dA2.sum(0)
    dA1 = (dA2 @ P["W2"]) * (A1 > 0)
    g["W1"] = dA1.T @ Xn
    g["b1"] = dA1.sum(0)
    return loss, pack(g)


def sgd_step(p, v, g, lr: float, momentum: float):
    """Momentum SGD: v <- momentum v + g; p <- p - lr v."""
    v = momentum * np.asarray(v, np.float64) + np.asarray(g, np.float64)
    return np.asarray(p, np.float64) - lr * v, v


# ---- selection ---------------------------------------------------------------------

def chunk_costs(n: int, es: int, bits, cfg: dict, rates=None):
    """Modelled end-to-end cost in ns of sending an n-element chunk coded at
    each L with `bits` bits per element, and raw: codec time (measured ns per
    input byte, compression plus decompression: cfg['ns_per_byte'][k], or
    this chunk's own rates[k] when given) plus the bytes over a link of
    cfg['link_gbs'] GB/s (bytes per ns)."""
    bytes_in = n * es
    link = cfg["link_gbs"]
    rate = cfg["ns_per_byte"] if rates is None else rates
    coded = [bytes_in * rate[k] + n * bits[k] / 8.0 / link for k in range(4)]
    raw = bytes_in * cfg["raw_ns_per_byte"] + (32.0 + bytes_in) / link
    return coded, raw


def judged_rates(yt, cfg: dict):
    """The codec rates a time prediction yt (log2 ns per input byte at each L)
    stands for: 2^yt[k] where yt[k] is finite and within
    cfg['judge_time_log2'] of log2 cfg['ns_per_byte'][k], else the measured
    batch-wide rate cfg['ns_per_byte'][k] (the judge of the time network)."""
    out = []
    for k in range(4):
        c = cfg["ns_per_byte"][k]
        t = float(yt[k])
        ok = math.isfinite(t) and abs(t - math.log2(c)) <= cfg["judge_time_log2"]
        out.append(2.0 ** t if ok else c)
    return out


def heuristic_choice(n: int, es: int, f: np.ndarray, cfg: dict) -> int:
    """L = 32, or raw (0) unless the sampled estimate f1 says coding pays."""
    if not np.isfinite(f[1]):
        return 0
    coded, raw = chunk_costs(n, es, [f[1]] * 4, cfg)
    return 32 if coded[1] < raw else 0


def mlp_choice(n: int, es: int, f: np.ndarray, y: np.ndarray, cfg: dict, yt=None):
    """(choice, fell_back): the L minimising the modelled cost with bits
    2^y_k, raw (0) when that is cheaper, or the heuristic's choice when a
    prediction is not finite or the chosen L's prediction is more than
    cfg['judge_log2'] away from log2 of the sampled estimate.  With a time
    prediction yt the codec rates are judged_rates(yt, cfg)."""
    if not (np.all(np.isfinite(y)) and np.all(np.isfinite(f[:4]))):
        return heuristic_choice(n, es, f, cfg), True
    bits = [2.0 ** float(v) for v in y]
    rates = None if yt is None else judged_rates(yt, cfg)
    coded, raw = chunk_costs(n, es, bits, cfg, rates)
    k = int(np.argmin(coded))
    if abs(float(y[k]) - math.log2(f[k])) > cfg["judge_log2"]:
        return heuristic_choice(n, es, f, cfg), True
    return (BLOCKS[k] if coded[k] < raw else 0), False


def best_choice(n: int, es: int, true_bits, cfg: dict):
    """What the measured sizes say is best, and every option's cost."""
    coded, raw = chunk_costs(n, es, true_bits, cfg)
    k = int(np.argmin(coded))
    return (BLOCKS[k] if coded[k] < raw else 0), coded, raw
