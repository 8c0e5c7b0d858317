"""Host side of the per-chunk codec selector: data sets, labels, training and
evaluation.  Every computation on chunk data runs in libzc's kernels
(statistics, MLP forward / gradient / SGD, selection, the codec itself); this
module allocates buffers, orders the calls and does the bookkeeping of the
results (numpy on a few numbers per chunk).

The selector trades codec time against link bytes per 64 KiB chunk, the
trade Sec. 3.2.2 and Sec. 3.3.3 of the paper make per collective: it picks the
block size L in {16, 32, 64, 128} or raw storage.  Its network predicts the
log2 bits per element of each L from 16 sampled statistics; the fixed
heuristic (L = 32, raw when the sampled estimate says coding does not pay) is
both its fallback and its judge.  Labels come from the codec itself: every
training chunk is compressed at every L and its stream lengths are read.  A
second network of the same shape predicts the codec's time: the log2 of its
ns per input byte (compression plus decompression) at each L, labelled by
timing the codec on groups of similar training chunks (one input type, close
stream sizes), each group as one batch at every L; the measured batch-wide
rate judges it.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import workloads as W
from . import zc

CHUNK_BYTES = 1 << 16
BLOCKS = (16, 32, 64, 128)


# ---- data ---------------------------------------------------------------------------

def split_chunks(xs, ebs, chunk_bytes: int = CHUNK_BYTES):
    """Views of every message cut into chunks of chunk_bytes (the last one of a
    message may be shorter); empty messages are skipped."""
    views, cebs = [], []
    for x, eb in zip(xs, ebs):
        x = x.reshape(-1)
        per = chunk_bytes // x.element_size()
        for a in range(0, x.numel(), per):
            views.append(x[a:a + per])
            cebs.append(float(eb))
    return views, cebs


def _kind_messages(kind: int, seed: int, device, scale: int):
    """Messages of one workload kind (1: 1-D sinusoids, 2: 3-D GRF at a
    relative bound, 3: image-stacking rank images, 4: uneven mixed-precision
    gradient-like messages) with their absolute bounds."""
    r = np.random.Generator(np.random.PCG64(seed))
    if kind == 1:
        return [W.sinusoids_1d(1 << 20, seed=seed, device=device)], [1e-4]
    if kind == 2:
        x = W.grf_3d(side=scale, seed=seed, device=device)
        rel = float([1e-2, 1e-3, 1e-4][r.integers(3)])
        return [x], [rel * float(x.max() - x.min())]
    if kind == 3:
        base = W.stacking_base(side=scale * 4, seed=seed, device=device)
        img = W.stacking_rank(base, int(r.integers(64)), seed=seed)
        return [img], [1e-3 * float(img.max() - img.min())]
    specs = W.message_specs(m=8, lo_bytes=4096, hi_bytes=16 << 20, seed=seed)
    return [W.message(sp, device=device) for sp in specs], [sp["eb"] for sp in specs]


def mixed_chunks(n_chunks: int, seed: int, device="cuda", scale: int = 256):
    """About n_chunks chunks of 64 KiB drawn evenly from the four workload
    kinds (seeded; scale: GRF side, image side / 4).  Returns (views, ebs,
    kinds)."""
    per_kind = (n_chunks + 3) // 4
    views, ebs, kinds = [], [], []
    for kind in (1, 2, 3, 4):
        kv, ke = [], []
        s = seed * 100 + kind * 10000
        while len(kv) < per_kind:
            xs, es = _kind_messages(kind, s, device, scale)
            v, e = split_chunks(xs, es)
            kv += v
            ke += e
            s += 1
        pick = np.random.Generator(np.random.PCG64(seed + kind)).choice(len(kv), per_kind,
                                                                       replace=False)
        for i in sorted(pick):
            views.append(kv[i])
            ebs.append(ke[i])
            kinds.append(kind)
    return views[:n_chunks], ebs[:n_chunks], kinds[:n_chunks]


def mixed_messages(total_bytes: int, seed: int, device="cuda", scale: int = 256):
    """Whole messages of the four workload kinds, taken in turn until about
    total_bytes are reached (a mixed workload).  Returns (xs, ebs, kinds)."""
    xs, ebs, kinds = [], [], []
    tot, s, kind = 0, seed * 100, 1
    while tot < total_bytes:
        mx, me = _kind_messages(kind, s + kind * 10000, device, scale)
        for x, e in zip(mx, me):
            xs.append(x)
            ebs.append(e)
            kinds.append(kind)
            tot += x.numel() * x.element_size()
        kind = kind % 4 + 1
        if kind == 1:
            s += 1
    return xs, ebs, kinds


# ---- the codec's own measurements ------------------------------------------------------

def packed_capacity(views) -> int:
    """Packed bytes that hold every chunk at its largest choice (L = 16 or raw)."""
    tot = 0
    for v in views:
        n = v.numel()
        tot += max(zc.zc_max_compressed_bytes(n, 16), zc.zc_raw_stream_bytes(n, zc.dtype_code(v)))
    return tot


class ChunkBatch:
    """A batched-compression plan over chunk views, with its decompression
    plan and the buffers of the selector."""

    def __init__(self, views, ebs, stream=None):
        self.views = views
        self.M = len(views)
        self.n = np.array([v.numel() for v in views], np.int64)
        self.es = np.array([v.element_size() for v in views], np.int64)
        self.stream = stream
        # grouped: whatever block sizes the selection writes, tiles of one size
        # run together (a batch that alternates sizes tile by tile compresses
        # about twice as slowly)
        self.batch = zc.BatchCompress(views, [32] * self.M, ebs, cap=packed_capacity(views),
                                      stream=stream, grouped=True)
        dev = views[0].device
        self.outs = [torch.empty(v.numel(), dtype=v.dtype, device=dev) for v in views]
        self.dec = zc.BatchDecompress(self.batch.packed, self.batch.msg_off, self.outs,
                                      stream=stream, grouped=True)
        self.feat = torch.empty((self.M, zc.N_STATS), dtype=torch.float32, device=dev)
        self.pred = torch.empty((self.M, 4), dtype=torch.float32, device=dev)
        self.pred_time = torch.empty((self.M, 4), dtype=torch.float32, device=dev)
        self.choice = torch.zeros(self.M, dtype=torch.int32, device=dev)
        self.counts = torch.zeros(2, dtype=torch.int32, device=dev)

    def sync(self):
        """Wait for the plan's stream (a torch pool stream does not order
        itself with the default stream that host reads use)."""
        if self.stream is not None:
            self.stream.synchronize()
        else:
            torch.cuda.current_stream().synchronize()

    @property
    def raw_bytes(self) -> int:
        return int((self.n * self.es).sum())

    def set_all(self, block: int):
        for i in range(self.M):
            self.batch.msgs[i].block = block
        self.batch.replan(self.batch.plan.tile_chunks, self.batch.plan.grid)

    def sizes(self) -> np.ndarray:
        """Stream length of every chunk (from the streams' headers)."""
        self.sync()
        off = self.batch.msg_off.cpu().numpy()
        hdr = self.batch.packed[:int(off[-1])].view(-1)
        idx = torch.from_numpy(off[:-1, None] + np.arange(32)[None, :]).to(hdr.device)
        h = np.ascontiguousarray(hdr[idx].cpu().numpy())
        flags = h[:, 6].astype(np.int64)
        nb = h[:, 20:24].copy().view(np.uint32)[:, 0].astype(np.int64)
        payload = h[:, 24:32].copy().view(np.uint64)[:, 0].astype(np.int64)
        pad = lambda v: (v + 15) // 16 * 16
        coded = 32 + pad(nb) + np.where(flags & 2, pad(3 * nb), 0) + pad(payload)
        return np.where(flags & 1, 32 + pad(payload), coded)

    def stats(self):
        zc._check(zc.zc_batch_chunk_stats(self.batch.plan, self.feat.data_ptr(),
                                          zc._stream(self.stream)), "zc_batch_chunk_stats")
        return self.feat

    def true_bits(self) -> np.ndarray:
        """[M, 4] bits per element of every chunk's stream at each L (the
        codec run at every L; the plan is left at L = 32)."""
        out = np.zeros((self.M, 4))
        for k, L in enumerate(BLOCKS):
            self.set_all(L)
            self.batch.run(self.stream)
            out[:, k] = 8.0 * self.sizes() / self.n
        self.set_all(32)
        return out

    def time_ms(self, reps: int = 3):
        """Median device time of one batched compression and one batched
        decompression of the plan as it stands."""
        s = self.stream if self.stream is not None else torch.cuda.current_stream()
        ts = []
        for _ in range(reps + 1):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(s)
            self.batch.run(s)
            e1.record(s)
            self.dec.run(s)
            e2.record(s)
            e2.synchronize()
            ts.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
        ts = ts[1:]
        return (float(np.median([t[0] for t in ts])), float(np.median([t[1] for t in ts])))

    def cost_model(self, link_gbs: float, judge_log2: float = 1.0, reps: int = 5,
                   judge_time_log2: float = 2.0):
        """The codec's time per input byte at each choice, measured on this
        batch (compression + decompression, CUDA events), as a zc_select_cfg:
        every block size timed on a plan that uses it throughout, raw storage
        likewise.  The batch is grouped by block size, so a mixed selection
        runs each chunk at its block size's own rate; the round-robin mix
        (every tile a different size) is timed too, for the record
        (self.mixed_ns_per_byte)."""
        cfg = zc.ZcSelectCfg()
        cfg.link_gbs = link_gbs
        cfg.judge_log2 = judge_log2
        cfg.judge_time_log2 = judge_time_log2
        self.uniform_ns_per_byte = []
        for k, L in enumerate(BLOCKS):
            self.set_all(L)
            c, d = self.time_ms(reps)
            self.uniform_ns_per_byte.append((c + d) * 1e6 / self.raw_bytes)
            cfg.ns_per_byte[k] = self.uniform_ns_per_byte[-1]
        for i in range(self.M):
            self.batch.msgs[i].block = BLOCKS[i % 4]
        self.batch.replan(self.batch.plan.tile_chunks, self.batch.plan.grid)
        c, d = self.time_ms(reps)
        self.mixed_ns_per_byte = (c + d) * 1e6 / self.raw_bytes
        self.set_all(zc.RAW)
        c, d = self.time_ms(reps)
        cfg.raw_ns_per_byte = (c + d) * 1e6 / self.raw_bytes
        self.set_all(32)
        return cfg

    def run_selected(self, cfg, mlp: "Mlp | None", tmlp: "Mlp | None" = None):
        """The selector path: statistics, (networks,) selection into the
        plan, batched compression -- all launches on the plan's stream.
        tmlp: the time network (used only with the bits network mlp)."""
        self.stats()
        pred = pred_time = None
        if mlp is not None:
            pred = mlp.forward(self.feat, out=self.pred, stream=self.stream)
            if tmlp is not None:
                pred_time = tmlp.forward(self.feat, out=self.pred_time, stream=self.stream)
        self.select(cfg, pred, pred_time)
        self.batch.run(self.stream)

    def select(self, cfg, pred: torch.Tensor | None, pred_time: torch.Tensor | None = None):
        zc._check(zc.zc_batch_select_timed(self.batch.plan, self.feat.data_ptr(),
                                           None if pred is None else pred.data_ptr(),
                                           None if pred_time is None else pred_time.data_ptr(),
                                           cfg, self.choice.data_ptr(), self.counts.data_ptr(),
                                           zc._stream(self.stream)), "zc_batch_select_timed")
        return self.choice


def _copies(views, stream=None, align: int = 64):
    """Copies of the views in one fresh buffer, each starting at a multiple
    of `align` elements (the originals' dtype)."""
    offs, tot = [], 0
    for v in views:
        offs.append(tot)
        tot += (v.numel() + align - 1) // align * align
    buf = torch.empty(max(tot, 1), dtype=views[0].dtype, device=views[0].device)
    s = stream if stream is not None else torch.cuda.current_stream()
    s.wait_stream(torch.cuda.current_stream())
    out = []
    with torch.cuda.stream(s):
        for v, o in zip(views, offs):
            d = buf[o:o + v.numel()]
            d.copy_(v.reshape(-1))
            out.append(d)
    return out


def time_labels(views, ebs, true_bits, groups: int = 16, reps: int = 3, stream=None,
                min_group: int = 8, min_bytes: int = 256 << 20):
    """[M, 4] measured codec ns per input byte (compression plus
    decompression) of every chunk at L = 16 .. 128, and the groups.  The
    chunks of each input type are sorted by their true bits per element at
    L = 32 and cut into `groups` runs of about equal count (at least
    min_group chunks each); every run is compressed and decompressed as one
    grouped batch at each L (CUDA events, median of reps) and its chunks take
    the run's rate.  A run is timed repeated until the batch holds at least
    min_bytes of input, so that every rate is the codec's rate on a full GPU
    (a small batch would charge its launch and its last partial wave to its
    few bytes); the copies are distinct memory (no copy is read from L2
    because an earlier one was).  Returns (rates, group index of every
    chunk)."""
    M = len(views)
    es = np.array([v.element_size() for v in views])
    rates = np.zeros((M, 4))
    gid = np.full(M, -1, np.int64)
    g = 0
    for e in sorted(set(es.tolist())):
        idx = np.nonzero(es == e)[0]
        idx = idx[np.argsort(true_bits[idx, 1], kind="stable")]
        k = max(1, min(groups, len(idx) // min_group))
        for part in np.array_split(idx, k):
            nbytes = int(sum(views[i].numel() for i in part)) * int(e)
            rep = max(1, -(-min_bytes // max(nbytes, 1)))
            sel = np.tile(part, rep)
            gv = _copies([views[i] for i in sel], stream)
            cb = ChunkBatch(gv, [ebs[i] for i in sel], stream=stream)
            for j, L in enumerate(BLOCKS):
                cb.set_all(L)
                c, d = cb.time_ms(reps)
                rates[part, j] = (c + d) * 1e6 / cb.raw_bytes
            gid[part] = g
            g += 1
            del cb
    return rates, gid


# ---- the network -----------------------------------------------------------------------

def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, in the
    library's parameter layout."""
    r = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for shape in ((64, 16), (64,), (64, 64), (64,), (4, 64), (4,)):
        if len(shape) == 2:
            b = math.sqrt(6.0 / shape[1])
            parts.append(r.uniform(-b, b, shape).reshape(-1))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


class Mlp:
    """The 16-64-64-4 network, its optimizer state and input normalisation,
    all in device memory; trained by zc_mlp_grad + zc_mlp_sgd."""

    def __init__(self, seed: int = 0, device="cuda"):
        self.device = device
        self.params = torch.from_numpy(init_params(seed)).to(device)
        self.vel = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.norm = torch.cat([torch.zeros(16), torch.ones(16)]).to(device)

    def set_norm(self, X: torch.Tensor):
        x = X.double().cpu().numpy()
        mu = x.mean(0)
        sd = x.std(0)
        inv = np.where(sd > 1e-12, 1.0 / np.maximum(sd, 1e-12), 1.0)
        self.norm = torch.from_numpy(np.concatenate([mu, inv]).astype(np.float32)).to(self.device)

    def forward(self, X: torch.Tensor, out: torch.Tensor | None = None, stream=None):
        X = X.contiguous()
        out = out if out is not None else torch.empty((X.shape[0], 4), dtype=torch.float32,
                                                      device=X.device)
        zc._check(zc.zc_mlp_forward(self.params.data_ptr(), self.norm.data_ptr(), X.data_ptr(),
                                    X.shape[0], out.data_ptr(), zc._stream(stream)),
                  "zc_mlp_forward")
        return out

    def fit(self, X: torch.Tensor, T: torch.Tensor, epochs: int = 60, batch: int = 256,
            lr: float = 0.02, momentum: float = 0.9, seed: int = 0, stream=None):
        """Minibatch momentum SGD on the mean squared error; returns the mean
        minibatch loss of every epoch."""
        X, T = X.contiguous(), T.contiguous()
        N = X.shape[0]
        steps = (N + batch - 1) // batch
        scratch = torch.empty(zc.zc_mlp_scratch_bytes(batch) // 4 + 1, dtype=torch.float32,
                              device=X.device)
        losses = torch.zeros(steps, dtype=torch.float32, device=X.device)
        idx = torch.empty(N, dtype=torch.int32, device=X.device)
        g = torch.Generator(device=X.device)
        g.manual_seed(seed)
        s = zc._stream(stream)
        ts = stream if stream is not None else torch.cuda.current_stream()
        ts.wait_stream(torch.cuda.current_stream())  # X, T and the buffers above
        hist = []
        for _ in range(epochs):
            with torch.cuda.stream(ts):
                idx.copy_(torch.randperm(N, generator=g, device=X.device).to(torch.int32))
            for k in range(steps):
                b0 = k * batch
                B = min(batch, N - b0)
                zc._check(zc.zc_mlp_grad(self.params.data_ptr(), self.norm.data_ptr(),
                                         X.data_ptr(), T.data_ptr(), idx.data_ptr() + 4 * b0, B,
                                         self.grad.data_ptr(), losses.data_ptr() + 4 * k,
                                         scratch.data_ptr(), scratch.numel() * 4, s),
                          "zc_mlp_grad")
                zc._check(zc.zc_mlp_sgd(self.params.data_ptr(), self.vel.data_ptr(),
                                        self.grad.data_ptr(), lr, momentum, s), "zc_mlp_sgd")
            with torch.cuda.stream(ts):
                m = losses.mean()
            ts.synchronize()
            hist.append(float(m))
        return hist


# ---- evaluation ----------------------------------------------------------------------

def costs(n, es, bits, cfg, rates=None):
    """Modelled ns per chunk: coded at each L with the given bits per element
    ([M, 4]) and raw ([M]); codec time at the batch-wide rates of cfg, or at
    every chunk's own measured rates ([M, 4] ns per input byte)."""
    bytes_in = n * es
    if rates is None:
        rates = np.array([cfg.ns_per_byte[k] for k in range(4)])[None, :]
    coded = bytes_in[:, None] * rates + n[:, None] * bits / 8.0 / cfg.link_gbs
    raw = bytes_in * cfg.raw_ns_per_byte + (32.0 + bytes_in) / cfg.link_gbs
    return coded, raw


def evaluate(choice: np.ndarray, n, es, true_bits, cfg, rates=None) -> dict:
    """Modelled cost of the choices with the measured sizes (and, given,
    every chunk's measured codec rates), against the best choice per chunk:
    total ns, regret (total / best total - 1), mispredict rate (chunks whose
    choice costs more than 0.1 % above their best)."""
    coded, raw = costs(n, es, true_bits, cfg, rates)
    allc = np.concatenate([coded, raw[:, None]], 1)
    col = np.array([{16: 0, 32: 1, 64: 2, 128: 3, 0: 4}[int(c)] for c in choice])
    got = allc[np.arange(len(col)), col]
    best = allc.min(1)
    return {"cost_ns": float(got.sum()), "best_ns": float(best.sum()),
            "regret": float(got.sum() / best.sum() - 1.0),
            "mispredict": float(np.mean(got > best * 1.001)),
            "raw_frac": float(np.mean(col == 4))}


def dataset(cb: ChunkBatch):
    """Features and labels (log2 true bits per element) of a chunk batch,
    rows with a NaN feature removed; returns (X, T, keep mask, true bits)."""
    cb.stats()
    cb.sync()
    X = cb.feat.clone()
    bits = cb.true_bits()
    keep = torch.isfinite(X).all(1).cpu().numpy() & np.all(bits > 0, 1)
    T = torch.from_numpy(np.log2(np.where(bits > 0, bits, 1.0)).astype(np.float32)).to(X.device)
    k = torch.from_numpy(keep).to(X.device)
    return X[k].contiguous(), T[k].contiguous(), keep, bits
