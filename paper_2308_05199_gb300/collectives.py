"""Compression-accelerated Allreduce algorithms simulated on one GPU: every
"rank" is a buffer in this GPU's HBM, every step is one batched launch of
libzc kernels over all ranks (no bytes move between GPUs).

  RingAllreduce               Sec. 3.2.3 / 3.3.3: reduce-scatter in P - 1
                              fused decode + add + re-encode steps on 1/P
                              chunks, the last step also emitting the
                              reduced chunk's stream (the Allgather stage's
                              one compression), then the Allgather stage:
                              each rank decodes the P - 1 chunks it does not
                              own (one batched decompression for all ranks).
  RecursiveDoublingAllreduce  Sec. 3.3.4 (gZ-Allreduce ReDoub): the
                              remainder ranks fold into their odd neighbours,
                              log2 steps of whole-buffer exchanges among the
                              2^k others (fused decode + add + re-encode),
                              then the results go back to the folded ranks.

Both build their work-descriptor tables once (set-up) and launch them with
``run()``; nothing is read back, so a run can be captured in a CUDA graph.
``model()`` turns measured launch times and stream sizes into the time one
rank would spend with its own GPU and a link of a given bandwidth, the basis
of the algorithm choice the paper makes between the two (Sec. 3.3.3).
"""
from __future__ import annotations

import ctypes

import torch

from . import zc


U32 = 2.0 ** -24  # unit roundoff of FP32 round-to-nearest


def ring_error_bounds(P: int, eb: float, abs_sum):
    """Worst-case |result - exact sum| per element of the ring Allreduce of P
    ranks at the absolute bound eb (the FP32 bound the codec uses); abs_sum
    is sum_r |x_r| of the element (a float or an array).

    A decoded value carries at most eb of quantization error (Sec. 3.3.3:
    one compression per reduce-scatter step, N - 1 in all) plus the FP32
    rounding of q * 2eb; an FP32 addition rounds once more.  Every partial
    sum is at most abs_sum + E in magnitude, E the bound itself, so after
    the P - 1 steps
        E = (P - 1) eb + 2 (P - 1) u (abs_sum + E),   u = 2^-24,
    solved for E: the bound of the chunk a rank reduced itself (kept as the
    FP32 sum).  The chunks a rank decodes in the Allgather stage carry one
    more compression and one more rounding:
        E_dec = E + eb + u (abs_sum + E + eb).
    Returns (E, E_dec)."""
    k = P - 1
    own = (k * eb + 2 * k * U32 * abs_sum) / (1.0 - 2 * k * U32)
    dec = own + eb + U32 * (abs_sum + own + eb)
    return own, dec


def ring_target_bound(P: int, eb: float, abs_sum):
    """The stated per-element target for the reduced sums, (P - 1) eb +
    1e-6 sum_r |x_r|.  Its sum term covers the worst-case FP32 roundings
    only while 2 (P - 1) 2^-24 <= 1e-6 (P <= 9); for larger rings it is a
    measured property of the data."""
    return (P - 1) * eb + 1e-6 * abs_sum


def chunk_bounds(n: int, P: int):
    """Chunk c of a rank buffer is [b[c], b[c + 1]): equal parts, the remainder
    spread over the first chunks."""
    base, rem = divmod(n, P)
    b = [0]
    for c in range(P):
        b.append(b[-1] + base + (1 if c < rem else 0))
    return b


class _Steps:
    """Launch list of one collective: reduce-step plans and decompression
    plans, run in order on one stream."""

    def __init__(self, ws, stream):
        self.ws = ws
        self.stream = stream
        self.launches = []   # (kind, plan, table, label, n_ranks_active)

    def reduce(self, items, eb_abs, block, label, active):
        P = len(items)
        arr = (zc.ZcReduceItem * P)(*items)
        plan = zc.ZcPlan()
        table = torch.empty(max(zc.zc_plan_table_bytes(P), 16), dtype=torch.uint8,
                            device=self.ws.buf.device)
        zc._check(zc.zc_plan_reduce(plan, P, arr, eb_abs, block, table.data_ptr(), table.numel()),
                  "zc_plan_reduce")
        self.launches.append(("reduce", plan, table, label, active))

    def decompress(self, streams, caps, outs, label, active):
        M = len(outs)
        msgs = (zc.ZcMessage * M)()
        for i, o in enumerate(outs):
            msgs[i].in_ = None
            msgs[i].out = o.data_ptr() if o.numel() else None
            msgs[i].n = o.numel()
            msgs[i].dtype = zc.dtype_code(o)
        hs = (ctypes.c_void_p * M)(*streams)
        hc = (ctypes.c_uint64 * M)(*caps)
        plan = zc.ZcBatch()
        table = torch.empty(zc.zc_batch_table_bytes(M), dtype=torch.uint8,
                            device=self.ws.buf.device)
        zc._check(zc.zc_plan_decompress_streams(plan, M, hs, hc, msgs, table.data_ptr(),
                                                table.numel()), "zc_plan_decompress_streams")
        self.launches.append(("decompress", plan, table, label, active))

    def run(self, events=None):
        s = self.stream.cuda_stream
        for i, (kind, plan, _, _, _) in enumerate(self.launches):
            if events is not None:
                events[i].record(self.stream)
            if kind == "reduce":
                zc._check(zc.zc_reduce_step_batch(plan, self.ws.ptr, self.ws.nbytes, s),
                          "zc_reduce_step_batch")
            else:
                zc._check(zc.zc_decompress_batch(plan, self.ws.ptr, self.ws.nbytes, s),
                          "zc_decompress_batch")
        if events is not None:
            events[len(self.launches)].record(self.stream)

    def timed(self, reps=3):
        """Median device ms of every launch over reps runs (after one untimed)."""
        self.run()
        per = [[] for _ in self.launches]
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(self.launches) + 1)]
            self.run(ev)
            ev[-1].synchronize()
            for i in range(len(self.launches)):
                per[i].append(ev[i].elapsed_time(ev[i + 1]))
        return [sorted(p)[len(p) // 2] for p in per]


class RingAllreduce:
    """Ring Allreduce of P FP32 rank buffers (P >= 2) with a fixed absolute
    bound.  After ``run()``, ``out[r]`` holds rank r's result: its own chunk
    (r + 1) mod P as the FP32 sum, the others decoded from their final
    streams."""

    def __init__(self, ranks, eb_abs: float, block: int = 32, stream=None):
        P = len(ranks)
        if P < 2:
            raise ValueError("a ring needs at least two ranks")
        self.P, self.n = P, ranks[0].numel()
        self.ranks = [x.contiguous() for x in ranks]
        dev = self.ranks[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        b = self.bounds = chunk_bounds(self.n, P)
        m_max = max(b[c + 1] - b[c] for c in range(P))
        self.cap = zc.zc_max_compressed_bytes(m_max, block)
        self.bufs = torch.empty((2, P, self.cap), dtype=torch.uint8, device=dev)
        self.sizes = torch.zeros((P, P), dtype=torch.int64, device=dev)  # [step][rank]
        self.out = [torch.empty_like(x) for x in self.ranks]
        # the largest launch is the Allgather: P (P - 1) chunks, (P - 1) n elements
        self.ws = zc.Workspace(P * self.n, P * P, dev, self.stream)
        self.steps = _Steps(self.ws, self.stream)

        def chunk(t, c):
            return t[b[c]:b[c + 1]]

        Z = zc.ZcReduceItem
        # initial compression of every rank's own chunk r into buffer set 0
        items = [Z(None, chunk(self.ranks[r], r).data_ptr(), self.bufs[0, r].data_ptr(), None,
                   self.sizes[0, r].data_ptr(), b[r + 1] - b[r], 0, self.cap) for r in range(P)]
        self.steps.reduce(items, eb_abs, block, "compress", P)
        for t in range(P - 1):
            last = t == P - 2
            src, dst = t % 2, (t + 1) % 2
            items = []
            for r in range(P):
                c = (r - 1 - t) % P
                items.append(Z(self.bufs[src, (r - 1) % P].data_ptr(),
                               chunk(self.ranks[r], c).data_ptr(), self.bufs[dst, r].data_ptr(),
                               chunk(self.out[r], c).data_ptr() if last else None,
                               self.sizes[t + 1, r].data_ptr(), b[c + 1] - b[c], self.cap,
                               self.cap))
            self.steps.reduce(items, eb_abs, block, "step%d" % t, P)
        fin = (P - 1) % 2  # buffer set of the final streams; rank r's encodes chunk (r + 1) mod P
        streams, caps, outs = [], [], []
        for r in range(P):
            for c in range(P):
                if c == (r + 1) % P:
                    continue
                owner = (c - 1) % P
                streams.append(self.bufs[fin, owner].data_ptr())
                caps.append(self.cap)
                outs.append(chunk(self.out[r], c))
        self.steps.decompress(streams, caps, outs, "allgather", P)

    def run(self, events=None):
        self.steps.run(events)
        return self.out

    def model(self, link_gbs: float, reps: int = 3):
        """Per-rank time of the collective with one GPU per rank: every
        launch's device time divided by the ranks it served, plus, per
        communication step, the largest stream any rank sends over a link of
        link_gbs GB/s (P - 1 reduce-scatter steps, P - 1 Allgather steps)."""
        ms = self.steps.timed(reps)
        sizes = self.sizes.cpu()
        compute = sum(t / a for t, (_, _, _, _, a) in zip(ms, self.steps.launches))
        rs = sum(int(sizes[t].max()) for t in range(self.P - 1))      # streams sent at steps 0..P-2
        ag = (self.P - 1) * int(sizes[self.P - 1].max())              # final streams, P - 1 hops
        link_ms = (rs + ag) / (link_gbs * 1e6)
        return {"device_ms": round(sum(ms), 4), "launches": len(ms),
                "per_rank_compute_ms": round(compute, 4), "link_ms": round(link_ms, 4),
                "per_rank_ms": round(compute + link_ms, 4),
                "bytes_sent_per_rank": rs + ag}


def redoub_plan(N: int):
    """k = floor(log2 N), r = N - 2^k, and the original rank of every new rank
    of the 2^k-rank stage (the odd ranks below 2r, then the ranks from 2r)."""
    k = N.bit_length() - 1
    r = N - (1 << k)
    active = [i for i in range(2 * r) if i % 2 == 1] + list(range(2 * r, N))
    return k, r, active


class RecursiveDoublingAllreduce:
    """Recursive-doubling Allreduce of N FP32 rank buffers (N >= 2) with a
    fixed absolute bound.  After ``run()``, ``out[i]`` holds rank i's result."""

    def __init__(self, ranks, eb_abs: float, block: int = 32, stream=None):
        N = len(ranks)
        if N < 2:
            raise ValueError("recursive doubling needs at least two ranks")
        self.N, self.n = N, ranks[0].numel()
        self.ranks = [x.contiguous() for x in ranks]
        dev = self.ranks[0].device
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        k, r, active = self.k, self.r, self.active = redoub_plan(N)
        n = self.n
        self.cap = zc.zc_max_compressed_bytes(n, block)
        self.sbuf = torch.empty((2, N, self.cap), dtype=torch.uint8, device=dev)
        self.sizes = torch.zeros((k + 3, N), dtype=torch.int64, device=dev)
        # current values: ping-pong buffers per rank; out is the last one written
        self.val = torch.empty((2, N, n), dtype=torch.float32, device=dev)
        self.ws = zc.Workspace(N * n, N, dev, self.stream)  # a launch covers up to N whole buffers
        self.steps = _Steps(self.ws, self.stream)
        self.comm = []  # size rows of the communication steps
        Z = zc.ZcReduceItem
        cur = {i: self.ranks[i] for i in range(N)}
        where = {i: None for i in range(N)}  # ping-pong slot of rank i's current value
        row = 0

        def next_slot(i):
            s = 0 if where[i] is None else 1 - where[i]
            where[i] = s
            return self.val[s, i]

        if r > 0:
            # stage 1: even ranks below 2r compress, odd neighbours decode + add
            evens = list(range(0, 2 * r, 2))
            self.steps.reduce([Z(None, cur[i].data_ptr(), self.sbuf[0, i].data_ptr(), None,
                                 self.sizes[row, i].data_ptr(), n, 0, self.cap) for i in evens],
                              eb_abs, block, "fold_compress", len(evens))
            self.comm.append(row)
            row += 1
            items = []
            for i in evens:
                dst = next_slot(i + 1)
                items.append(Z(self.sbuf[0, i].data_ptr(), cur[i + 1].data_ptr(), None,
                               dst.data_ptr(), None, n, self.cap, 0))
                cur[i + 1] = dst
            self.steps.reduce(items, eb_abs, block, "fold_add", len(evens))
        K = 1 << k
        # stage 2: every active rank compresses its current buffer ...
        self.steps.reduce([Z(None, cur[active[j]].data_ptr(), self.sbuf[0, active[j]].data_ptr(),
                             None, self.sizes[row, active[j]].data_ptr(), n, 0, self.cap)
                           for j in range(K)], eb_abs, block, "compress", K)
        self.comm.append(row)
        row += 1
        # ... then log2 K steps: decode the partner's stream, add, re-encode
        for s in range(k):
            last = s == k - 1
            src, dst_set = s % 2, (s + 1) % 2
            items = []
            new_cur = {}
            for j in range(K):
                i, p = active[j], active[j ^ (1 << s)]
                dst = next_slot(i)
                items.append(Z(self.sbuf[src, p].data_ptr(), cur[i].data_ptr(),
                               None if last else self.sbuf[dst_set, i].data_ptr(), dst.data_ptr(),
                               None if last else self.sizes[row, i].data_ptr(), n, self.cap,
                               self.cap))
                new_cur[i] = dst
            cur.update(new_cur)
            self.steps.reduce(items, eb_abs, block, "step%d" % s, K)
            if not last:
                self.comm.append(row)
                row += 1
        if r > 0:
            # final stage: the odd neighbours send their results back, compressed
            odds = list(range(1, 2 * r, 2))
            self.steps.reduce([Z(None, cur[i].data_ptr(), self.sbuf[0, i].data_ptr(), None,
                                 self.sizes[row, i].data_ptr(), n, 0, self.cap) for i in odds],
                              eb_abs, block, "return_compress", len(odds))
            self.comm.append(row)
            row += 1
            outs = []
            for i in odds:
                d = next_slot(i - 1)
                outs.append(d)
                cur[i - 1] = d
            self.steps.decompress([self.sbuf[0, i].data_ptr() for i in odds],
                                  [self.cap] * len(odds), outs, "return_decompress", len(odds))
        self.out = [cur[i] for i in range(N)]

    def run(self, events=None):
        self.steps.run(events)
        return self.out

    def model(self, link_gbs: float, reps: int = 3):
        """Per-rank time with one GPU per rank: launch times divided by the
        ranks each served, plus the largest stream of every communication
        step over the link (fold, log2 steps, return)."""
        ms = self.steps.timed(reps)
        sizes = self.sizes.cpu()
        compute = sum(t / a for t, (_, _, _, _, a) in zip(ms, self.steps.launches))
        sent = sum(int(sizes[rw].max()) for rw in self.comm)
        link_ms = sent / (link_gbs * 1e6)
        return {"device_ms": round(sum(ms), 4), "launches": len(ms),
                "per_rank_compute_ms": round(compute, 4), "link_ms": round(link_ms, 4),
                "per_rank_ms": round(compute + link_ms, 4), "bytes_sent_per_rank": sent}
