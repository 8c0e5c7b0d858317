"""Benchmark of the codec hot path on one GB300 (replicas across GPUs).

One step runs every hot-path kernel once, each from its own inputs already
resident in HBM:

  range + compress   512^3 FP32 Gaussian random field (P(k) ~ k^-3, scaled to
                     [-1, 1], 512 MiB), relative bound 1e-3, L = 32
  decompress         that stream -> FP32 field
  ring Allreduce     8 rank images of 8192^2 FP32 (shared base + per-rank
                     Poisson noise), bound fixed at 1e-3 of the range: initial
                     compression, 7 fused decode + add + re-encode steps (one
                     batched launch each), the Allgather stage's batched
                     decompression
  scatter pack       8 segments compressed as independent packed streams
  batched compress   1000 messages, 4 KiB - 64 MiB log-uniform, half FP32 /
                     half BF16, Student-t(3) x sigma, eb = 1e-3 sigma: one
                     persistent launch (autotuned block size, tile and grid)
                     from a CUDA graph
  selector path      a held-out mixed workload (about 4 GiB of the four
                     workload kinds) cut into 64 KiB chunks: statistics, the
                     bits and time networks, selection of block size or raw,
                     batched compression, all from one CUDA graph (networks
                     trained at set-up on 10^5 chunks by the library's own
                     gradient and SGD kernels; time labels from the codec
                     timed on groups of similar training chunks)

``value`` is the algorithmic bytes of one step (every kernel's input read
plus output written, the extra input read of the relative bound included)
divided by the device time of the step (CUDA events on the launch stream),
summed over ranks.  Inputs exceed the 129 MB L2, so no flush is needed.
``e2e`` repeats the step through the same C ABI with every input copied from
pinned host memory and every compressed output copied back, in the timed
region (copies on their own streams, each row waiting only for its input).  ``batched`` and ``selector`` report the comparisons of those two
paths with the plain per-message form.

--impl reference times the CPU oracle (test infrastructure, the only other
place this file runs it) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress/decompress/fused-reduce GB/s vs HBM peak; ratio at stated eb"
P_RING = 8
BLOCK = 32
REL = 1e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--chunks", type=int, default=0, help="2048-element chunks per CTA tile")
    ap.add_argument("--train-chunks", type=int, default=100000,
                    help="64 KiB chunks the selector's network is trained on")
    ap.add_argument("--heldout-gib", type=float, default=4.0,
                    help="size of the selector's held-out mixed workload")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--ring-ranks", type=int, default=8)
    ap.add_argument("--ring-side", type=int, default=8192, help="rank image side (8192 = 64 Mi)")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the compressor's size sweep")
    ap.add_argument("--collective-ranks", default="8,32,64",
                    help="rank counts of the ring vs recursive-doubling report ('' = none)")
    ap.add_argument("--batch-messages", type=int, default=1000,
                    help="messages of the batched-compression workload (1000 = the full one)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs.  Entering
    waits (at most 5 s) for the tool's first sample, so that the samples
    after it fall inside the timed region; only those are summarised."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t_end = time.time() + 5.0
            while not self.lines and self.proc.poll() is None and time.time() < t_end:
                time.sleep(0.01)
            self.first = len(self.lines)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.first:] or self.lines
        for ln in lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal


def kernel_times(samples):
    """Mean, median and best (minimum) of every kernel's per-step durations."""
    return ({k: statistics.mean(v) for k, v in samples.items()},
            {k: statistics.median(v) for k, v in samples.items()},
            {k: min(v) for k, v in samples.items()})


# The sources the encoder kernels (k_compress, k_batch, k_reduce, k_scatter) are
# built from: a DRAM-traffic figure taken with ncu stays valid while these are
# unchanged.
ENCODER_SOURCES = ("zc_device.cuh", "zc_codec.cuh", "zc_launch.h", "zc_kbatch.cu",
                   "zc_kenc.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2308_05199_gb300", "csrc")
    for name in ENCODER_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("source_hash") == source_hash():
            return e
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------
# our arm

class Workload:
    """Device buffers and launch descriptors for one bench step."""

    def __init__(self, torch, zc, workloads, side, device):
        self.torch, self.zc = torch, zc
        self.n = n = side ** 3
        self.field = workloads.grf_3d(side=side, seed=2000, device=device)
        t = torch
        self.stream = t.cuda.Stream(device=device)  # capturable (not the legacy stream)
        self.s = self.stream.cuda_stream
        self.ws = zc.Workspace(n, P_RING + 1, device, self.stream)
        self.cap = zc.zc_max_compressed_bytes(n, BLOCK)
        self.cmp = t.empty(self.cap, dtype=t.uint8, device=device)
        self.cmp_n = t.zeros(1, dtype=t.int64, device=device)
        self.dec = t.empty(n, dtype=t.float32, device=device)
        # ring bound: fixed once from the field range (relative 1e-3)
        mm = t.zeros(2, dtype=t.float32, device=device)
        assert zc.zc_minmax(self.field.data_ptr(), n, 0, mm.data_ptr(), self.ws.ptr,
                            self.ws.nbytes, self.s) == 0
        self.stream.synchronize()
        lo, hi = mm.tolist()
        self.eb_abs = REL * (float(hi) - float(lo))
        self.m = n // P_RING
        self.ccap = zc.zc_max_compressed_bytes(self.m, BLOCK)
        # scatter pack: 8 segments of the field
        self.counts = [self.m] * P_RING
        self.displs = [r * self.m for r in range(P_RING)]
        import ctypes
        self.hc = (ctypes.c_uint64 * P_RING)(*self.counts)
        self.hd = (ctypes.c_uint64 * P_RING)(*self.displs)
        self.pcap = P_RING * self.ccap
        self.packed = t.empty(self.pcap, dtype=t.uint8, device=device)
        self.seg = t.zeros(P_RING + 1, dtype=t.int64, device=device)
        # range, compress; width scan, decompress; scatter pack; batched compress
        # (tile map, persistent kernel); selector (statistics, MLP, selection, the
        # three grouping kernels, batched compress); the ring adds its own
        self.launches_per_step = 14

    # the rows of one step, in step order: (name, input buffer index or None)
    ROWS = ("compress", "decompress", "ring_allreduce", "scatter_pack", "batched_compress",
            "selector_compress")

    def run_row(self, k):
        zc, s, ws = self.zc, self.s, self.ws
        if k == 0:
            assert zc.zc_compress(self.field.data_ptr(), self.n, 0, zc.EB_REL, REL, BLOCK,
                                  self.cmp.data_ptr(), self.cap, self.cmp_n.data_ptr(), ws.ptr,
                                  ws.nbytes, s) == 0
        elif k == 1:
            assert zc.zc_decompress(self.cmp.data_ptr(), self.cap, self.dec.data_ptr(), self.n, 0,
                                    ws.ptr, ws.nbytes, s) == 0
        elif k == 2:
            self.ring_row.ring.run()
        elif k == 3:
            assert zc.zc_scatter_pack(self.field.data_ptr(), 0, P_RING, self.hc, self.hd,
                                      zc.EB_ABS, self.eb_abs, BLOCK, self.packed.data_ptr(),
                                      self.pcap, self.seg.data_ptr(), ws.ptr, ws.nbytes, s) == 0
        elif k == 4:
            self.batch_row.graph.launch()
        else:
            self.sel_row.graph.launch()

    def step(self, ev=None, waits=None, order=None):
        """One pass of every row on the step's stream.  ev: 7 events, ev[0]
        before the first row and ev[k + 1] after row k; waits: events the
        stream waits for before row k (the end-to-end run's input copies);
        order: the rows' order (step order by default; every row runs once,
        decompression after compression)."""
        st = self.stream
        waits = waits or {}
        if ev:
            ev[0].record(st)
        for k in (order or range(len(self.ROWS))):
            if k in waits:
                st.wait_event(waits[k])
            self.run_row(k)
            if ev:
                ev[k + 1].record(st)

    def sizes(self):
        C = int(self.cmp_n.item())
        packed = int(self.seg[-1].item())
        n4 = 4 * self.n
        parts = {
            "compress": n4 + n4 + C,          # range read + compress read + stream write
            "decompress": C + n4,
            "ring_allreduce": self.ring_row.step_bytes(),
            "scatter_pack": n4 + packed,
            "batched_compress": self.batch_row.step_bytes(),
            "selector_compress": self.sel_row.step_bytes(),
        }
        return C, parts


def ring_step_bytes(P, n, stage):
    """Algorithmic bytes of one ring Allreduce of P ranks of n FP32 elements;
    stage[t] = total length of the P streams written at stage t (0: the first
    compression of every rank's own chunk, t = 1 .. P - 1: the fused steps).
      first compression   one chunk of every rank read (4n in all), stage 0 written
      step t              stage t - 1 read, one local chunk per rank (4n), stage t written
      last step           also the FP32 sums of the owned chunks (4n)
      Allgather           every final stream decoded by the P - 1 other ranks"""
    tot = 4 * n + stage[0]
    for t in range(1, P):
        tot += stage[t - 1] + 4 * n + stage[t]
    tot += 4 * n
    tot += (P - 1) * (stage[P - 1] + 4 * n)
    return tot


def ring_errors(torch, ranks, out, eb_abs):
    """Largest |result - exact FP64 sum| of a ring Allreduce, split into the
    chunk each rank reduced itself (owned) and the chunks it decoded in the
    Allgather stage: in units of eb, and over the provable per-element bounds
    (ring_error_bounds: (P - 1) eb owned, P eb decoded, plus the FP32
    roundings) and, for the owned chunks, over the stated target (P - 1) eb
    + 1e-6 sum|x| (ring_target_bound).  Ratios <= 1 mean the bound holds."""
    from paper_2308_05199_gb300.collectives import (chunk_bounds, ring_error_bounds,
                                                    ring_target_bound)
    import numpy as np
    P, n = len(ranks), ranks[0].numel()
    dev = ranks[0].device
    exact = torch.zeros(n, dtype=torch.float64, device=dev)
    absum = torch.zeros_like(exact)
    for x in ranks:
        exact += x.double()
        absum += x.double().abs()
    eb = float(np.float32(eb_abs))
    own_b, dec_b = ring_error_bounds(P, eb, absum)
    tgt = ring_target_bound(P, eb, absum)
    B = chunk_bounds(n, P)
    w = {"owned_err_over_eb": 0.0, "decoded_err_over_eb": 0.0, "owned_over_provable": 0.0,
         "decoded_over_provable": 0.0, "owned_over_target": 0.0}
    for r in range(P):
        err = (out[r].double() - exact).abs()
        c = (r + 1) % P
        mine = torch.zeros(n, dtype=torch.bool, device=dev)
        mine[B[c]:B[c + 1]] = True
        e_own, e_dec = err[mine], err[~mine]
        w["owned_err_over_eb"] = max(w["owned_err_over_eb"], float(e_own.max()) / eb)
        w["owned_over_provable"] = max(w["owned_over_provable"],
                                       float((e_own / own_b[mine]).max()))
        w["owned_over_target"] = max(w["owned_over_target"], float((e_own / tgt[mine]).max()))
        if e_dec.numel():
            w["decoded_err_over_eb"] = max(w["decoded_err_over_eb"], float(e_dec.max()) / eb)
            w["decoded_over_provable"] = max(w["decoded_over_provable"],
                                             float((e_dec / dec_b[~mine]).max()))
    del exact, absum, own_b, dec_b, tgt
    out_ = {k: round(v, 4) for k, v in w.items()}
    out_.update({"eb_abs": eb, "bound_owned_over_eb": P - 1, "bound_decoded_over_eb": P,
                 "target": "(P - 1) eb + 1e-6 sum|x| per element, owned chunks"})
    return out_


def pack_tensors(torch, ts, device):
    """One device buffer holding every tensor of ts at 256-byte aligned offsets,
    and views of it in place of the tensors (so a whole workload moves
    between host and device in one copy)."""
    offs, tot = [], 0
    for t in ts:
        offs.append(tot)
        tot += (t.numel() * t.element_size() + 255) // 256 * 256
    buf = torch.empty(max(tot, 256), dtype=torch.uint8, device=device)
    views = []
    for t, o in zip(ts, offs):
        nbytes = t.numel() * t.element_size()
        v = buf[o:o + nbytes].view(t.dtype)
        v.copy_(t.reshape(-1))
        views.append(v)
    return buf, views


class RingRow:
    """The image-stacking ring Allreduce: P rank images of 8192^2 FP32 (a
    shared base of 8 plane waves plus per-rank standardized Poisson(50) noise
    at 1e-2), the bound fixed once as 1e-3 of the largest rank range; initial
    compression, P - 1 fused steps, the Allgather stage's batched
    decompression."""

    def __init__(self, torch, zc, workloads, stream, device, P=8, side=8192):
        from paper_2308_05199_gb300.collectives import RingAllreduce
        self.torch, self.P = torch, P
        with torch.cuda.stream(stream):
            base = workloads.stacking_base(side=side, seed=3000, device=device)
            ranks = [workloads.stacking_rank(base, r, seed=3000) for r in range(P)]
            rng = max(float(x.max() - x.min()) for x in ranks)
            self.buf, self.ranks = pack_tensors(torch, ranks, device)
        stream.synchronize()
        del base, ranks
        self.eb_abs = REL * rng
        self.ring = RingAllreduce(self.ranks, self.eb_abs, BLOCK, stream=stream)
        self.n = self.ranks[0].numel()
        # launches: initial compression (tile map + fused kernel), P - 1 steps
        # (width scan + tile map + fused kernel), Allgather (width scan + tile map +
        # decompression)
        self.launches = 2 + 3 * (P - 1) + 3

    def step_bytes(self):
        """Algorithmic bytes of one Allreduce (ring_step_bytes over the
        stream lengths of every stage)."""
        sz = self.ring.sizes.cpu()
        return ring_step_bytes(self.P, self.n, [int(sz[t].sum()) for t in range(self.P)])

    def errors(self):
        """Largest |result - exact FP64 sum| over all ranks (ring_errors)."""
        return ring_errors(self.torch, self.ranks, self.ring.out, self.eb_abs)


class BatchRow:
    """Batched compression of the 1000-message workload: one persistent
    launch (block size, tile size and grid from the library's autotuner) in a
    CUDA graph, against the plain form (one zc_compress per message at the
    same block size)."""

    def __init__(self, torch, zc, workloads, stream, device, M=1000):
        self.torch, self.zc, self.stream = torch, zc, stream
        self.M = M
        specs = workloads.message_specs(self.M)
        with torch.cuda.stream(stream):
            xs = [workloads.message(sp, device=device) for sp in specs]
            self.buf, self.xs = pack_tensors(torch, xs, device)
        stream.synchronize()
        del xs
        self.ebs = [sp["eb"] for sp in specs]
        self.raw = sum(x.numel() * x.element_size() for x in self.xs)
        self.n_f32 = sum(1 for sp in specs if sp["dtype"] == "f32")
        self.b = zc.BatchCompress(self.xs, [32] * self.M, self.ebs, stream=stream)
        # the library's autotuner over block size, tile size and grid (the
        # fastest candidate: no link term)
        self.best, self.points = self.b.autotune(tune_block=True, link_gbs=0.0, reps=3,
                                                 stream=stream)
        self.b.run(stream)
        stream.synchronize()
        self.graph = zc.Graph(stream)
        with self.graph.capture():
            self.b.run(stream)

    def step_bytes(self):
        return self.raw + int(self.b.msg_off[-1].item())

    def compare(self, reps=5):
        """Device ms of the graph launch vs the per-message loop (same streams
        byte for byte: checked on the total length)."""
        torch, zc, st = self.torch, self.zc, self.stream
        outs = [torch.empty(zc.zc_max_compressed_bytes(x.numel(), 16), dtype=torch.uint8,
                            device=x.device) for x in self.xs]
        obs = torch.zeros(self.M, dtype=torch.int64, device=self.xs[0].device)
        ws = self.b.ws

        L = self.best["block"]

        def loop():
            for i, x in enumerate(self.xs):
                zc._check(zc.zc_compress(x.data_ptr(), x.numel(), zc.dtype_code(x), zc.EB_ABS,
                                         self.ebs[i], L, outs[i].data_ptr(), outs[i].numel(),
                                         obs.data_ptr() + 8 * i, ws.ptr, ws.nbytes,
                                         st.cuda_stream), "zc_compress")

        def timed(f):
            f()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                f()
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        loop_ms = timed(loop)
        batch_ms = timed(self.graph.launch)
        same = int(obs.sum().item()) == int(self.b.msg_off[-1].item())
        del outs
        return {"messages": self.M, "fp32_messages": self.n_f32, "raw_bytes": self.raw,
                "ratio": round(self.raw / int(self.b.msg_off[-1].item()), 4),
                "per_message_loop_ms": round(loop_ms, 3), "batched_graph_ms": round(batch_ms, 3),
                "speedup": round(loop_ms / batch_ms, 2),
                "per_message_loop_gbs": round(self.step_bytes() / loop_ms / 1e6, 1),
                "batched_gbs": round(self.step_bytes() / batch_ms / 1e6, 1),
                "same_total_bytes": same,
                "autotuned": {"block": self.best["block"], "tile_chunks": self.best["tile_chunks"],
                              "grid": self.best["grid"], "candidates": len(self.points)}}


class SelectorRow:
    """The learned per-chunk selector on a held-out mixed workload: network
    trained at set-up (10^5 chunks of the four workload kinds, labels from the
    codec at every L), then statistics + MLP + selection + batched compression
    from one CUDA graph."""

    LINK_GBS = 12.5  # the paper's 100 Gb/s network, as a model parameter

    def __init__(self, torch, zc, stream, device, train_chunks, heldout_bytes, epochs):
        import numpy as np
        from paper_2308_05199_gb300 import selector as S
        self.torch, self.zc, self.S, self.stream = torch, zc, S, stream
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            tv, te, _ = S.mixed_chunks(train_chunks, seed=1, device=device)
        tr = S.ChunkBatch(tv, te, stream=stream)
        self.cfg = {}
        for link in (self.LINK_GBS, 100.0):
            self.cfg[link] = tr.cost_model(link_gbs=link)
        self.uniform_ns = [round(v, 6) for v in tr.uniform_ns_per_byte]
        X, T, keep, bits = S.dataset(tr)
        # time labels: the codec timed on groups of similar training chunks
        rates, _ = S.time_labels(tv, te, bits, groups=16, stream=stream)
        TT = torch.from_numpy(np.log2(rates[keep]).astype(np.float32)).to(device)
        self.mlp = S.Mlp(seed=0)
        self.mlp.set_norm(X)
        self.tmlp = S.Mlp(seed=1)
        self.tmlp.set_norm(X)
        t1 = time.perf_counter()
        self.hist = self.mlp.fit(X, T, epochs=epochs, batch=256, lr=0.02, momentum=0.9, seed=0,
                                 stream=stream)
        self.thist = self.tmlp.fit(X, TT, epochs=epochs, batch=256, lr=0.02, momentum=0.9,
                                   seed=1, stream=stream)
        stream.synchronize()
        self.train_s = time.perf_counter() - t1
        self.n_train = int(keep.sum())
        self.setup_s = t1 - t0
        del tr, tv, te, X, T, TT
        torch.cuda.empty_cache()
        with torch.cuda.stream(stream):
            xs, ebs, kinds = S.mixed_messages(heldout_bytes, seed=7, device=device)
            self.buf, xs = pack_tensors(torch, xs, device)
        stream.synchronize()
        self.xs, self.ebs = xs, ebs
        hv, he = S.split_chunks(xs, ebs)
        self.heldout_ebs = he
        self.cb = S.ChunkBatch(hv, he, stream=stream)
        cfg = self.cfg[self.LINK_GBS]
        self.cb.run_selected(cfg, self.mlp, self.tmlp)
        stream.synchronize()
        self.graph = zc.Graph(stream)
        with self.graph.capture():
            self.cb.run_selected(cfg, self.mlp, self.tmlp)

    def step_bytes(self):
        # sampled statistics read + codec read + packed write (the network and
        # the selection touch a few bytes per chunk)
        sample = int(sum(min(v.numel(), 2048) * v.element_size() for v in self.cb.views))
        return sample + self.cb.raw_bytes + int(self.cb.batch.msg_off[-1].item())

    def breakdown(self, cfg, reps=3):
        """Device ms of each launch of the learned selector path, and of the
        batched decompression of its output."""
        torch, zc, st, cb = self.torch, self.zc, self.stream, self.cb
        parts = [("stats", cb.stats),
                 ("mlp_forward", lambda: self.mlp.forward(cb.feat, out=cb.pred, stream=st)),
                 ("mlp_forward_time", lambda: self.tmlp.forward(cb.feat, out=cb.pred_time,
                                                                stream=st)),
                 ("select", lambda: cb.select(cfg, cb.pred, cb.pred_time)),
                 ("compress", lambda: cb.batch.run(st)),
                 ("decompress", lambda: cb.dec.run(st))]
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)]
               for _ in range(reps + 1)]
        for r in range(reps + 1):
            evs[r][0].record(st)
            for i, (_, f) in enumerate(parts):
                f()
                evs[r][i + 1].record(st)
        st.synchronize()
        return {nm: round(statistics.median(evs[r][i].elapsed_time(evs[r][i + 1])
                                            for r in range(1, reps + 1)), 4)
                for i, (nm, _) in enumerate(parts)}

    def report(self, reps=3):
        """Mispredicts and modelled end-to-end GB/s of the plain per-message
        form, the batched heuristic and the batched learned selector (bits
        network alone, and with the time network)."""
        import numpy as np
        torch, zc, S, st = self.torch, self.zc, self.S, self.stream
        cb = self.cb
        bits = cb.true_bits()
        # the held-out chunks' own codec rates, measured like the training labels
        hrates, _ = S.time_labels(cb.views, [float(e) for e in self.heldout_ebs], bits,
                                  groups=16, stream=st)
        cb.stats()
        pt = self.tmlp.forward(cb.feat, out=cb.pred_time, stream=st)
        cb.sync()
        okr = torch.isfinite(cb.feat).all(1).cpu().numpy()
        lt = np.log2(hrates[okr])
        uni = np.log2(np.array(self.uniform_ns))[None, :]
        ev = lambda: torch.cuda.Event(enable_timing=True)
        out = {"train_chunks": self.n_train, "epochs": len(self.hist),
               "loss_first": round(self.hist[0], 5), "loss_last": round(self.hist[-1], 5),
               "time_loss_first": round(self.thist[0], 5),
               "time_loss_last": round(self.thist[-1], 5),
               "time_rmse_log2": {
                   "network": round(float(np.sqrt(np.mean(
                       (pt.cpu().numpy().astype(np.float64)[okr] - lt) ** 2))), 4),
                   "batch_wide_rate": round(float(np.sqrt(np.mean((uni - lt) ** 2))), 4)},
               "train_s": round(self.train_s, 2), "heldout_chunks": cb.M,
               "heldout_bytes": cb.raw_bytes, "messages": len(self.xs), "links": {}}
        # plain per-message form: one zc_compress + one zc_decompress per whole message, L = 32
        outs = [torch.empty(zc.zc_max_compressed_bytes(x.numel(), 32), dtype=torch.uint8,
                            device=x.device) for x in self.xs]
        decs = [torch.empty_like(x) for x in self.xs]
        obs = torch.zeros(len(self.xs), dtype=torch.int64, device=self.xs[0].device)
        ws = cb.batch.ws

        def plain():
            for i, x in enumerate(self.xs):
                zc._check(zc.zc_compress(x.data_ptr(), x.numel(), zc.dtype_code(x), zc.EB_ABS,
                                         self.ebs[i], 32, outs[i].data_ptr(), outs[i].numel(),
                                         obs.data_ptr() + 8 * i, ws.ptr, ws.nbytes,
                                         st.cuda_stream), "zc_compress")
            for i, x in enumerate(self.xs):
                zc._check(zc.zc_decompress(outs[i].data_ptr(), outs[i].numel(), decs[i].data_ptr(),
                                           x.numel(), zc.dtype_code(x), ws.ptr, ws.nbytes,
                                           st.cuda_stream), "zc_decompress")

        def timed(f):
            f()
            e0, e1 = ev(), ev()
            e0.record(st)
            for _ in range(reps):
                f()
            e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        plain_ms = timed(plain)
        plain_bytes = int(obs.sum().item())
        raw = cb.raw_bytes
        for link, cfg in self.cfg.items():
            rec = {"plain_per_message": {
                "device_ms": round(plain_ms, 3), "bytes": plain_bytes,
                "e2e_gbs": round(raw / (plain_ms * 1e6 + plain_bytes / link), 3)}}
            for name, mlp, tmlp in (("batched_heuristic", None, None),
                                    ("batched_learned_bits_only", self.mlp, None),
                                    ("batched_learned", self.mlp, self.tmlp)):
                ms = timed(lambda: (cb.run_selected(cfg, mlp, tmlp), cb.dec.run(st)))
                choice = cb.choice.cpu().numpy().copy()
                counts = cb.counts.cpu().numpy()
                ev_ = S.evaluate(choice, cb.n, cb.es, bits, cfg)
                evr = S.evaluate(choice, cb.n, cb.es, bits, cfg, rates=hrates)
                packed = int(cb.batch.msg_off[-1].item())
                rec[name] = {"device_ms": round(ms, 3), "bytes": packed,
                             "e2e_gbs": round(raw / (ms * 1e6 + packed / link), 3),
                             "mispredict": round(ev_["mispredict"], 4),
                             "regret": round(ev_["regret"], 5),
                             "mispredict_measured_rates": round(evr["mispredict"], 4),
                             "regret_measured_rates": round(evr["regret"], 5),
                             "raw_frac": round(ev_["raw_frac"], 4),
                             "fallbacks": int(counts[0]) if mlp is not None else None,
                             "blocks": {str(b): int((choice == b).sum())
                                        for b in (16, 32, 64, 128, 0)}}
            rec["cost_model_ns_per_byte"] = {"coded_mixed": cfg.ns_per_byte[0],
                                              "raw": cfg.raw_ns_per_byte,
                                              "uniform_L16_L32_L64_L128": self.uniform_ns}
            out["links"][str(link)] = rec
        out["breakdown_ms"] = self.breakdown(self.cfg[self.LINK_GBS])
        # leave the plan as the graph expects it
        cb.run_selected(self.cfg[self.LINK_GBS], self.mlp, self.tmlp)
        st.synchronize()
        del outs, decs
        return out


def heads_report(torch, zc, W, reps=5):
    """The heads-apart format against the plain one on the 512^3 field and on
    the same field shifted by +100 (a DC offset far above eb = 2e-3): ratio
    and compression / decompression GB/s (L = 32, absolute bound of the REL
    1e-3 field)."""
    st = W.stream
    s = st.cuda_stream
    n = W.n
    eb = REL * 2.0  # the field spans [-1, 1]
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(f):
        f()
        e0, e1 = ev(), ev()
        e0.record(st)
        for _ in range(reps):
            f()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    shifted = torch.empty_like(W.field)
    with torch.cuda.stream(st):
        shifted.copy_(W.field)
        shifted.add_(100.0)
    cap = zc.zc_max_compressed_bytes_heads(n, BLOCK)
    buf = torch.empty(cap, dtype=torch.uint8, device=W.field.device)
    nb = torch.zeros(1, dtype=torch.int64, device=W.field.device)
    for name, x in (("field", W.field), ("field_plus_100", shifted)):
        rec = {}
        for fmt, fn in (("plain", zc.zc_compress), ("heads_apart", zc.zc_compress_heads)):
            c = lambda: zc._check(fn(x.data_ptr(), n, zc.F32, zc.EB_ABS, eb, BLOCK, buf.data_ptr(),
                                     cap, nb.data_ptr(), W.ws.ptr, W.ws.nbytes, s), "compress")
            tc = timed(c)
            C = int(nb.item())
            d = lambda: zc._check(zc.zc_decompress(buf.data_ptr(), cap, W.dec.data_ptr(), n, zc.F32,
                                                   W.ws.ptr, W.ws.nbytes, s), "decompress")
            td = timed(d)
            rec[fmt] = {"ratio": round(4 * n / C, 3), "compress_gbs": round((4 * n + C) / tc / 1e6, 1),
                        "decompress_gbs": round((4 * n + C) / td / 1e6, 1)}
        out[name] = rec
    del shifted, buf
    torch.cuda.empty_cache()
    st_, _ = W.ws.status(st)
    out["status"] = st_
    return out


L2_BYTES = 129 << 20  # GB300 L2


def config1_report(torch, zc, workloads, stream, device, reps=20):
    """The small correctness workload: 2^20 FP32 sinusoids (4 MiB, fits in
    L2), absolute bound 1e-4, L = 32.  Before every timed call a buffer of
    twice the L2 size is written, so the input starts in HBM; compression
    and decompression are timed alone (CUDA events on the launch stream),
    best and median of `reps`.  GB/s on algorithmic bytes (compress: 4n + |C|;
    decompress: |C| + 4n); ratio; largest |x - x^| over eb."""
    n, eb = 1 << 20, 1e-4
    with torch.cuda.stream(stream):
        x = workloads.sinusoids_1d(n, seed=1000, device=device)
    stream.synchronize()
    s = stream.cuda_stream
    ws = zc.Workspace(n, 1, device, stream)
    cap = zc.zc_max_compressed_bytes(n, BLOCK)
    cmp = torch.empty(cap, dtype=torch.uint8, device=device)
    nb = torch.zeros(1, dtype=torch.int64, device=device)
    y = torch.empty(n, dtype=torch.float32, device=device)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=device)

    def comp():
        zc._check(zc.zc_compress(x.data_ptr(), n, zc.F32, zc.EB_ABS, eb, BLOCK, cmp.data_ptr(),
                                 cap, nb.data_ptr(), ws.ptr, ws.nbytes, s), "zc_compress")

    def dec():
        zc._check(zc.zc_decompress(cmp.data_ptr(), cap, y.data_ptr(), n, zc.F32, ws.ptr,
                                   ws.nbytes, s), "zc_decompress")

    def timed(f):
        ts = []
        for i in range(reps + 3):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f()
            e1.record(stream)
            e1.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        return min(ts), statistics.median(ts)

    cb, cm = timed(comp)
    C = int(nb.item())
    db, dm = timed(dec)
    eb_f = float(torch.tensor(eb, dtype=torch.float32))
    with torch.cuda.stream(stream):
        e = (y.double() - x.double()).abs()
        err = float(e.max())
        # the codec's bound: eb (of the quantization) plus half an FP32 ulp of x^
        over = float((e / (eb_f + 2.0 ** -24 * y.double().abs())).max())
    st, _ = ws.status(stream)
    del flush
    torch.cuda.empty_cache()
    return {"n": n, "eb_abs": eb, "block": BLOCK, "status": st, "ratio": round(4 * n / C, 3),
            "compress_ms_best": round(cb, 4), "compress_ms_median": round(cm, 4),
            "compress_gbs_best": round((4 * n + C) / cb / 1e6, 1),
            "compress_gbs_median": round((4 * n + C) / cm / 1e6, 1),
            "decompress_ms_best": round(db, 4), "decompress_ms_median": round(dm, 4),
            "decompress_gbs_best": round((4 * n + C) / db / 1e6, 1),
            "decompress_gbs_median": round((4 * n + C) / dm / 1e6, 1),
            "max_err_over_eb": round(err / eb_f, 6), "max_err_over_bound": round(over, 6),
            "bound": "eb + 2^-24 |x^| per element",
            "l2": "flushed before every call (%d MB written)" % (2 * L2_BYTES >> 20)}


def bound_sweep(torch, zc, W, rels=(1e-2, 1e-3, 1e-4), reps=5):
    """The 512^3 field at three relative bounds (range + compress, and
    decompress, L = 32): ratio, GB/s (algorithmic bytes as the step's rows)
    and the largest error over eb, checked on the device."""
    st = W.stream
    s = st.cuda_stream
    n = W.n
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(f):
        f()
        e0, e1 = ev(), ev()
        e0.record(st)
        for _ in range(reps):
            f()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = []
    lo, hi = float(W.field.min()), float(W.field.max())
    for rel in rels:
        c = lambda: zc._check(zc.zc_compress(W.field.data_ptr(), n, zc.F32, zc.EB_REL, rel, BLOCK,
                                             W.cmp.data_ptr(), W.cap, W.cmp_n.data_ptr(), W.ws.ptr,
                                             W.ws.nbytes, s), "compress")
        tc = timed(c)
        C = int(W.cmp_n.item())
        d = lambda: zc._check(zc.zc_decompress(W.cmp.data_ptr(), W.cap, W.dec.data_ptr(), n, zc.F32,
                                               W.ws.ptr, W.ws.nbytes, s), "decompress")
        td = timed(d)
        eb = float(torch.tensor(rel * (hi - lo), dtype=torch.float32))
        with torch.cuda.stream(st):
            e = (W.dec.double() - W.field.double()).abs()
            err = float(e.max())
            over = float((e / (eb + 2.0 ** -24 * W.dec.double().abs())).max())
            del e
        out.append({"rel": rel, "eb_abs": eb, "ratio": round(4 * n / C, 3),
                    "compress_gbs": round((8 * n + C) / tc / 1e6, 1),
                    "decompress_gbs": round((4 * n + C) / td / 1e6, 1),
                    "max_err_over_eb": round(err / eb, 4),
                    "max_err_over_bound": round(over, 6)})
    st.synchronize()
    return {"status": W.ws.status()[0], "points": out}


def size_sweep(torch, zc, workloads, stream, device, max_bytes=646 << 20, reps=5):
    """Compression / decompression time over message sizes (the paper's
    characterization of its GPU compressor, Sec. 3.2.2, on uniform synthetic
    data up to 646 MB): one plain call per message against the same bytes cut
    into messages of that size and compressed in one batched launch.  Absolute
    bound 1e-3, L = 32, FP32."""
    out = []
    total = max_bytes // 4
    with torch.cuda.stream(stream):
        x = workloads.uniform(total, seed=6000, device=device)
    stream.synchronize()
    ws = zc.Workspace(total, 4096, device, stream)
    cap = zc.zc_max_compressed_bytes(total, BLOCK)
    cmp = torch.empty(cap, dtype=torch.uint8, device=device)
    dec = torch.empty(total, dtype=torch.float32, device=device)
    nb = torch.zeros(1, dtype=torch.int64, device=device)
    s = stream.cuda_stream
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(f):
        f()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(reps):
            f()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    size = 4096
    while size <= max_bytes:
        n = size // 4
        c = lambda: zc._check(zc.zc_compress(x.data_ptr(), n, zc.F32, zc.EB_ABS, 1e-3, BLOCK,
                                             cmp.data_ptr(), cap, nb.data_ptr(), ws.ptr,
                                             ws.nbytes, s), "zc_compress")
        d = lambda: zc._check(zc.zc_decompress(cmp.data_ptr(), cap, dec.data_ptr(), n, zc.F32,
                                               ws.ptr, ws.nbytes, s), "zc_decompress")
        tc = timed(c)
        td = timed(d)
        M = min(total // n, 4096)
        views = [x[i * n:(i + 1) * n] for i in range(M)]
        b = zc.BatchCompress(views, [BLOCK] * M, [1e-3] * M, ws=ws, stream=stream)
        bd = zc.BatchDecompress(b.packed, b.msg_off, [dec[i * n:(i + 1) * n] for i in range(M)],
                                ws=ws, stream=stream)
        tb = timed(lambda: b.run(stream))
        tbd = timed(lambda: bd.run(stream))
        out.append({"bytes": size, "plain_compress_us": round(tc * 1e3, 2),
                    "plain_decompress_us": round(td * 1e3, 2),
                    "plain_compress_gbs": round(size / tc / 1e6, 1),
                    "plain_decompress_gbs": round(size / td / 1e6, 1),
                    "batched_messages": M,
                    "batched_compress_us_per_message": round(tb * 1e3 / M, 3),
                    "batched_decompress_us_per_message": round(tbd * 1e3 / M, 3),
                    "batched_compress_gbs": round(size * M / tb / 1e6, 1),
                    "batched_decompress_gbs": round(size * M / tbd / 1e6, 1)})
        del b, bd, views
        size = size * 4 if size * 4 <= max_bytes or size == max_bytes else max_bytes
    st, _ = ws.status(stream)
    del x, cmp, dec
    torch.cuda.empty_cache()
    return {"status": st, "points": out}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value over all ranks: a replicated job's time is its
    slowest rank's (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(step_bytes: int, world: int, ms_per_step: float) -> float:
    """Whole-job GB/s of N replicas, each moving step_bytes per step (weak
    scaling: the work per GPU is fixed)."""
    return step_bytes * world / (ms_per_step * 1e-3) / 1e9


def collectives_report(torch, workloads, stream, device, ranks_list, side, reps=2):
    """Ring vs recursive-doubling Allreduce on the image-stacking workload for
    each rank count: measured device time, the modelled per-rank time with one
    GPU per rank at 12.5 and 100 GB/s links, the largest error against the
    exact FP64 sum (the ring: ring_errors, against its provable bounds and
    the stated target; recursive doubling: in units of eb with the
    FP32-addition slack removed), and the algorithm the model picks (the paper's ring / recursive-doubling
    choice, Sec. 3.3.3)."""
    from paper_2308_05199_gb300 import collectives as C
    out = []
    for P in ranks_list:
        with torch.cuda.stream(stream):
            base = workloads.stacking_base(side=side, seed=3000, device=device)
            ranks = [workloads.stacking_rank(base, r, seed=3000) for r in range(P)]
            del base
            eb = REL * max(float(x.max() - x.min()) for x in ranks)
            exact = torch.zeros(ranks[0].numel(), dtype=torch.float64, device=device)
            absum = torch.zeros_like(exact)
            for x in ranks:
                exact += x.double()
                absum += x.double().abs()
        stream.synchronize()
        rec = {"ranks": P, "n_per_rank": ranks[0].numel(), "eb_abs": eb}
        k = P.bit_length() - 1
        for name, cls in (("ring", C.RingAllreduce), ("recursive_doubling",
                                                     C.RecursiveDoublingAllreduce)):
            alg = cls(ranks, eb, BLOCK, stream=stream)
            alg.run()
            stream.synchronize()
            if name == "ring":
                errs = ring_errors(torch, ranks, alg.out, eb)
            else:
                worst = 0.0
                for r in range(P):
                    err = (alg.out[r].double() - exact).abs() - P * 2.0 ** -24 * absum
                    worst = max(worst, float((err / eb).max()))
            st, _ = alg.ws.status(stream)
            m12 = alg.model(12.5, reps)
            m100 = alg.model(100.0, reps)
            rec[name] = {"status": st, "device_ms": m12["device_ms"], "launches": m12["launches"],
                         "per_rank_ms_link12.5": m12["per_rank_ms"],
                         "per_rank_ms_link100": m100["per_rank_ms"],
                         "bytes_sent_per_rank": m12["bytes_sent_per_rank"]}
            if name == "ring":
                rec[name]["errors"] = errs
            else:
                # worst case e = (2^k - 1) eb (+ 2^k eb with remainder ranks, + eb folded)
                bound = (1 << k) - 1 + ((1 << k) + 1 if P > (1 << k) else 0)
                rec[name]["max_err_over_eb"] = round(worst, 3)
                rec[name]["bound_over_eb"] = bound
            del alg
            torch.cuda.empty_cache()
        for link in ("12.5", "100"):
            key = "per_rank_ms_link" + link
            rec["choice_link" + link] = min(("ring", "recursive_doubling"),
                                            key=lambda a: rec[a][key])
        out.append(rec)
        del ranks, exact, absum
        torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2308_05199_gb300 import build, workloads, zc

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if args.chunks:
        assert zc.zc_set_tile_chunks(args.chunks) == 0
    W = Workload(torch, zc, workloads, args.side, dev)
    W.batch_row = BatchRow(torch, zc, workloads, W.stream, dev, args.batch_messages)
    W.ring_row = RingRow(torch, zc, workloads, W.stream, dev, P=args.ring_ranks,
                         side=args.ring_side)
    W.launches_per_step += W.ring_row.launches
    W.sel_row = SelectorRow(torch, zc, W.stream, dev, args.train_chunks,
                            int(args.heldout_gib * (1 << 30)), args.epochs)
    args.warmup = max(args.warmup, 3)
    for _ in range(args.warmup):
        W.step()
    torch.cuda.synchronize()
    batched = W.batch_row.compare()
    selector = W.sel_row.report()
    sweep = size_sweep(torch, zc, workloads, W.stream, dev) if args.sweep else None
    heads = heads_report(torch, zc, W)
    bounds = bound_sweep(torch, zc, W)
    cfg1 = config1_report(torch, zc, workloads, W.stream, dev)
    coll = collectives_report(torch, workloads, W.stream, dev,
                              [int(v) for v in args.collective_ranks.split(",") if v],
                              args.ring_side) if args.collective_ranks else None
    W.step()  # the side reports reuse the step's buffers: sizes come from a step
    torch.cuda.synchronize()
    st, det = W.ws.status()
    if st != 0:
        raise RuntimeError("device status %d at %d during warm-up" % (st, det))
    C, parts = W.sizes()
    step_bytes = sum(parts.values())

    # timed region: K steps, per-kernel events on the launch stream
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(K)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")  # profilers can select the timed launches
        t0.record(W.stream)
        for k in range(K):
            W.step(evs[k])
        t1.record(W.stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    st, det = W.ws.status()
    if st != 0:
        raise RuntimeError("device status %d at %d in the timed region" % (st, det))
    names = ["compress", "decompress", "ring_allreduce", "scatter_pack", "batched_compress",
             "selector_compress"]
    samples = {nm: [evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K)]
               for i, nm in enumerate(names)}
    per, med, best = kernel_times(samples)
    ms_per_step = total_ms / K
    value = job_gbs(step_bytes, world, ms_per_step)
    hbm, peak_kind = peaks()
    kern_gbs = {nm: parts[nm] / (per[nm] * 1e-3) / 1e9 for nm in names}
    dom = max(names, key=lambda nm: per[nm])
    traffic = load_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(kern_gbs[dom], 1),
                "peak": hbm, "unit": "GB/s", "frac": round(kern_gbs[dom] / hbm, 4),
                "peak_kind": peak_kind,
                "frac_of_nominal": round(kern_gbs[dom] / HBM_NOMINAL_GBS, 4),
                "traffic": traffic["bytes_per_launch"] if traffic else None,
                "algorithmic_bytes": parts[dom]}
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic, seeded: 512^3 Gaussian random field (P(k)~k^-3) in place of the "
                "paper's RTM volumes; Student-t messages; mixed held-out workload of the four "
                "kinds",
        "config": {"workload": "grf512_rel1e-3_L32+stacking_ring8x8192sq+batch1000"
                               "+selector_heldout",
                   "n": W.n, "rel_eb": REL,
                   "eb_abs_ring": W.ring_row.eb_abs, "block": BLOCK,
                   "batch_block": W.batch_row.best["block"],
                   "ring_ranks": W.ring_row.P, "ring_n_per_rank": W.ring_row.n,
                   "scatter_segments": P_RING, "batch_messages": W.batch_row.M,
                   "selector_heldout_bytes": W.sel_row.cb.raw_bytes,
                   "selector_chunks": W.sel_row.cb.M,
                   "l2": "inputs larger than L2 (no flush)"},
        "ratio": round(4 * W.n / C, 3),
        "kernels_gbs": {k: round(v, 1) for k, v in kern_gbs.items()},
        "kernels_ms": {k: round(v, 4) for k, v in per.items()},
        "kernels_ms_median": {k: round(v, 4) for k, v in med.items()},
        "kernels_ms_best": {k: round(v, 4) for k, v in best.items()},
        "kernels_frac_of_hbm": {k: round(v / hbm, 4) for k, v in kern_gbs.items()},
        "roofline": roofline,
        "gpu_launches": W.launches_per_step * K,
        "clocks": clk.summary(),
        "batched": batched,
        "selector": selector,
        "ring": dict(W.ring_row.errors(), ranks=W.ring_row.P, n_per_rank=W.ring_row.n),
        "collectives": coll,
        "size_sweep": sweep,
        "heads_apart": heads,
        "bound_sweep": bounds,
        "config1": cfg1,
    }
    if not args.no_e2e:
        out["e2e"] = e2e_ours(torch, W, args, step_bytes, world)
    return out


def e2e_ours(torch, W, args, step_bytes, world):
    """The same step with every input (the two fields, the 1000 messages, the
    held-out workload) copied in from pinned host memory and every compressed
    output (the field's stream, both packed batches) copied back, inside the
    timed region.  Copies run on two copy streams beside the step's stream:
    each row waits only for its own input, and each output goes back as soon
    as its row is done (its length is read first), so the step's compute
    hides under the host link, which bounds this number (about 210 GB/s in,
    190 GB/s out, 340 GB/s both ways on this machine's host link)."""
    st = W.stream
    cs_in = torch.cuda.Stream(device=st.device)
    cs_out = torch.cuda.Stream(device=st.device)
    # every workload lives in one buffer per row: four copies in, three out
    # inputs in copy order; the rows run in the order their inputs arrive,
    # the ring (no output to copy back) last, so the tail after the last
    # input copy is one row's compute
    dev_in = [W.field, W.batch_row.buf, W.sel_row.buf, W.ring_row.buf]
    rows_in = [0, 4, 5, 2]  # the row that first reads each input
    order = [0, 1, 3, 4, 5, 2]
    host_in = [t.cpu().pin_memory() for t in dev_in]
    # outputs with the event recorded after the row that writes them
    outs = [(W.cmp, W.cmp_n[0:1], 1), (W.batch_row.b.packed, W.batch_row.b.msg_off[-1:], 5),
            (W.sel_row.cb.batch.packed, W.sel_row.cb.batch.msg_off[-1:], 6)]
    host_out = [torch.empty(o.numel(), dtype=torch.uint8).pin_memory() for o, _, _ in outs]
    host_len = torch.zeros(len(outs), dtype=torch.int64).pin_memory()
    K = max(3, args.steps // 4)
    stats = {"d2h": 0}

    def one():
        waits = {}
        with torch.cuda.stream(cs_in):
            for d, h, row in zip(dev_in, host_in, rows_in):
                d.copy_(h, non_blocking=True)
                e = torch.cuda.Event()
                e.record(cs_in)
                waits[row] = e
        ev = [torch.cuda.Event() for _ in range(7)]
        W.step(ev, waits, order)
        d2h = 0
        for i, (o, ln, row) in enumerate(outs):
            with torch.cuda.stream(cs_out):
                cs_out.wait_event(ev[row])
                host_len[i:i + 1].copy_(ln, non_blocking=True)
                e = torch.cuda.Event()
                e.record(cs_out)
            e.synchronize()
            c = int(host_len[i])
            with torch.cuda.stream(cs_out):
                host_out[i][:c].copy_(o[:c], non_blocking=True)
            d2h += c + 8
        torch.cuda.synchronize()
        stats["d2h"] = d2h

    for _ in range(2):
        one()
    torch.cuda.synchronize()
    walls = []
    t = time.perf_counter()
    for _ in range(K):
        t1 = time.perf_counter()
        one()  # ends with a device synchronize
        walls.append(time.perf_counter() - t1)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / K
    h2d = sum(h.numel() * h.element_size() for h in host_in)
    return {"value": round(step_bytes * world / dt / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": stats["d2h"],
            "ms_per_step": round(dt * 1e3, 3), "steps": K,
            # the mean above is the reported value; the median and the range of
            # the single steps show how the host link varies between steps
            "ms_per_step_median": round(statistics.median(walls) * 1e3, 3),
            "ms_per_step_min_max": [round(min(walls) * 1e3, 3), round(max(walls) * 1e3, 3)]}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and --impl reference)

def oracle_step(x, ring_ranks, sample_n, msgs, chunks):
    """The bench step on bounded samples, run by the CPU oracle; returns
    (seconds, algorithmic bytes).  Samples: the first sample_n elements of
    the field (range, compress, decompress, ring step over 8 chunks, scatter
    pack of 8 segments), the first messages of the 1000-message workload
    (one compression each), and 64 KiB chunks through the selector
    (statistics, network, choice, compression); the ring Allreduce on
    smaller rank images of the same recipe."""
    import numpy as np
    import oracle
    from oracle import selector as OS
    xs = x[:sample_n]
    m = sample_n // P_RING
    t0 = time.perf_counter()
    mn, mx = oracle.minmax(xs)
    eb = oracle.eb_from_rel(REL, mn, mx)
    s = oracle.compress(xs, eb, 5)
    oracle.decompress(s, sample_n)
    ring_eb = REL * max(float(r.max() - r.min()) for r in ring_ranks)
    ring_stage = []
    oracle.ring_allreduce(ring_ranks, ring_eb, 5, stage_bytes=ring_stage)
    packed, _ = oracle.scatter_pack(xs, [m] * P_RING, [r * m for r in range(P_RING)], eb, 5)
    batch_out = sum(len(oracle.compress(a, e, 5)) for a, e in msgs)
    feats = np.array([OS.chunk_stats(a, e) for a, e in chunks])
    params = OS.init_params(0).astype(np.float64)
    norm = np.concatenate([np.zeros(16), np.ones(16)])
    pred = OS.forward(params, norm, np.nan_to_num(feats))
    cfg = {"link_gbs": 12.5, "ns_per_byte": [0.0] * 4, "raw_ns_per_byte": 0.0, "judge_log2": 1.0}
    sel_out = 0
    for (a, e), f, y in zip(chunks, feats, pred):
        c, _ = OS.mlp_choice(a.size, a.itemsize, f, y, cfg)
        sel_out += len(oracle.compress_raw(a) if c == 0 else oracle.compress(a, e, c.bit_length() - 1))
    t3 = time.perf_counter()
    secs = t3 - t0
    n4 = 4 * sample_n
    P, nr = len(ring_ranks), ring_ranks[0].size
    ring_bytes = ring_step_bytes(P, nr, ring_stage)
    raw_msgs = sum(a.nbytes for a, _ in msgs)
    raw_chunks = sum(a.nbytes for a, _ in chunks)
    nbytes = (n4 + n4 + len(s)) + (len(s) + n4) + \
        ring_bytes + (n4 + len(packed)) + \
        (raw_msgs + batch_out) + (raw_chunks + sel_out)
    return secs, nbytes


def cpu_fields(side):
    """The field, 8 rank images of 512^2 (the ring's recipe), a sample of the 1000-message workload (the
    first messages that fit in 16 MiB together, at most 64) and 16 chunks of 64 KiB (8 of the field, 8 of
    the messages), as numpy arrays (BF16 as uint16 bits)."""
    import torch
    from paper_2308_05199_gb300 import workloads
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    x = workloads.grf_3d(side=side, seed=2000, device=dev).cpu().numpy()
    base = workloads.stacking_base(side=512, seed=3000, device=dev)
    ring = [workloads.stacking_rank(base, r, seed=3000).cpu().numpy() for r in range(P_RING)]
    msgs, tot = [], 0
    for sp in workloads.message_specs(1000):
        if tot + sp["n"] * (4 if sp["dtype"] == "f32" else 2) > 16 << 20:
            continue  # keep the sample bounded: skip (without drawing) what does not fit
        t = workloads.message(sp, device=dev)
        a = t.cpu().numpy() if t.dtype == torch.float32 else workloads.bf16_bits(t)
        msgs.append((a, sp["eb"]))
        tot += a.nbytes
        if len(msgs) >= 64:
            break
    eb_x = REL * float(x.max() - x.min())
    chunks = [(x[i * (x.size // 8):i * (x.size // 8) + 16384], eb_x) for i in range(8)]
    for a, e in msgs:
        if len(chunks) >= 16:
            break
        per = 65536 // a.itemsize
        chunks.append((a[:per], e))
    return x, ring, msgs, chunks


def _oracle_piece(args):
    """One core's share of the block-parallel oracle run: range, compress and
    decompress of one field segment (its own stream, at the common bound; the
    segment is read from shared memory, not copied), then the compression of
    its messages.  Returns algorithmic bytes."""
    shm_name, lo, hi, eb, msgs = args
    import numpy as np
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        seg = np.ndarray((hi - lo,), dtype=np.float32, buffer=shm.buf, offset=4 * lo)
        oracle.minmax(seg)
        s = oracle.compress(seg, eb, 5)
        oracle.decompress(s, seg.size)
        n4 = 4 * seg.size
        nbytes = (n4 + n4 + len(s)) + (len(s) + n4)
        del seg
    finally:
        shm.close()
    for a, e in msgs:
        nbytes += a.nbytes + len(oracle.compress(a, e, 5))
    return nbytes


def cpu_parallel(x, msgs, sample_n):
    """The oracle block-parallel over all host cores: the field sample split
    into one segment per core (independent blocks, as in a scatter pack),
    the messages dealt round-robin; one spawned process per core, the field
    shared with them through shared memory."""
    import multiprocessing as mp
    import numpy as np
    from multiprocessing import shared_memory
    cores = os.cpu_count() or 1
    xs = np.ascontiguousarray(x[:sample_n], dtype=np.float32)
    eb = REL * float(xs.max() - xs.min())
    m = (sample_n // cores) // 32 * 32
    shm = shared_memory.SharedMemory(create=True, size=max(xs.nbytes, 4))
    try:
        np.ndarray(xs.shape, dtype=np.float32, buffer=shm.buf)[:] = xs
        bounds = [(i * m, (i + 1) * m if i < cores - 1 else sample_n) for i in range(cores)]
        parts = [(shm.name, lo, hi, eb, msgs[i::cores]) for i, (lo, hi) in enumerate(bounds)]
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_piece, [(shm.name, 0, min(1024, sample_n), eb, [])] * cores)  # start-up
            t = time.perf_counter()
            nbytes = sum(pool.map(_oracle_piece, parts))
            secs = time.perf_counter() - t
    finally:
        shm.close()
        shm.unlink()
    return {"value": round(nbytes / secs / 1e9, 4), "unit": "GB/s", "cores": cores,
            "sample": "first %d elements of the field (range, compress, decompress) in %d "
                      "segments and the first %d messages, one spawned process per core"
                      % (sample_n, cores, len(msgs)),
            "seconds": round(secs, 2)}


def oracle_config1(reps=5):
    """The oracle on the small correctness workload (2^20 FP32 sinusoids,
    absolute bound 1e-4, L = 32), single-threaded: best and median of reps
    compressions and decompressions, GB/s on the same algorithmic bytes as
    the GPU's."""
    import oracle
    from paper_2308_05199_gb300 import workloads
    x = workloads.sinusoids_1d(1 << 20, seed=1000).numpy()
    n = x.size
    tc, td = [], []
    for _ in range(reps):
        t = time.perf_counter()
        s = oracle.compress(x, 1e-4, 5)
        tc.append(time.perf_counter() - t)
        t = time.perf_counter()
        oracle.decompress(s, n)
        td.append(time.perf_counter() - t)
    b = 4 * n + len(s)
    return {"cores": 1, "ratio": round(4 * n / len(s), 3),
            "compress_gbs_best": round(b / min(tc) / 1e9, 4),
            "compress_gbs_median": round(b / statistics.median(tc) / 1e9, 4),
            "decompress_gbs_best": round(b / min(td) / 1e9, 4),
            "decompress_gbs_median": round(b / statistics.median(td) / 1e9, 4)}


def cpu_baseline(side, sample_n=1 << 25):
    x, ring, msgs, chunks = cpu_fields(side)
    sample_n = min(sample_n, x.size)
    secs, nbytes = oracle_step(x, ring, sample_n, msgs, chunks)
    return {"value": round(nbytes / secs / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d elements of the same field (range, compress, decompress, "
                      "scatter pack of 8 segments), the ring Allreduce of 8 rank images of "
                      "512^2, the first %d of the "
                      "1000 messages, %d chunks of 64 KiB through the selector; single-threaded "
                      "plain C and numpy" % (sample_n, len(msgs), len(chunks)),
            "seconds": round(secs, 2),
            "parallel": cpu_parallel(x, msgs, x.size),
            "config1": oracle_config1()}


def run_reference(args):
    x, ring, msgs, chunks = cpu_fields(args.side)
    sample_n = min(1 << 22, x.size)
    ring = [r[:1 << 15] for r in ring]
    msgs = msgs[:4]
    chunks = chunks[:4]
    for _ in range(args.warmup):
        oracle_step(x, ring, sample_n, msgs, chunks)
    tot_s, tot_b = 0.0, 0
    for _ in range(args.steps):
        s, b = oracle_step(x, ring, sample_n, msgs, chunks)
        tot_s += s
        tot_b += b
    v = tot_b / tot_s / 1e9
    ms = tot_s / args.steps * 1e3
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded 512^3 Gaussian random field)",
            "config": {"workload": "grf512_rel1e-3_L32+stacking_ring8x8192sq+batch1000"
                                   "+selector_heldout",
                       "n": x.size, "rel_eb": REL, "block": BLOCK, "ring_ranks": P_RING,
                       "scatter_segments": P_RING, "batch_messages": 1000},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: first %d elements of the field, %d messages, "
                                       "%d selector chunks; single-threaded plain C and numpy"
                                       % (sample_n, len(msgs), len(chunks))},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args)))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.side)
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
