"""Benchmark of the codec hot path on one GB300 (replicas across GPUs).

Workload: the 512^3 FP32 Gaussian random field (P(k) ~ k^-3, scaled to
[-1, 1], 512 MiB), relative error bound 1e-3, block size 32.  One step runs
every hot-path kernel once over that field, each from its own inputs:

  range + compress   field -> stream (the bound resolved on the device)
  decompress         stream -> FP32 field
  ring step          8 chunks: decode received stream + add local chunk +
                     re-encode (one batched launch, the fixed ring bound)
  scatter pack       8 segments compressed as independent packed streams

``value`` is the algorithmic bytes of one step (every kernel's input read
plus output written, the extra input read of the relative bound included)
divided by the device time of the step (CUDA events on the launch stream),
summed over ranks.  Inputs (1 GiB) exceed the 129 MB L2, so no flush is
needed between steps.  ``e2e`` repeats the step through the same C ABI with
the inputs copied from pinned host memory and the compressed stream copied
back inside the timed region.

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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--chunks", type=int, default=0, help="2048-element chunks per CTA tile")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
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
        for ln in self.lines:
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


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2308_05199_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
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
        self.local = workloads.grf_3d(side=side, seed=2001, device=device)
        t = torch
        self.stream = t.cuda.current_stream()
        self.s = self.stream.cuda_stream
        self.ws = zc.Workspace(n, P_RING + 1)
        self.cap = zc.zc_max_compressed_bytes(n, BLOCK)
        self.cmp = t.empty(self.cap, dtype=t.uint8, device=device)
        self.cmp_n = t.zeros(1, dtype=t.int64, device=device)
        self.dec = t.empty(n, dtype=t.float32, device=device)
        # ring bound: fixed once from the field range (relative 1e-3)
        mm = t.zeros(2, dtype=t.float32, device=device)
        assert zc.zc_minmax(self.field.data_ptr(), n, 0, mm.data_ptr(), self.ws.ptr,
                            self.ws.nbytes, self.s) == 0
        lo, hi = mm.tolist()
        self.eb_abs = REL * (float(hi) - float(lo))
        # ring step inputs: the field's chunks compressed (the received streams)
        self.m = n // P_RING
        self.ccap = zc.zc_max_compressed_bytes(self.m, BLOCK)
        self.cin = t.empty(P_RING, self.ccap, dtype=t.uint8, device=device)
        self.cin_n = t.zeros(P_RING, dtype=t.int64, device=device)
        self.cout = t.empty(P_RING, self.ccap, dtype=t.uint8, device=device)
        self.cout_n = t.zeros(P_RING, dtype=t.int64, device=device)
        for r in range(P_RING):
            ch = self.field[r * self.m:(r + 1) * self.m]
            assert zc.zc_compress(ch.data_ptr(), self.m, 0, 0, self.eb_abs, BLOCK,
                                  self.cin[r].data_ptr(), self.ccap, self.cin_n[r].data_ptr(),
                                  self.ws.ptr, self.ws.nbytes, self.s) == 0
        items = (zc.ZcReduceItem * P_RING)()
        for r in range(P_RING):
            loc = self.local[r * self.m:(r + 1) * self.m]
            items[r] = zc.ZcReduceItem(self.cin[r].data_ptr(), loc.data_ptr(),
                                       self.cout[r].data_ptr(), None,
                                       self.cout_n[r].data_ptr(), self.m, self.ccap, self.ccap)
        self.plan = zc.ZcPlan()
        self.table = t.empty(zc.zc_plan_table_bytes(P_RING), dtype=t.uint8, device=device)
        assert zc.zc_plan_reduce(self.plan, P_RING, items, self.eb_abs, BLOCK,
                                 self.table.data_ptr(), self.table.numel()) == 0
        # scatter pack: 8 segments of the field
        self.counts = [self.m] * P_RING
        self.displs = [r * self.m for r in range(P_RING)]
        import ctypes
        self.hc = (ctypes.c_uint64 * P_RING)(*self.counts)
        self.hd = (ctypes.c_uint64 * P_RING)(*self.displs)
        self.pcap = P_RING * self.ccap
        self.packed = t.empty(self.pcap, dtype=t.uint8, device=device)
        self.seg = t.zeros(P_RING + 1, dtype=t.int64, device=device)
        # range, compress, width scan, decompress, width scan, ring step, scatter pack
        self.launches_per_step = 7

    def step(self, ev=None):
        zc, s, ws = self.zc, self.s, self.ws
        if ev:
            ev[0].record()
        assert zc.zc_compress(self.field.data_ptr(), self.n, 0, zc.EB_REL, REL, BLOCK,
                              self.cmp.data_ptr(), self.cap, self.cmp_n.data_ptr(), ws.ptr,
                              ws.nbytes, s) == 0
        if ev:
            ev[1].record()
        assert zc.zc_decompress(self.cmp.data_ptr(), self.cap, self.dec.data_ptr(), self.n, 0,
                                ws.ptr, ws.nbytes, s) == 0
        if ev:
            ev[2].record()
        assert zc.zc_reduce_step_batch(self.plan, ws.ptr, ws.nbytes, s) == 0
        if ev:
            ev[3].record()
        assert zc.zc_scatter_pack(self.field.data_ptr(), 0, P_RING, self.hc, self.hd, zc.EB_ABS,
                                  self.eb_abs, BLOCK, self.packed.data_ptr(), self.pcap,
                                  self.seg.data_ptr(), ws.ptr, ws.nbytes, s) == 0
        if ev:
            ev[4].record()

    def sizes(self):
        C = int(self.cmp_n.item())
        cin = int(self.cin_n.sum().item())
        cout = int(self.cout_n.sum().item())
        packed = int(self.seg[-1].item())
        n4 = 4 * self.n
        parts = {
            "compress": n4 + n4 + C,          # range read + compress read + stream write
            "decompress": C + n4,
            "ring_step": cin + n4 + cout,
            "scatter_pack": n4 + packed,
        }
        return C, parts


def run_ours(args, rank, world):
    import torch
    from paper_2308_05199_gb300 import build, workloads, zc

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if args.chunks:
        assert zc.zc_set_tile_chunks(args.chunks) == 0
    W = Workload(torch, zc, workloads, args.side, dev)
    args.warmup = max(args.warmup, 3)
    for _ in range(args.warmup):
        W.step()
    torch.cuda.synchronize()
    st, det = W.ws.status()
    if st != 0:
        raise RuntimeError("device status %d at %d during warm-up" % (st, det))
    C, parts = W.sizes()
    step_bytes = sum(parts.values())

    # timed region: K steps, per-kernel events on the launch stream
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for k in range(K):
            W.step(evs[k])
        t1.record()
        torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    st, det = W.ws.status()
    if st != 0:
        raise RuntimeError("device status %d at %d in the timed region" % (st, det))
    names = ["compress", "decompress", "ring_step", "scatter_pack"]
    per = {nm: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K))
           for i, nm in enumerate(names)}
    ms_per_step = total_ms / K
    value = step_bytes * world / (ms_per_step * 1e-3) / 1e9
    hbm, peak_kind = peaks()
    kern_gbs = {nm: parts[nm] / (per[nm] * 1e-3) / 1e9 for nm in names}
    dom = max(names, key=lambda nm: per[nm])
    traffic = load_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(kern_gbs[dom], 1),
                "peak": hbm, "unit": "GB/s", "frac": round(kern_gbs[dom] / hbm, 4),
                "peak_kind": peak_kind,
                "traffic": traffic["bytes_per_launch"] if traffic else None,
                "algorithmic_bytes": parts[dom]}
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded 512^3 Gaussian random field, P(k)~k^-3, in place of the "
                "paper's RTM volumes)",
        "config": {"workload": "grf512_rel1e-3_L32", "n": W.n, "rel_eb": REL,
                   "eb_abs_ring": W.eb_abs, "block": BLOCK, "ring_ranks": P_RING,
                   "scatter_segments": P_RING, "l2": "inputs larger than L2 (no flush)"},
        "ratio": round(4 * W.n / C, 3),
        "kernels_gbs": {k: round(v, 1) for k, v in kern_gbs.items()},
        "kernels_ms": {k: round(v, 4) for k, v in per.items()},
        "kernels_frac_of_hbm": {k: round(v / hbm, 4) for k, v in kern_gbs.items()},
        "roofline": roofline,
        "gpu_launches": W.launches_per_step * K,
        "clocks": clk.summary(),
    }
    if not args.no_e2e:
        out["e2e"] = e2e_ours(torch, W, args, step_bytes, world)
    return out


def e2e_ours(torch, W, args, step_bytes, world):
    """Same step with the two input fields copied in from pinned host memory
    and the compressed stream copied back, inside the timed region."""
    hf = W.field.cpu().pin_memory()
    hl = W.local.cpu().pin_memory()
    hout = torch.empty(W.cap, dtype=torch.uint8).pin_memory()
    hn = torch.zeros(1, dtype=torch.int64).pin_memory()
    K = max(3, args.steps // 2)
    C = int(W.cmp_n.item())

    def one():
        W.field.copy_(hf, non_blocking=True)
        W.local.copy_(hl, non_blocking=True)
        W.step()
        hn.copy_(W.cmp_n, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        c = int(hn.item())
        hout[:c].copy_(W.cmp[:c], non_blocking=True)

    for _ in range(2):
        one()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(K):
        one()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / K
    return {"value": round(step_bytes * world / dt / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": 8 * W.n, "d2h_bytes_per_step": C + 8,
            "ms_per_step": round(dt * 1e3, 3)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and --impl reference)

def oracle_step(x, loc, sample_n):
    """The bench step on the first sample_n elements, run by the CPU oracle;
    returns (seconds, algorithmic bytes).  The ring step's received streams
    are prepared outside the timed part (they are that step's input)."""
    import oracle
    xs, ls = x[:sample_n], loc[:sample_n]
    m = sample_n // P_RING
    t0 = time.perf_counter()
    mn, mx = oracle.minmax(xs)
    eb = oracle.eb_from_rel(REL, mn, mx)
    s = oracle.compress(xs, eb, 5)
    oracle.decompress(s, sample_n)
    t1 = time.perf_counter()
    cin = [oracle.compress(xs[r * m:(r + 1) * m], eb, 5) for r in range(P_RING)]
    t2 = time.perf_counter()
    cout = [oracle.reduce_step(cin[r], ls[r * m:(r + 1) * m], eb, 5)[0] for r in range(P_RING)]
    packed, _ = oracle.scatter_pack(xs, [m] * P_RING, [r * m for r in range(P_RING)], eb, 5)
    t3 = time.perf_counter()
    secs = (t1 - t0) + (t3 - t2)
    n4 = 4 * sample_n
    nbytes = (n4 + n4 + len(s)) + (len(s) + n4) + \
        (sum(map(len, cin)) + n4 + sum(map(len, cout))) + (n4 + len(packed))
    return secs, nbytes


def cpu_fields(side):
    import torch
    from paper_2308_05199_gb300 import workloads
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    x = workloads.grf_3d(side=side, seed=2000, device=dev).cpu().numpy()
    loc = workloads.grf_3d(side=side, seed=2001, device=dev).cpu().numpy()
    return x, loc


def cpu_baseline(side, sample_n=1 << 25):
    x, loc = cpu_fields(side)
    sample_n = min(sample_n, x.size)
    secs, nbytes = oracle_step(x, loc, sample_n)
    return {"value": round(nbytes / secs / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d elements of the same field (one step: range, compress, "
                      "decompress, ring step over 8 chunks, scatter pack of 8 segments), "
                      "single-threaded plain C" % sample_n,
            "seconds": round(secs, 2)}


def run_reference(args):
    x, loc = cpu_fields(args.side)
    sample_n = min(1 << 22, x.size)
    for _ in range(args.warmup):
        oracle_step(x, loc, sample_n)
    tot_s, tot_b = 0.0, 0
    for _ in range(args.steps):
        s, b = oracle_step(x, loc, sample_n)
        tot_s += s
        tot_b += b
    v = tot_b / tot_s / 1e9
    ms = tot_s / args.steps * 1e3
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded 512^3 Gaussian random field)",
            "config": {"workload": "grf512_rel1e-3_L32", "n": x.size, "rel_eb": REL,
                       "block": BLOCK, "ring_ranks": P_RING, "scatter_segments": P_RING},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "first %d elements per step, single-threaded plain C"
                                       % sample_n},
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
