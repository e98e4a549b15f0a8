#!/usr/bin/env python
"""Benchmark of the semiring product/closure hot path on GB300.

Default workload (one "step" = the whole hot path over one batch):
  anti-distance closure D=4096 u8 (edge p=0.05, length U{1..31}, seed 1) plus
  the product antidist_mul 4096x4096x4096 u8 (A = that graph, B = stream 3):
  encode A -> T, encode A, encode B, closure(T) in place, C = A ⊗ B.
  Metric: semiring ops per second, counting D^3 for the closure and R·K·N for
  the product (2·4096^3 per step), in Gop/s.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
        [--workload cfg2|cfg2-8192|u16|u32|cfg1|cfg3|prod16k|cfg4|cfg4-200|cfg5] [--no-cpu] [--no-e2e]
Under torchrun each rank runs an independent replica on its own GPU (the
closure does not shard without an exchange step; replicas only) and rank 0
prints one JSON line with the max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "closure/product semiring Gop/s (D³/s) vs int-pipe peak; batched p50/p99 ms"
UNIT = "Gop/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg2")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end pass")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-8192", action="store_true", help="default workload: skip the D=8192 closure timing")
    ap.add_argument("--no-batched", action="store_true", help="default workload: skip the batched (config 4) summary")
    ap.add_argument("--no-bool", action="store_true",
                    help="default workload: skip the Boolean closure (config 3, D=16384) summary")
    ap.add_argument("--closure", default="auto", choices=["auto", "persistent", "fused", "stream"],
                    help="anti-distance closure schedule (auto: the library's choice with the workspace it asks for)")
    ap.add_argument("--tuning", default="", help="batched workloads: cluster,threshold,ctas_per_sm (skips autotune)")
    ap.add_argument("--only", default="", choices=["", "mul", "closure"],
                    help="profiling aid: run only one part of the step (not a bench line)")
    return ap.parse_args()


# --------------------------------------------------------------------------- ranks
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling (200 ms) during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- workloads
CLOSURE_TUNED = {}


def closure_ctx(D, sdt, mode="auto"):
    """A context for the anti-distance closure: its workspace holds what the persistent and
    fused-pass schedules need (sr_workspace_query).  mode "auto": the library's autotuner
    times every schedule at this size (stream blocks of 128/256/512, persistent, fused
    passes) before any timed step and the closure follows its choice; "persistent" /
    "fused" / "stream" force one."""
    import paper_1705_08743_gb300 as sr
    ws = sr.sr_workspace_query(sr.SR_OP_ANTIDIST_CLOSURE, sdt, D) if sdt in (sr.SR_U8, sr.SR_U16) else 0
    ctx = sr.sr_create(workspace_bytes=ws)
    sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_PERSISTENT, {"auto": 1, "persistent": 2, "fused": 0, "stream": 0}[mode])
    sr.sr_set_option(ctx, sr.SR_OPT_CLOSURE_FUSED, {"auto": 1, "persistent": 0, "fused": 2, "stream": 0}[mode])
    if mode == "auto":
        choice, ms = sr.sr_autotune_closure(ctx, sdt, D, reps=2)
        name = {sr.SR_TUNE_PERSISTENT: "persistent", sr.SR_TUNE_FUSED: "fused passes (one launch per pivot block)"}
        CLOSURE_TUNED[D] = {"choice": name.get(choice, f"stream, {choice}-wide blocks"),
                            "best_ms_at_bucket": ms, "bucket": D}
    return ctx


def bench_config(wl, world):
    """The JSON line's `config`: the same dict in both arms (ours and the reference)."""
    c = {"workload": wl.name, "ops_per_step": wl.ops,
         "l2": f"flushed before each step ({L2_FLUSH_BYTES >> 20} MiB write)",
         "parallelism": "replicas" if world > 1 else "single GPU"}
    c.update(getattr(wl, "config_extra", {}))
    return c


def measured_bf16_tflops():
    """Dense bf16 burst throughput measured on the GB300s (MEASURED_PEAKS.json),
    else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def sha_of(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


FUSED_SOURCES = ["paper_1705_08743_gb300/csrc/closure_fused.cu", "paper_1705_08743_gb300/csrc/antidist_tile.cuh",
                 "paper_1705_08743_gb300/csrc/diag128.cuh", "paper_1705_08743_gb300/csrc/sr_common.cuh"]


def load_traffic(kernel_key: str, sources, workload: str):
    """DRAM bytes per launch from a committed ncu capture of this workload's launch, if the
    kernel is unchanged since (traffic does not scale with the op count, so a capture at
    another size does not stand in for this one)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(f"{kernel_key} @ {workload}")
    if not e or e.get("source_sha") != sha_of(sources):
        return None
    return e.get("dram_bytes_per_launch")


class Cfg2:
    """Anti-distance closure + product, D x D u8 (or u16, u32)."""

    def __init__(self, D=4096, dtype="u8"):
        self.D, self.dtype = D, dtype
        self.name = (f"antidist_closure D={D} {dtype} + antidist_mul {D}x{D}x{D} {dtype} "
                     f"(edge p=0.05, length U{{1..31}}, seed 1; B: stream 3)")
        self.ops = 2 * D ** 3
        self.config_extra = {"step": "encode x3 + closure (in place) + product"}

    def host_inputs(self):
        import numpy as np
        import synth
        npdt = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32}[self.dtype]
        WA = synth.cfg2_antidist(D=self.D, seed=1, s_edge=0, dtype=npdt)
        WB = synth.cfg2_antidist(D=self.D, seed=1, s_edge=3, dtype=npdt)
        return WA, WB

    def setup_device(self, WA, WB, dev):
        import torch
        import paper_1705_08743_gb300 as sr
        tdt = {"u8": torch.uint8, "u16": torch.int16, "u32": torch.int32}[self.dtype]
        self.sdt = {"u8": sr.SR_U8, "u16": sr.SR_U16, "u32": sr.SR_U32}[self.dtype]
        view = self._view
        self.WA = torch.from_numpy(view(WA)).to(dev)
        self.WB = torch.from_numpy(view(WB)).to(dev)
        D = self.D
        self.T = torch.empty((D, D), dtype=tdt, device=dev)
        self.A = torch.empty_like(self.T)
        self.B = torch.empty_like(self.T)
        self.C = torch.empty_like(self.T)
        self.mul_events = []
        self.closure_events = []
        self.ctx = closure_ctx(D, self.sdt, self.closure_mode)
        sr.antidist_encode(None, self.WA, D, self.A, D, D, D, self.sdt)
        sr.antidist_encode(None, self.WB, D, self.B, D, D, D, self.sdt)

    only = ""
    closure_mode = "auto"

    def step(self, stream, record_mul=False):
        import torch
        import paper_1705_08743_gb300 as sr
        D, s = self.D, stream.cuda_stream
        if self.only == "mul":
            sr.antidist_mul(None, self.A, D, self.B, D, self.C, D, D, D, D, self.sdt, 0, s)
            return
        if self.only == "closure":
            sr.antidist_encode(None, self.WA, D, self.T, D, D, D, self.sdt, s)
            sr.antidist_closure(self.ctx, self.T, D, D, self.sdt, s)
            return
        sr.antidist_encode(None, self.WA, D, self.T, D, D, D, self.sdt, s)
        sr.antidist_encode(None, self.WA, D, self.A, D, D, D, self.sdt, s)
        sr.antidist_encode(None, self.WB, D, self.B, D, D, D, self.sdt, s)
        if record_mul:
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
        sr.antidist_closure(self.ctx, self.T, D, D, self.sdt, s)
        if record_mul:
            c1.record(stream)
            self.closure_events.append((c0, c1))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        sr.antidist_mul(None, self.A, D, self.B, D, self.C, D, D, D, D, self.sdt, 0, s)
        if record_mul:
            e1.record(stream)
            self.mul_events.append((e0, e1))

    # host-buffer path: H2D of both weight matrices, the step, D2H of T and C
    def e2e_setup(self, WA, WB):
        import torch
        view = self._view
        self.hWA = torch.from_numpy(view(WA)).pin_memory()
        self.hWB = torch.from_numpy(view(WB)).pin_memory()
        self.hT = torch.empty(self.hWA.shape, dtype=self.hWA.dtype).pin_memory()
        self.hC = torch.empty_like(self.hT).pin_memory()
        self.h2d = 2 * self.hWA.numel() * self.hWA.element_size()
        self.d2h = 2 * self.hT.numel() * self.hT.element_size()
        import paper_1705_08743_gb300 as sr
        # kernels read the inputs and write C in pinned host memory where the device maps it
        self.zero_copy = all(sr.sr_host_mapped(t) for t in (self.hWA, self.hWB, self.hC))
        self.transfer = ("zero-copy: the encodes read WA and WB and the product writes C in pinned host memory "
                         "over the host link; T copied back on a copy stream during the product"
                         if self.zero_copy else
                         "copies: WA uploaded before the closure, WB on a copy stream beside it, T downloaded "
                         "during the product, C after it")

    def e2e_step(self, stream):
        """Host buffers in and out, transfers overlapped with compute the way a user of the
        library would.  Zero-copy where pinned host memory is mapped into the device address
        space (sr_host_mapped): WA's encode reads host memory, WB's encode does so on a copy
        stream beside the closure, the product writes C into host memory, T's download runs
        beside the product.  Otherwise copies: WB's upload and T's download run on a copy
        stream while the closure and the product compute on `stream`."""
        import torch
        import paper_1705_08743_gb300 as sr
        D, s = self.D, stream.cuda_stream
        if self.zero_copy:
            if not hasattr(self, "copy_stream"):
                self.copy_stream = torch.cuda.Stream(device=stream.device)
                self.ev = [torch.cuda.Event() for _ in range(4)]
            cs = self.copy_stream
            self.ev[0].record(stream)                      # step start: buffers free
            cs.wait_event(self.ev[0])
            sr.antidist_encode(None, self.hWA, D, self.T, D, D, D, self.sdt, s)   # reads host memory
            self.A.copy_(self.T)                           # the product's A: the encoded input
            with torch.cuda.stream(cs):
                sr.antidist_encode(None, self.hWB, D, self.B, D, D, D, self.sdt, cs.cuda_stream)
                self.ev[1].record(cs)
            sr.antidist_closure(self.ctx, self.T, D, D, self.sdt, s)
            self.ev[2].record(stream)                      # T final
            with torch.cuda.stream(cs):
                cs.wait_event(self.ev[2])
                self.hT.copy_(self.T, non_blocking=True)
                self.ev[3].record(cs)
            stream.wait_event(self.ev[1])
            sr.antidist_mul(None, self.A, D, self.B, D, self.hC, D, D, D, D, self.sdt, 0, s)   # writes host memory
            stream.wait_event(self.ev[3])                  # the step ends when both results are home
            return
        if not hasattr(self, "copy_stream"):
            self.copy_stream = torch.cuda.Stream(device=stream.device)
            self.ev = [torch.cuda.Event() for _ in range(4)]
        cs = self.copy_stream
        self.ev[0].record(stream)                          # step start: buffers free
        cs.wait_event(self.ev[0])
        self.WA.copy_(self.hWA, non_blocking=True)         # on `stream`
        with torch.cuda.stream(cs):
            self.WB.copy_(self.hWB, non_blocking=True)
            self.ev[1].record(cs)
        sr.antidist_encode(None, self.WA, D, self.T, D, D, D, self.sdt, s)
        sr.antidist_encode(None, self.WA, D, self.A, D, D, D, self.sdt, s)
        sr.antidist_closure(self.ctx, self.T, D, D, self.sdt, s)
        self.ev[2].record(stream)                          # T final
        with torch.cuda.stream(cs):
            cs.wait_event(self.ev[2])
            self.hT.copy_(self.T, non_blocking=True)
            self.ev[3].record(cs)
        stream.wait_event(self.ev[1])
        sr.antidist_encode(None, self.WB, D, self.B, D, D, D, self.sdt, s)
        sr.antidist_mul(None, self.A, D, self.B, D, self.C, D, D, D, D, self.sdt, 0, s)
        self.hC.copy_(self.C, non_blocking=True)
        stream.wait_event(self.ev[3])                      # the step ends when both results are home

    def _view(self, a):
        """numpy array -> a view torch can hold (16- and 32-bit entries as signed bit patterns)."""
        return {"u8": a, "u16": a.view("int16"), "u32": a.view("int32")}[self.dtype]

    # roofline of the dominant kernel: the product kernel (also the closure's phase 3)
    @property
    def roofline_kernel(self):
        return {"u8": "antidist_mul_kernel<KindU8,128,128,32,8,16>",
                "u16": "antidist_mul_kernel<KindU16,128,128,32,8,16>",
                "u32": "antidist32_mul_kernel<128,64,8,8,8>"}[self.dtype]

    @property
    def roofline_sources(self):
        if self.dtype == "u32":
            return ["paper_1705_08743_gb300/csrc/antidist32.cu", "paper_1705_08743_gb300/csrc/sr_common.cuh"]
        return ["paper_1705_08743_gb300/csrc/antidist.cu", "paper_1705_08743_gb300/csrc/antidist_tile.cuh",
                "paper_1705_08743_gb300/csrc/sr_common.cuh"]

    def cpu_sample(self, WA, WB):
        """Oracle on a bounded sample: full closure at this D, product on the first rows."""
        import numpy as np
        import oracle
        S = {"u8": 255, "u16": 65535, "u32": 2 ** 32 - 1}[self.dtype]
        D = self.D
        rows = max(1, D // 4)
        t0 = time.perf_counter()
        A = oracle.encode_antidist(WA, S)
        B = oracle.encode_antidist(WB, S)
        oracle.warshall(A, S)
        oracle.mul(A[:rows], B, S)
        dt = time.perf_counter() - t0
        ops = D ** 3 + rows * D * D
        return {"ops": ops, "seconds": dt,
                "sample": f"oracle encode + Warshall closure D={D} + product rows 0..{rows - 1} of {D}^3 "
                          f"({ops / 1e9:.1f} Gop)"}


class Cfg4:
    """Batched anti-distance closure: n graphs, D log-uniform [32, 1024], u16, one
    persistent launch per step (captured in a CUDA graph, tuned once by the library's
    autotuner before timing).  The graphs live in one pool; each step restores the pool
    from a pristine device copy outside the timed events (the closure is in place)."""

    dtype = "u16"
    only = ""
    tuning = (2, 384, 2)

    # the dominant kernels follow the schedule the autotuner picked (cluster 0: grouped)
    @property
    def roofline_kernel(self):
        if self.tuning[0] == 0:
            return "grouped schedule: antidist_mul_grouped_kernel<KindU16> + antidist_pivot_grouped_kernel<KindU16,128>"
        return "batched_closure_kernel<KindU16,64,NC>"

    @property
    def roofline_sources(self):
        src = ["paper_1705_08743_gb300/csrc/batched.cu", "paper_1705_08743_gb300/csrc/sr_common.cuh"]
        if self.tuning[0] == 0:
            src += ["paper_1705_08743_gb300/csrc/antidist.cu", "paper_1705_08743_gb300/csrc/antidist_tile.cuh"]
        return src

    fixed_tuning = None

    def __init__(self, n=2000):
        self.n = n
        self.name = (f"batched antidist_closure: {n} graphs, D log-uniform [32,1024], u16, "
                     f"length U{{1..4000}}, p=8/D, seed 3; one persistent launch")
        self.config_extra = {"pool": "restored from a device copy before each step, outside the events"}

    def host_inputs(self):
        import numpy as np
        import synth
        sizes, W = synth.cfg4_batched(n=self.n)
        self.sizes = sizes
        self.ops = float(sum(D ** 3 for D in sizes))
        self.alg_bytes = float(sum(4 * D * D for D in sizes))      # read + write every u16 entry once
        # rows padded to 8 entries (16 bytes) so every graph takes the vector path
        self.lds = [D + (-D) % 8 for D in sizes]
        parts = []
        for w, D, ld in zip(W, sizes, self.lds):
            p = np.zeros((D, ld), np.uint16)
            p[:, :D] = w
            parts.append(p.reshape(-1))
        pool = np.concatenate(parts)
        return pool, None

    def setup_device(self, pool, _unused, dev):
        import torch
        import paper_1705_08743_gb300 as sr
        self.sr = sr
        self.Wpool = torch.from_numpy(pool.view("int16")).to(dev)
        self.T0 = torch.empty_like(self.Wpool)
        n = self.Wpool.numel()
        sr.antidist_encode(None, self.Wpool, n, self.T0, n, 1, n, sr.SR_U16)
        self.T = self.T0.clone()
        self.descs, off = [], 0
        for D, ld in zip(self.sizes, self.lds):
            self.descs.append(sr.closure_desc(self.T.data_ptr() + 2 * off, ld, D, sr.SR_U16))
            off += D * ld
        self.ctx = sr.sr_create()
        self.batch = sr.sr_batch_create(self.ctx, self.descs)
        if self.fixed_tuning:
            sr.sr_batch_set_tuning(self.batch, *self.fixed_tuning)
        else:
            sr.sr_batch_autotune(self.ctx, self.batch, reps=1)
        self.tuning = sr.sr_batch_get_tuning(self.batch)
        self.mul_events = []

    def pre_step(self, stream):
        self.T.copy_(self.T0, non_blocking=True)              # restore, outside the events

    def step(self, stream, record_mul=False):
        import torch
        if record_mul:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        self.sr.sr_batch_launch(self.batch, 1, stream.cuda_stream)
        if record_mul:
            e1.record(stream)
            self.mul_events.append((e0, e1))

    def completion_ms(self, stream, flush, launches=5):
        """Per-graph completion times inside one batch launch (device clock stamps at each
        graph's end, sr_batch_set_timing), over `launches` launches on restored inputs
        with the L2 flushed before each: every graph of every launch is one sample."""
        import torch
        sr = self.sr
        sr.sr_batch_set_timing(self.batch, True)
        samples = []
        try:
            for _ in range(launches):
                with torch.cuda.stream(stream):
                    self.pre_step(stream)
                    flush.zero_()
                    sr.sr_batch_launch(self.batch, 1, stream.cuda_stream)
                torch.cuda.synchronize()
                samples += sr.sr_batch_completion_ms(self.batch)
        finally:
            sr.sr_batch_set_timing(self.batch, False)
        return samples

    def loop_of_single_calls_ms(self, stream, reps=2):
        import torch
        sr = self.sr
        ts = []
        for r in range(reps + 1):
            self.T.copy_(self.T0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for d in self.descs:
                sr.antidist_closure(None, d.C, d.ldc, d.R, sr.SR_U16, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        return min(ts)

    def e2e_setup(self, pool, _unused):
        import torch
        self.hW = torch.from_numpy(pool.view("int16")).pin_memory()
        self.hT = torch.empty_like(self.hW).pin_memory()
        self.h2d = self.hW.numel() * 2
        self.d2h = self.hT.numel() * 2

    def e2e_step(self, stream):
        sr = self.sr
        n = self.Wpool.numel()
        self.Wpool.copy_(self.hW, non_blocking=True)
        sr.antidist_encode(None, self.Wpool, n, self.T, n, 1, n, sr.SR_U16, stream.cuda_stream)
        sr.sr_batch_launch(self.batch, 1, stream.cuda_stream)
        self.hT.copy_(self.T, non_blocking=True)

    def cpu_sample(self, pool, _unused):
        """Oracle Warshall on a prefix of the graph list worth ~6 % of the batch's ops."""
        import numpy as np
        import oracle
        t0 = time.perf_counter()
        off, ops, k = 0, 0.0, 0
        for D, ld in zip(self.sizes, self.lds):
            W = pool[off:off + D * ld].reshape(D, ld)[:, :D]
            off += D * ld
            oracle.warshall(oracle.encode_antidist(W, 65535), 65535)
            ops += D ** 3
            k += 1
            if ops >= 0.06 * self.ops:
                break
        dt = time.perf_counter() - t0
        return {"ops": ops, "seconds": dt,
                "sample": f"oracle encode + Warshall on the first {k} graphs ({ops / 1e9:.1f} Gop)"}


class Cfg5:
    """Served request stream: Poisson arrivals at swept rates; each request uniformly
    one of {Bool closure, Bool product, u8 closure, u8 product, u16 closure, u16
    product}, D log-uniform in [64, 8192], inputs drawn per request from seeds as in
    configurations 2-4 (a pool of distinct requests, cycled).  The served form (the
    library's loop: admission by device memory, 4 stream slots, small closures
    batched) is compared with serial single calls (one request at a time, direct
    C-ABI calls) on the same arrival sequence."""

    dtype = "mixed"
    only = ""
    KINDS = ["bool_closure", "bool_mul", "u8_closure", "u8_mul", "u16_closure", "u16_mul"]

    def __init__(self, pool=36, per_rate=1000, fracs=(0.2, 0.4, 0.6, 0.8, 1.0, 1.2, 1.4), dmax=8192):
        self.pool, self.per_rate, self.fracs, self.dmax = pool, per_rate, fracs, dmax
        self.name = (f"served stream: Poisson arrivals, rates {list(fracs)} x capacity, {per_rate} requests per "
                     f"rate from a pool of {pool}; kinds uniform over {self.KINDS}; D log-uniform [64,{dmax}]")

    def host_inputs(self):
        import numpy as np
        import synth
        sizes = synth.log_uniform_sizes(self.pool, 64, self.dmax, seed=5, s=2)
        reqs = []
        for i, D in enumerate(sizes):
            kind = self.KINDS[synth.h_int(5, 9, i, 0) % 6]
            seed = synth.graph_seed(5, i)
            if kind.startswith("bool"):
                A = synth.bool_dag_union(D, seed)
                B = synth.bool_dag_union(D, seed + 1) if kind.endswith("mul") else None
            elif kind.startswith("u8"):
                A = synth.cfg2_antidist(D, seed=seed, s_edge=0)
                B = synth.cfg2_antidist(D, seed=seed, s_edge=3) if kind.endswith("mul") else None
            else:
                A = synth.weighted_graph(D, D, min(1.0, 8.0 / D), 1, 4000, seed, 0, dtype=np.uint16)
                B = synth.weighted_graph(D, D, min(1.0, 8.0 / D), 1, 4000, seed, 3, dtype=np.uint16) \
                    if kind.endswith("mul") else None
            reqs.append((kind, D, A, B))
        self.ops_of = [float(D) ** 3 for _, D, _, _ in reqs]
        return reqs, None

    def setup_device(self, reqs, _unused, dev):
        """Encode / pack every pooled input on the GPU (library kernels), keep pinned host copies."""
        import torch
        import paper_1705_08743_gb300 as sr
        self.sr = sr
        self.items = []
        for kind, D, A, B in reqs:
            mats = []
            for X in (A, B):
                if X is None:
                    mats.append(None)
                    continue
                if kind.startswith("bool"):
                    nw = (D + 63) // 64
                    Xd = torch.from_numpy(X).to(dev)
                    P = torch.empty((D, nw), dtype=torch.int64, device=dev)
                    sr.bool_pack(None, Xd, D, P, nw, D, D, sr.SR_BOOL_W64)
                    mats.append(P.cpu().pin_memory())
                else:
                    u8 = kind.startswith("u8")
                    Xd = torch.from_numpy(X if u8 else X.view("int16")).to(dev)
                    E = torch.empty_like(Xd)
                    sr.antidist_encode(None, Xd, D, E, D, D, D, sr.SR_U8 if u8 else sr.SR_U16)
                    mats.append(E.cpu().pin_memory())
            out = torch.empty_like(mats[0]).pin_memory()
            dt = {"bool": sr.SR_BOOL_W64, "u8": sr.SR_U8, "u16": sr.SR_U16}[kind.split("_")[0]]
            op = {("bool", "closure"): sr.SR_OP_BOOL_CLOSURE, ("bool", "mul"): sr.SR_OP_BOOL_MUL,
                  ("u8", "closure"): sr.SR_OP_ANTIDIST_CLOSURE, ("u8", "mul"): sr.SR_OP_ANTIDIST_MUL,
                  ("u16", "closure"): sr.SR_OP_ANTIDIST_CLOSURE, ("u16", "mul"): sr.SR_OP_ANTIDIST_MUL}[
                tuple(kind.split("_"))]
            self.items.append(dict(kind=kind, D=D, op=op, dtype=dt, A=mats[0], B=mats[1], out=out))
        torch.cuda.synchronize()

    # one request through the direct C-ABI calls on `stream` (serial baseline)
    def run_single(self, it, stream, bufs):
        import torch
        sr = self.sr
        D, s = it["D"], stream.cuda_stream
        A = bufs.setdefault(("A", id(it)), torch.empty(it["A"].shape, dtype=it["A"].dtype, device="cuda"))
        A.copy_(it["A"], non_blocking=True)
        if it["op"] in (sr.SR_OP_ANTIDIST_CLOSURE, sr.SR_OP_BOOL_CLOSURE):
            if it["op"] == sr.SR_OP_ANTIDIST_CLOSURE:
                sr.antidist_closure(None, A, A.shape[1], D, it["dtype"], s)
            else:
                sr.bool_closure(None, A, A.shape[1], D, it["dtype"], sr.SR_CLOSURE_WARSHALL, s)
            it["out"].copy_(A, non_blocking=True)
        else:
            B = bufs.setdefault(("B", id(it)), torch.empty(it["B"].shape, dtype=it["B"].dtype, device="cuda"))
            B.copy_(it["B"], non_blocking=True)
            C = bufs.setdefault(("C", id(it)), torch.empty_like(A))
            fn = sr.antidist_mul if it["op"] == sr.SR_OP_ANTIDIST_MUL else sr.bool_mul
            fn(None, A, A.shape[1], B, B.shape[1], C, C.shape[1], D, D, D, it["dtype"], 0, s)
            it["out"].copy_(C, non_blocking=True)
        stream.synchronize()

    def arrivals(self, rate, n, seed):
        import numpy as np
        rng = np.random.default_rng(seed)
        return np.cumsum(rng.exponential(1.0 / rate, size=n)), rng.integers(0, len(self.items), size=n)

    def serve_run(self, rate, n, seed):
        sr = self.sr
        times, which = self.arrivals(rate, n, seed)
        ctx = sr.sr_create()
        sr.sr_serve_start(ctx, arena_bytes=8 << 30, slots=4, batch_max_d=512, batch_max_graphs=64, backfill_ms=50)
        t0 = time.perf_counter()
        tickets = []
        for t_arr, w in zip(times, which):
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            it = self.items[w]
            r = sr.make_request(it["op"], it["dtype"], it["D"], it["D"], it["D"], A=it["A"], B=it["B"], out=it["out"])
            tickets.append(sr.sr_submit(ctx, r))
        lat = []
        for t in tickets:
            sr.sr_wait(ctx, t, 600000)
            lat.append(sr.sr_result(ctx, t).latency_ms)
        makespan = time.perf_counter() - t0
        stats = sr.sr_serve_stats(ctx)
        sr.sr_destroy(ctx)
        ops = sum(self.ops_of[w] for w in which)
        return lat, ops / makespan / 1e9, stats

    def serial_run(self, rate, n, seed, stream):
        times, which = self.arrivals(rate, n, seed)
        bufs = {}
        t0 = time.perf_counter()
        lat = []
        for t_arr, w in zip(times, which):
            now = time.perf_counter() - t0
            if now < t_arr:
                time.sleep(t_arr - now)
            self.run_single(self.items[w], stream, bufs)
            lat.append((time.perf_counter() - t0 - t_arr) * 1e3)
        makespan = time.perf_counter() - t0
        ops = sum(self.ops_of[w] for w in which)
        return lat, ops / makespan / 1e9

    def cpu_sample(self, reqs, _unused):
        return {"ops": 0, "seconds": 1.0, "sample": "not measured for the served stream"}


class CfgBool:
    """Boolean workloads.  cfg1: product 512x512x512, Bernoulli(0.02), 32 columns per
    word (latency-bound; reported in us).  cfg3: transitive closure D=16384, 64-bit
    words, DAG (i<j, p=2/D) union random digraph (mean out-degree 1.5), seed 2; the
    step packs the dense 0/1 input and closes it by blocked Warshall; the squaring
    form (A ⊗ (I ⊕ A)^(2^14), 15 products of 16384^3 on the tensor cores) is timed
    beside it.  prod16k: the product A ⊗ A of the config-3 graph (16384^3, 32 columns
    per word) off the tensor cores, where the library picks the Four Russians table
    kernel; the masked-OR and tensor-core forms are timed beside it."""

    only = ""

    def __init__(self, kind):
        self.kind = kind
        self.dtype = "bits"
        if kind == "cfg1":
            self.D, self.name = 512, "bool_mul 512x512x512, Bernoulli(0.02), seed 0, 32 columns per uint32"
        elif kind == "prod16k":
            self.D, self.name = 16384, ("bool_mul A x A, A = the D=16384 config-3 graph (DAG p=2/D union p=1.5/D, "
                                        "seed 2), 32 columns per uint32, word path (Four Russians)")
        else:
            self.D, self.name = 16384, ("bool_closure D=16384 bit-packed uint64: DAG (i<j, p=2/D) union random "
                                        "digraph (p=1.5/D), seed 2; pack + blocked Warshall (2048-bit blocks, "
                                        "panels and phase 3 on the tensor cores)")
        self.ops = float(self.D) ** 3

    def host_inputs(self):
        import synth
        if self.kind == "cfg1":
            return synth.cfg1_bool_product()
        return synth.cfg3_bool_closure(self.D), None

    def setup_device(self, A, B, dev):
        import torch
        import paper_1705_08743_gb300 as sr
        self.sr = sr
        D = self.D
        self.w = 64 if self.kind == "cfg3" else 32
        self.dt = sr.SR_BOOL_W32 if self.w == 32 else sr.SR_BOOL_W64
        tdt = torch.int32 if self.w == 32 else torch.int64
        self.nw = D // self.w
        self.dense = torch.from_numpy(A).to(dev)
        self.T = torch.zeros((D, self.nw), dtype=tdt, device=dev)
        if self.kind == "cfg1":
            self.denseB = torch.from_numpy(B).to(dev)
            self.A = torch.zeros_like(self.T)
            self.B = torch.zeros_like(self.T)
            sr.bool_pack(None, self.dense, D, self.A, self.nw, D, D, self.dt)
            sr.bool_pack(None, self.denseB, D, self.B, self.nw, D, D, self.dt)
            self.ctx = None
        elif self.kind == "prod16k":
            self.A = torch.zeros_like(self.T)
            sr.bool_pack(None, self.dense, D, self.A, self.nw, D, D, self.dt)
            self.B = self.A
            self.ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_MUL, self.dt, D))
            sr.sr_set_option(self.ctx, sr.SR_OPT_BOOL_TENSOR, 0)      # word path: auto picks the tables
        else:
            self.ctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, self.dt, D,
                                                                          sr.SR_CLOSURE_SQUARING))
            self.wctx = sr.sr_create(workspace_bytes=sr.sr_workspace_query(sr.SR_OP_BOOL_CLOSURE, self.dt, D,
                                                                           sr.SR_CLOSURE_WARSHALL))
        self.mul_events = []

    def step(self, stream, record_mul=False, dense=None):
        """dense: where config 3 packs its input from (default: the device copy)."""
        import torch
        sr, D, s = self.sr, self.D, stream.cuda_stream
        if record_mul:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        if self.kind == "cfg1":
            sr.bool_mul(None, self.A, self.nw, self.B, self.nw, self.T, self.nw, D, D, D, self.dt, 0, s)
        elif self.kind == "prod16k":
            sr.bool_mul(self.ctx, self.A, self.nw, self.B, self.nw, self.T, self.nw, D, D, D, self.dt, 0, s)
        else:
            sr.bool_pack(None, self.dense if dense is None else dense, D, self.T, self.nw, D, D, self.dt, s)
            sr.bool_closure(self.wctx, self.T, self.nw, D, self.dt, sr.SR_CLOSURE_WARSHALL, s)
        if record_mul:
            e1.record(stream)
            self.mul_events.append((e0, e1))

    def other_forms_ms(self, stream, reps=2):
        """The same closure by the squaring form and by the 128-bit word schedule (no
        workspace); bits identical to the step's."""
        import torch
        sr, D, s = self.sr, self.D, stream.cuda_stream
        ref = self.T.clone()
        out = {}
        for name, ctx, method in [("squaring", self.ctx, sr.SR_CLOSURE_SQUARING),
                                  ("warshall_128bit_words", None, sr.SR_CLOSURE_WARSHALL)]:
            ts = []
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sr.bool_pack(None, self.dense, D, self.T, self.nw, D, D, self.dt, s)
                sr.bool_closure(ctx, self.T, self.nw, D, self.dt, method, s)
                e1.record(stream)
                torch.cuda.synchronize()
                if r:
                    ts.append(e0.elapsed_time(e1))
            out[name + "_ms"] = min(ts)
            out[name + "_identical"] = bool(torch.equal(self.T, ref))
        return out

    def forms_ms(self, stream, reps=3):
        """The same product by each Boolean product kernel: masked OR, Four Russians,
        tensor cores (count, then test); bits identical to the step's."""
        import torch
        sr, D, s = self.sr, self.D, stream.cuda_stream
        ref = self.T.clone()
        out = {}
        for name, tc, m4r in [("masked_or", 0, 0), ("four_russians", 0, 2), ("tensor", 2, 0)]:
            sr.sr_set_option(self.ctx, sr.SR_OPT_BOOL_TENSOR, tc)
            sr.sr_set_option(self.ctx, sr.SR_OPT_BOOL_FOUR_RUSSIANS, m4r)
            ts = []
            for r in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sr.bool_mul(self.ctx, self.A, self.nw, self.B, self.nw, self.T, self.nw, D, D, D, self.dt, 0, s)
                e1.record(stream)
                torch.cuda.synchronize()
                if r:
                    ts.append(e0.elapsed_time(e1))
            out[name] = min(ts)
            out[name + "_identical"] = bool(torch.equal(self.T, ref))
        sr.sr_set_option(self.ctx, sr.SR_OPT_BOOL_TENSOR, 0)
        sr.sr_set_option(self.ctx, sr.SR_OPT_BOOL_FOUR_RUSSIANS, 1)
        return out

    def e2e_setup(self, A, B):
        import torch
        self.hA = torch.from_numpy(A).pin_memory()
        self.hT = torch.empty(tuple(self.T.shape), dtype=self.T.dtype).pin_memory()
        self.h2d = self.hA.numel()
        self.d2h = self.hT.numel() * self.hT.element_size()
        if self.kind == "cfg1":
            self.hB = torch.from_numpy(B).pin_memory()
            self.h2d *= 2
        # the pack kernels read the dense 0/1 input in pinned host memory where the device maps it
        sr = self.sr
        self.zero_copy = sr.sr_host_mapped(self.hA) and (self.kind != "cfg1" or sr.sr_host_mapped(self.hB))
        self.transfer = ("zero-copy: the pack kernels read the dense input in pinned host memory over the host "
                         "link; the result copied back" if self.zero_copy else
                         "copies: the dense input uploaded, the result copied back")

    def e2e_step(self, stream):
        sr, D, s = self.sr, self.D, stream.cuda_stream
        if self.zero_copy:
            src_a, src_b = self.hA, getattr(self, "hB", None)
        else:
            self.dense.copy_(self.hA, non_blocking=True)
            src_a = self.dense
            if self.kind == "cfg1":
                self.denseB.copy_(self.hB, non_blocking=True)
                src_b = self.denseB
        if self.kind == "cfg1":
            sr.bool_pack(None, src_a, D, self.A, self.nw, D, D, self.dt, s)
            sr.bool_pack(None, src_b, D, self.B, self.nw, D, D, self.dt, s)
        elif self.kind == "prod16k":
            sr.bool_pack(None, src_a, D, self.A, self.nw, D, D, self.dt, s)
        self.step(stream, dense=src_a)
        self.hT.copy_(self.T, non_blocking=True)

    def cpu_sample(self, A, B):
        import oracle
        t0 = time.perf_counter()
        if self.kind == "cfg1":
            oracle.bool_mul_w64(oracle.pack_bits(A), oracle.pack_bits(B), self.D)
            ops, what = float(self.D) ** 3, "oracle packed product 512^3"
        elif self.kind == "prod16k":
            rows = 2048
            Ap = oracle.pack_bits(A)
            oracle.bool_mul_w64(Ap[:rows], Ap, self.D)
            ops, what = float(rows) * self.D * self.D, f"oracle packed product, rows 0..{rows - 1} of 16384^3"
        else:
            rows = 2048
            Ap = oracle.pack_bits(A)
            oracle.bool_mul_w64(Ap[:rows], Ap, self.D)
            ops, what = float(rows) * self.D * self.D, f"oracle packed product, rows 0..{rows - 1} of 16384^3"
        dt = time.perf_counter() - t0
        return {"ops": ops, "seconds": dt, "sample": what}


WORKLOADS = {
    "cfg2": lambda: Cfg2(4096, "u8"),
    "cfg2-8192": lambda: Cfg2(8192, "u8"),
    "u16": lambda: Cfg2(4096, "u16"),
    "u32": lambda: Cfg2(4096, "u32"),
    "cfg4": lambda: Cfg4(2000),
    "cfg4-200": lambda: Cfg4(200),
    "cfg5": lambda: Cfg5(),
    "cfg1": lambda: CfgBool("cfg1"),
    "cfg3": lambda: CfgBool("cfg3"),
    "prod16k": lambda: CfgBool("prod16k"),
}


def pct(xs, q):
    xs = sorted(float(x) for x in xs)
    return xs[min(len(xs) - 1, int(round(q * (len(xs) - 1))))]


def run_cfg5(args, wl):
    """Served stream against serial single calls.  The latency target is fixed before the
    sweep from isolated service times: every pooled request is run alone (best of two)
    and the p99 target is 3x the slowest of those times.  Each rate then gets
    wl.per_rate Poisson arrivals (the same sequence for both forms), and the line reports,
    per form, the highest throughput whose p99 latency meets the target."""
    import torch
    dev = torch.device("cuda", 0)
    reqs, _ = wl.host_inputs()
    wl.setup_device(reqs, None, dev)
    stream = torch.cuda.Stream(device=dev)
    bufs = {}
    alone = []
    for it in wl.items:
        best = None
        for _ in range(2):
            t0 = time.perf_counter()
            wl.run_single(it, stream, bufs)
            dt = (time.perf_counter() - t0) * 1e3
            best = dt if best is None else min(best, dt)
        alone.append(best)
    capacity = len(wl.items) / (sum(alone) * 1e-3)             # requests/s, one at a time
    target = 3.0 * max(alone)
    sweep = []
    for i, f in enumerate(wl.fracs):
        rate = f * capacity
        lat_s, gops_s, stats = wl.serve_run(rate, wl.per_rate, 100 + i)
        lat_1, gops_1 = wl.serial_run(rate, wl.per_rate, 100 + i, stream)
        sweep.append({"rate_x_capacity": f, "rate_req_s": rate,
                      "served": {"gops": gops_s, "p50_ms": pct(lat_s, 0.5), "p99_ms": pct(lat_s, 0.99),
                                 "meets_target": bool(pct(lat_s, 0.99) <= target),
                                 "batched_launches": stats["batches"],
                                 "arena_peak_bytes": stats["arena_peak_bytes"]},
                      "serial_single_calls": {"gops": gops_1, "p50_ms": pct(lat_1, 0.5), "p99_ms": pct(lat_1, 0.99),
                                              "meets_target": bool(pct(lat_1, 0.99) <= target)}})

    def best(form):
        ok = [x[form]["gops"] for x in sweep if x[form]["meets_target"]]
        return max(ok) if ok else None
    line = {"metric": METRIC, "value": best("served"), "unit": UNIT, "n_gpus": 1,
            "steps": wl.per_rate, "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
            "config": {"workload": wl.name, "capacity_req_s_serial": capacity,
                       "pool": [(it["kind"], it["D"]) for it in wl.items]},
            "p99_target_ms": target,
            "p99_target_rule": "3x the slowest pooled request served alone (best of two runs), fixed before the sweep",
            "within_target_gops": {"served": best("served"), "serial_single_calls": best("serial_single_calls")},
            "served_sweep": sweep}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- arms
def run_reference(args, world, rank):
    """The CPU oracle, as it stands, on the host cores; rank 0 only."""
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]()
    WA, WB = wl.host_inputs()
    for _ in range(args.warmup):
        wl.cpu_sample(WA, WB)
    times, sample = [], None
    for _ in range(args.steps):
        r = wl.cpu_sample(WA, WB)
        times.append(r["seconds"])
        sample = r
    mean = sum(times) / len(times)
    value = sample["ops"] / mean / 1e9
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
        "config": bench_config(wl, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    import paper_1705_08743_gb300 as sr

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]()
    if isinstance(wl, Cfg5):
        run_cfg5(args, wl)
        return
    wl.only = args.only
    if hasattr(wl, "closure_mode"):
        # a product-only run needs no closure autotune (its launches would come first)
        wl.closure_mode = "stream" if args.only == "mul" and args.closure == "auto" else args.closure
    if args.tuning:
        wl.fixed_tuning = tuple(int(x) for x in args.tuning.split(","))
    WA, WB = wl.host_inputs()

    # CPU baseline first (rank 0, N = 1): before any GPU work of this process
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        r = wl.cpu_sample(WA, WB)
        cpu = {"value": r["ops"] / r["seconds"] / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": r["sample"]}

    wl.setup_device(WA, WB, dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # pipe peak of the product's inner operation, measured on this GPU now
    with torch.cuda.stream(stream):
        probe = {"u8": sr.SR_PEAK_DPX_S16X2, "u16": sr.SR_PEAK_U16_PAIR,
                 "u32": sr.SR_PEAK_U32_PAIR}.get(wl.dtype, sr.SR_PEAK_LOP3)
        pk_ms, pk_ips, pk_ops = sr.sr_peak_probe(probe, iters=8192, blocks_per_sm=8, stream=stream.cuda_stream)
        f8 = None
        if getattr(wl, "kind", "") == "cfg3":       # the tensor-core count path's own instruction
            f8 = sr.sr_peak_probe(sr.SR_PEAK_TC_F8, iters=65536, blocks_per_sm=1, stream=stream.cuda_stream)[2]

    pre = getattr(wl, "pre_step", lambda st: None)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            pre(stream)
            flush.zero_()
            wl.step(stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    wl.mul_events = []
    wl.closure_events = []
    barrier(world)
    torch.cuda.synchronize()
    launches0 = sr.sr_kernel_launches()
    ev = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            pre(stream)
            flush.zero_()                                   # L2 flush, outside the events
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wl.step(stream, record_mul=True)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    launches = sr.sr_kernel_launches() - launches0
    barrier(world)
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    mul_ms = [a.elapsed_time(b) for a, b in wl.mul_events]
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = world * wl.ops / (ms_per_step * 1e-3) / 1e9

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        wl.e2e_setup(WA, WB)
        with torch.cuda.stream(stream):
            for _ in range(2):
                wl.e2e_step(stream)
        torch.cuda.synchronize()
        barrier(world)
        ee = []
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                pre(stream)
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                wl.e2e_step(stream)
                e1.record(stream)
                ee.append((e0, e1))
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ee), world) / args.steps
        e2e = {"value": world * wl.ops / (e2e_ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": wl.h2d, "d2h_bytes_per_step": wl.d2h}
        if getattr(wl, "transfer", None):
            e2e["transfer"] = wl.transfer

    if rank != 0:
        return
    if args.only:
        print(json.dumps({"only": args.only, "ms_per_step": ms_per_step, "gpu_launches": launches}), flush=True)
        return
    if isinstance(wl, CfgBool):
        t = sum(mul_ms) / len(mul_ms)
        extra = {"step_us": t * 1e3}
        if wl.kind == "cfg3":
            extra.update(wl.other_forms_ms(stream))
        if wl.kind == "prod16k":
            extra["forms_ms"] = wl.forms_ms(stream)
        kern = {"cfg1": "bool_mul_kernel<32,16,4,4,4> (split K)", "prod16k": "bool_m4r_kernel<8>"}.get(wl.kind)
        achieved = wl.ops / (t * 1e-3) / 1e9
        if wl.kind == "cfg1":            # A, B read and C written once: 3 x 512 x 512 bits
            extra["algorithmic_hbm_gbs"] = 3 * wl.D * wl.D / 8 / (t * 1e-3) / 1e9
        if wl.kind == "cfg3":            # D^3 multiply-adds on the tensor cores: 2 D^3 fp8 flops
            fp8 = f8 / 1e12
            tflops = 2.0 * wl.ops / (t * 1e-3) / 1e12
            roof = {"bound": "tensor", "kernel": "bool_tc_persistent_kernel (panels, phase 3, the diagonal blocks' "
                                                  "updates and squarings) + operand expansion + bit packing",
                    "achieved": tflops, "peak": fp8, "unit": "TFLOP/s", "frac": tflops / fp8,
                    "peak_source": "measured now: tcgen05.mma kind::f8f6f4 128x256x32 issue stream on all SMs "
                                   "(sr_peak_probe SR_PEAK_TC_F8, 0/1 e4m3 operands); MEASURED_PEAKS.json bf16 x 2 "
                                   "(nominal fp8:bf16 ratio) beside it",
                    "peak_bf16x2": 2.0 * measured_bf16_tflops(),
                    "launch_ms": t, "traffic": None,
                    "lop3_equivalent": {"achieved_gops": achieved, "lop3_peak_gops": pk_ops / 1e9}}
        else:
            roof = {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": pk_ops / 1e9, "unit": "Gop/s",
                    "frac": achieved / (pk_ops / 1e9),
                    "peak_source": "measured now: issue-bound LOP3 (acc | x & m, 32 columns per instruction) on "
                                   "all SMs" + ("; the table method needs fewer instructions per op than the "
                                                "masked OR" if wl.kind == "prod16k" else ""),
                    "launch_ms": t, "traffic": None}
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bits", "data": "synthetic",
            "config": bench_config(wl, world),
            "boolean": extra, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk}), flush=True)
        return
    if isinstance(wl, Cfg4):
        print(json.dumps(cfg4_line(args, wl, world, value, ms_per_step, step_ms, pk_ops, cpu, e2e, launches, clk,
                                   stream, flush)), flush=True)
        return
    mul_avg = sum(mul_ms) / len(mul_ms)
    achieved = wl.D ** 3 / (mul_avg * 1e-3) / 1e9
    peak = pk_ops / 1e9
    sr.sr_stream_status(wl.ctx, stream.cuda_stream)      # no bounded wait of the closure gave up
    clo_ms = [a.elapsed_time(b) for a, b in wl.closure_events]
    clo_avg = sum(clo_ms) / len(clo_ms)
    clo_achieved = wl.D ** 3 / (clo_avg * 1e-3) / 1e9
    n0 = sr.sr_kernel_launches()
    with torch.cuda.stream(stream):
        sr.antidist_closure(wl.ctx, wl.T, wl.D, wl.D, wl.sdt, stream.cuda_stream)
    torch.cuda.synchronize()
    nl = sr.sr_kernel_launches() - n0
    nb = (wl.D + 127) // 128
    fused = nl == nb + 1 and nl != 1
    fused_key = f"closure_fused_kernel<Kind{wl.dtype.upper()}>"
    kernel = ("antidist_closure stream schedule (pivot-block kernel, panel and phase-3 products)" if nl not in (1, nb + 1)
              else f"antidist_closure_persistent_kernel<Kind{wl.dtype.upper()}> (whole closure, one launch)" if nl == 1
              else f"{fused_key} (one launch per pivot block)")
    # one closure: nl launches on one stream; per launch D^3 / nl ops in clo_avg / nl ms
    roof_closure = {"bound": "alu", "kernel": kernel,
                    "achieved": clo_achieved, "peak": peak, "unit": "Gop/s", "frac": clo_achieved / peak,
                    "launch_ms": clo_avg / nl, "launches_per_closure": nl, "closure_ms": clo_avg,
                    "timing": "CUDA events around the antidist_closure call, encode excluded",
                    "traffic": load_traffic(fused_key, FUSED_SOURCES, args.workload) if fused else None,
                    "schedule": CLOSURE_TUNED.get(wl.D, "forced by --closure")}
    roof_product = {"bound": "alu", "kernel": wl.roofline_kernel, "achieved": achieved, "peak": peak,
                    "unit": "Gop/s", "frac": achieved / peak,
                    "peak_source": "measured now: issue-bound DPX add-max stream on all SMs (sr_peak_probe)",
                    "launch_ms": mul_avg,
                    "traffic": load_traffic(wl.roofline_kernel, wl.roofline_sources, args.workload)}
    # the dominant kernel by live time in the step: the product kernel, which the stream
    # schedule's phase 3 also runs, unless the closure is one kernel that takes longer
    if fused and clo_avg > mul_avg:
        roofline = dict(roof_closure, peak_source=roof_product["peak_source"], product=roof_product,
                        dominant="the closure's kernel: the larger share of the step's CUDA-event time")
    else:
        roofline = dict(roof_product, closure=roof_closure,
                        dominant="the product kernel (also the stream schedule's phase 3)")
    extra = {}
    if wl.D == 4096 and wl.dtype == "u8" and not args.no_8192:
        extra["closure_8192"] = closure_8192(dev, stream, flush, peak, local, args)
    if wl.D == 4096 and wl.dtype == "u8" and not args.no_batched:
        extra["batched_cfg4"] = batched_summary(dev, stream, flush, args)
    if wl.D == 4096 and wl.dtype == "u8" and not args.no_bool:
        extra["bool_closure_cfg3"] = bool_closure_summary(dev, stream, flush)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic",
        "config": {"workload": wl.name, "step": "encode x3 + closure (in place) + product",
                   "ops_per_step": wl.ops, "l2": f"flushed before each step ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline,
        "parts_ms": {"product": mul_avg, "closure": clo_avg, "encode_x3": ms_per_step - mul_avg - clo_avg},
        "extra": extra,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def closure_8192(dev, stream, flush, peak, local, args, reps=5):
    """The anti-distance closure at D = 8192 u8 (the config-2 generator at twice the size):
    `reps` closures timed with CUDA events, each on a fresh copy of the encoded matrix
    (copied and L2 flushed outside the events), clocks sampled during them."""
    import numpy as np
    import torch
    import synth
    import paper_1705_08743_gb300 as sr
    D = 8192
    W = synth.cfg2_antidist(D=D, seed=1, s_edge=0, dtype=np.uint8)
    Wd = torch.from_numpy(W).to(dev)
    T0 = torch.empty((D, D), dtype=torch.uint8, device=dev)
    T = torch.empty_like(T0)
    s = stream.cuda_stream
    ctx = closure_ctx(D, sr.SR_U8, args.closure)
    with torch.cuda.stream(stream):
        sr.antidist_encode(None, Wd, D, T0, D, D, D, sr.SR_U8, s)
        for _ in range(2):
            T.copy_(T0)
            sr.antidist_closure(ctx, T, D, D, sr.SR_U8, s)
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    ev = []
    with torch.cuda.stream(stream):
        for _ in range(reps):
            T.copy_(T0)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sr.antidist_closure(ctx, T, D, D, sr.SR_U8, s)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in ev]
    avg = sum(ms) / len(ms)
    achieved = D ** 3 / (avg * 1e-3) / 1e9
    sr.sr_stream_status(ctx, s)          # no bounded wait gave up
    sr.sr_destroy(ctx)
    del Wd, T0, T
    return {"workload": "antidist_closure D=8192 u8 (edge p=0.05, length U{1..31}, seed 1)", "reps": reps,
            "schedule": CLOSURE_TUNED.get(D, "forced by --closure"),
            "ms": avg, "ms_min": min(ms), "ms_max": max(ms), "achieved": achieved, "peak": peak, "unit": "Gop/s",
            "frac": achieved / peak, "clocks": clk}


def bool_closure_summary(dev, stream, flush, steps=5):
    """Config 3 (Boolean transitive closure, D=16384, 64-bit words) beside the default
    step: pack + blocked Warshall with phase 3 on the tensor cores, timed `steps` times
    with the L2 flushed, against the fp8 tensor-pipe peak probed now (D^3 multiply-adds
    of 0/1 e4m3 operands = 2 D^3 flops)."""
    import torch
    import paper_1705_08743_gb300 as sr
    wl = CfgBool("cfg3")
    A, _ = wl.host_inputs()
    wl.setup_device(A, None, dev)
    del A
    with torch.cuda.stream(stream):
        f8 = sr.sr_peak_probe(sr.SR_PEAK_TC_F8, iters=65536, blocks_per_sm=1, stream=stream.cuda_stream)[2] / 1e12
        for _ in range(2):
            wl.step(stream)
    torch.cuda.synchronize()
    ev = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wl.step(stream)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    sr.sr_stream_status(wl.wctx, stream.cuda_stream)
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    avg = sum(ms) / len(ms)
    tflops = 2.0 * wl.ops / (avg * 1e-3) / 1e12
    out = {"workload": wl.name, "steps": steps, "ms": avg, "ms_min": ms[0], "ms_max": ms[-1],
           "bound": "tensor", "achieved": tflops, "peak": f8, "unit": "TFLOP/s", "frac": tflops / f8,
           "peak_source": "measured now: tcgen05.mma kind::f8f6f4 issue stream on all SMs (SR_PEAK_TC_F8)",
           "l2": "flushed before each step"}
    sr.sr_destroy(wl.ctx)
    sr.sr_destroy(wl.wctx)
    del wl
    torch.cuda.empty_cache()
    return out


def batched_summary(dev, stream, flush, args, steps=5):
    """Config 4 (2000 graphs, D log-uniform [32,1024], u16) beside the default step: the
    autotuned batch launch timed `steps` times on restored inputs with the L2 flushed, its
    fraction of the u16 pipe peak (probed now), each graph's completion time inside a
    launch (device-clock stamps, every graph of `steps` launches), and a loop of single
    calls on the same graphs."""
    import torch
    import paper_1705_08743_gb300 as sr
    wl = Cfg4(2000)
    pool, _ = wl.host_inputs()
    wl.setup_device(pool, None, dev)
    with torch.cuda.stream(stream):
        pk = sr.sr_peak_probe(sr.SR_PEAK_U16_PAIR, iters=8192, blocks_per_sm=8, stream=stream.cuda_stream)[2] / 1e9
        for _ in range(3):
            wl.pre_step(stream)
            wl.step(stream)
    torch.cuda.synchronize()
    ev = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            wl.pre_step(stream)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wl.step(stream)
            e1.record(stream)
            ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    avg = sum(ms) / len(ms)
    comp = wl.completion_ms(stream, flush, launches=steps)
    loop_ms = wl.loop_of_single_calls_ms(stream, reps=1)
    out = {"workload": wl.name, "tuning(cluster,coop_threshold,ctas_per_sm)": wl.tuning, "launches": steps,
           "ms": avg, "value": wl.ops / (avg * 1e-3) / 1e9, "unit": UNIT, "peak": pk,
           "frac": wl.ops / (avg * 1e-3) / 1e9 / pk,
           "launch_ms": {"p50": pct(ms, 0.5), "p99": pct(ms, 0.99)},
           "graph_completion_ms": {"p50": pct(comp, 0.5), "p99": pct(comp, 0.99), "samples": len(comp)},
           "loop_of_single_calls_ms": loop_ms, "speedup_vs_loop": loop_ms / avg}
    sr.sr_batch_destroy(wl.batch)
    sr.sr_destroy(wl.ctx)
    del wl
    torch.cuda.empty_cache()
    return out


def cfg4_line(args, wl, world, value, ms_per_step, step_ms, pk_ops, cpu, e2e, launches, clk, stream, flush):
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
    comp = wl.completion_ms(stream, flush)
    loop_ms = wl.loop_of_single_calls_ms(stream)
    achieved = wl.ops / (ms_per_step * 1e-3) / 1e9
    traffic = load_traffic(wl.roofline_kernel, wl.roofline_sources, args.workload)
    peak = pk_ops / 1e9
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": bench_config(wl, world),
        "batched": {"tuning(cluster,coop_threshold,ctas_per_sm)": wl.tuning,
                    "graph_completion_ms": {"p50": pct(comp, 0.5), "p99": pct(comp, 0.99), "max": max(comp),
                                            "samples": len(comp),
                                            "what": "per graph: device-clock time from the batch launch's start "
                                                    "to that graph's completion (every graph of 5 launches)"},
                    "launch_ms": {"p50": p50, "p99": p99, "samples": len(srt),
                                  "what": "whole batch launch, one sample per timed step"},
                    "loop_of_single_calls_ms": loop_ms,
                    "speedup_vs_loop": loop_ms / ms_per_step},
        "roofline": {"bound": "alu", "kernel": wl.roofline_kernel, "achieved": achieved, "peak": peak,
                     "unit": "Gop/s", "frac": achieved / peak,
                     "peak_source": "measured now: issue-bound max.u16x2 + DPX add-max stream on all SMs",
                     "launch_ms": ms_per_step, "traffic": traffic,
                     "achieved_hbm_gbs": traffic / (ms_per_step * 1e-3) / 1e9 if traffic else None,
                     "algorithmic_hbm_gbs": wl.alg_bytes / (ms_per_step * 1e-3) / 1e9},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
    }


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
