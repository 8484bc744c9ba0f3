#!/usr/bin/env python
"""Throughput of batched MN-BaB bounding on one GB300: BaB nodes bounded / s.

Workload: the 28x28 conv net 1x28x28 -> conv16 4x4 s2 -> ReLU -> conv32 4x4 s2
-> ReLU -> FC100 -> ReLU -> FC10 (He-normal, seed 1), properties built from
seeded blurred-uniform images with the calibrated L-inf radius, margins
y_t - y_j as rows, 256-node budget per property, up to 512 subproblems per
BaB step, 20 projected-Adam steps per node with the adjoint kernels.  A
rolling window of 100 active properties keeps the queue full: a finished
property is replaced by the next seeded one.  All properties are uploaded to
HBM before timing; a new property's root bounding runs inside the step that
admits it.

One step = one mnbab_bab_step (re-bounding after splits, DeepPoly pass,
optimisation, counterexample check, ACS, queue step) over one batch.  Steps
are timed with CUDA events on the library's stream; L2 is flushed (256 MiB
write) between timed steps, outside the timed spans.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload instead.  Besides that arm, this file runs the oracle only in its CPU
baseline legs: the line's cpu_baseline and the intermediate-bounds block's.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

CFG = 1
WINDOW = 100
BATCH = 512
BUDGET = 256
ADAM_STEPS = 20
METRIC = "BaB nodes bounded/s & verdicts@timeout, batched/serving vs plain, 1 GB300"
SERVE_CAPACITY = 4096     # node slots per network in the serving context
SERVE_HBM = 64 << 30      # serving context's HBM budget (config 4: 64 GB)
WORKLOAD = ("conv_small_28: 1x28x28 -> conv16 4x4 s2 -> ReLU -> conv32 4x4 s2 -> ReLU -> FC100 -> "
            "ReLU -> FC10, 100 active properties (rolling window), 9 margin rows each, "
            "<=512 subproblems per step, 20 Adam steps per node, budget 256 nodes/property")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-nodes", type=int, default=512,
                    help="nodes of the plain one-subproblem-per-launch arm")
    ap.add_argument("--e2e-steps", type=int, default=2,
                    help="cold solves of the e2e arm (0 skips the e2e arm)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--node-capacity", type=int, default=65536,
                    help="node slots of the context (device memory ~ 122 KB per slot)")
    ap.add_argument("--window", type=int, default=WINDOW, help="active properties")
    ap.add_argument("--graphs", action="store_true",
                    help="replay the optimisation loop from captured CUDA graphs")
    ap.add_argument("--gemm-tc", action="store_true",
                    help="tensor-core GEMM check: conv_big_32 root bounding on the tcgen05 path")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving run (Poisson request stream), full size")
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests of the serving stream (default 24 in the main line, 400 with --serving)")
    ap.add_argument("--serve-rate", type=float, default=4.0)
    ap.add_argument("--mnc-big-only", action="store_true",
                    help="run only the conv_big_32 arm with multi-neuron constraints")
    ap.add_argument("--mnc-big-capacity", type=int, default=4096,
                    help="node slots of the conv_big_32 arm's context")
    ap.add_argument("--mnc-big-steps", type=int, default=3)
    ap.add_argument("--mnc-big-props", type=int, default=32,
                    help="properties of the conv-big arm with multi-neuron constraints (0 skips it)")
    ap.add_argument("--mnc-big-groups", type=int, default=2000,
                    help="constraint groups per ReLU layer in the conv-big arm")
    ap.add_argument("--inter-nodes", type=int, default=128,
                    help="root nodes of the optimised-intermediate-bounds arm (0 skips it)")
    ap.add_argument("--verdicts", default="0,2,3",
                    help="configurations of the verdicts-at-timeout runs (empty skips them)")
    ap.add_argument("--verdicts-full", action="store_true",
                    help="verdicts at the specified sizes (100 / 50 properties, 60 / 120 s "
                         "timeouts) instead of the bounded default sample; only these runs")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# Replicas: ranks bound disjoint seeded property streams (no data-path
# collective); the only exchange is the timing / node-count reduction.
RANK_STRIDE = 1_000_000


def rank_start(rank: int) -> int:
    """First property index of a rank's stream (disjoint across ranks)."""
    return rank * RANK_STRIDE


def reduce_timing(ms: float, nodes: int, device="cpu"):
    """(max of ms over ranks, sum of nodes over ranks); identity without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, nodes
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(nodes)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dominant(stats):
    kern = {k: v for k, v in stats.items() if not k.startswith(("step_", "phase_"))}
    return max(kern.items(), key=lambda kv: kv[1]["ms"])


CONTRACTIONS = ("backsub_fc_gemm", "backsub_conv_transpose", "forward_fc_gemm", "forward_conv",
                "opt_fused_chain", "backsub_conv_window", "backsub_rows_fused", "backsub_conv_tc",
                "forward_conv_tc", "opt_fused_chain_tc")


def measure_tf32(n=8192, reps=5):
    """Dense TF32 rate of cuBLAS on this GPU (torch.matmul of two n x n FP32
    matrices with TF32 allowed), best of `reps` after a warm-up, CUDA events."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = a @ b
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b, c
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def tf32x3_peak(peaks, src):
    """3xTF32 tensor peak: a measured dense TF32 rate / 3 when there is one
    (bench.py measures cuBLAS TF32 in the run), else the measured dense BF16
    burst rate x the nominal TF32:BF16 ratio 1/2, / 3 (three TF32 products per
    FP32-accurate product)."""
    if "tf32_tflops" in peaks:
        return peaks["tf32_tflops"] / 3.0, peaks.get("tf32_source", f"{src}: tf32_tflops") + " / 3"
    return (peaks["bf16_tflops"] / 2.0 / 3.0,
            f"derived from {src} bf16_tflops {peaks['bf16_tflops']}: x 1/2 (nominal TF32:BF16) "
            f"/ 3 (3xTF32 split products)")


def chain_macs(layers):
    """(C, d_R): MACs of one back-substitution row through every affine layer
    below the objective, and the width of the last ReLU layer."""
    C, dR = 0.0, 0
    for L in layers[:-1]:
        if L["kind"] == "fc":
            C += L["W"].shape[0] * L["W"].shape[1]
            dR = L["W"].shape[0]
        elif L["kind"] == "conv":
            co, ho, wo = L["out_shape"]
            C += co * ho * wo * L["W"].shape[1] * L["W"].shape[2] * L["W"].shape[3]
            dR = co * ho * wo
    return C, dR


def roofline(stats, peaks, src, kernels_hash, layers=None, adam_steps=ADAM_STEPS):
    """Dominant kernel class (largest summed launch time) against its roofline.

    Back-substitution and adjoint contractions are tensor-core work by the
    method's shape (dense Lambda W products), so they are measured against the
    3xTF32 peak whether or not the kernel uses the tensor pipe; their SIMT FP32
    fraction is reported beside it.  The other classes are HBM-bound."""
    name, st = dominant(stats)
    per_launch_ms = st["ms"] / max(1, st["launches"])
    ach_flops = st["flops"] / (st["ms"] * 1e-3) / 1e12
    if name in CONTRACTIONS:
        peak, psrc = tf32x3_peak(peaks, src)
        r = {"bound": "tensor", "achieved": ach_flops, "peak": peak, "unit": "TFLOP/s",
             "peak_kind": "3xTF32 (FP32-accurate split products)", "peak_source": psrc}
        simt = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        r["simt_fp32"] = {"peak": simt, "frac": ach_flops / simt,
                          "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
        if name in ("opt_fused_chain", "opt_fused_chain_tc") and layers is not None:
            # the library counts (steps + 1) back-substitution sweeps and steps
            # adjoint passes (one forward pass of the relaxed network each); the
            # second count charges a sweep plus a two-sweep adjoint per step
            C, dR = chain_macs(layers)
            ours = (adam_steps + 1) * (C + dR) + adam_steps * C
            three = 3.0 * adam_steps * C
            a2 = ach_flops * three / ours
            r["three_sweep_count"] = {"achieved": a2, "frac": a2 / peak,
                                      "flops_per_row": 2.0 * three,
                                      "library_flops_per_row": 2.0 * ours}
    else:
        peak = peaks["hbm_gbs"]
        ach = st["bytes"] / (st["ms"] * 1e-3) / 1e9
        r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
             "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
    r["frac"] = r["achieved"] / r["peak"]
    r["kernel"] = name
    r["launches"] = st["launches"]
    r["avg_launch_us"] = per_launch_ms * 1e3
    r["traffic"] = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        # DRAM bytes per row from one capture, scaled by the rows of an average
        # launch (its algorithmic flops over the flops of one row)
        sha = t.get("kernels_sha", {})
        if (isinstance(sha, dict) and sha.get(name) == kernels_sha(name)
                and name in t.get("dram_bytes_per_row", {})
                and name in t.get("flops_per_row", {})):
            rows = st["flops"] / max(1, st["launches"]) / t["flops_per_row"][name]
            r["traffic"] = t["dram_bytes_per_row"][name] * rows
    except (OSError, ValueError):
        pass
    return r


# sources a kernel class's code lives in (the traffic record of a class stays
# valid while these files are unchanged); other classes hash every source
KERNEL_SOURCES = {
    "opt_fused_chain": ("fused.cu", "epilogue.cuh", "mnbab_internal.h"),
    "opt_fused_chain_tc": ("fused.cu", "epilogue.cuh", "mnbab_internal.h", "tc_common.cuh"),
    "backsub_conv_tc": ("tc_conv.cu", "tc_common.cuh", "epilogue.cuh", "mnbab_internal.h"),
    "forward_conv_tc": ("tc_conv.cu", "tc_common.cuh", "epilogue.cuh", "mnbab_internal.h"),
}


def kernels_sha(kernel=None):
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2205_00263_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES.get(kernel) or os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
class Window:
    """Rolling window of active properties.

    With preload (the device-timed arm) every property of the pool is drawn and
    uploaded to HBM before any timing starts; admission inside the steps only
    hands the next uploaded property to bab_step, which starts it (root nodes,
    root bounds) in its own launches.  Without preload (the end-to-end arm)
    admission uploads the property from its host arrays inside the step, and a
    finished property's verdict and counterexample are read back.
    """

    def __init__(self, ctx, net, layers, eps, start, n_active, pool_size=None, preload=True):
        self.ctx, self.net, self.layers, self.eps = ctx, net, layers, eps
        self.next = 0
        self.preload = preload
        pool = synth.make_properties(CFG, layers, n=pool_size or 4 * n_active, eps=eps,
                                     start=start)
        self.h2d = 0
        self.d2h = 0
        self.pool = [self._upload(pr) for pr in pool] if preload else pool
        self.active = []
        self.verdicts = {1: 0, -1: 0, 0: 0}
        for _ in range(n_active):
            self.admit()

    def _upload(self, pr):
        p = self.ctx.set_property(self.net, pr.lo, pr.hi, pr.C, pr.d)
        self.ctx.set_budget(p, BUDGET)
        self.h2d += pr.lo.nbytes + pr.hi.nbytes + pr.C.nbytes + pr.d.nbytes
        return p

    def admit(self):
        if self.next >= len(self.pool):
            raise RuntimeError("property pool exhausted; raise pool_size")
        pr = self.pool[self.next]
        self.active.append(pr if self.preload else self._upload(pr))
        self.next += 1

    def step(self):
        st = self.ctx.bab_step(self.active, max_nodes=BATCH, steps=ADAM_STEPS)
        keep = []
        for p in self.active:
            if self.ctx.queue_size(p) == 0:
                v, _, _ = self.ctx.verdict(p)
                self.d2h += 8 + 4 * self.net.d0  # verdict, bound, minimiser
                self.verdicts[v] += 1
            else:
                keep.append(p)
        n_done = len(self.active) - len(keep)
        self.active = keep
        for _ in range(n_done):
            self.admit()
        self.h2d += st["h2d_bytes"]
        self.d2h += st["d2h_bytes"]
        return st


def run_ours(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2205_00263_gb300 import Context

    # a dedicated stream: the library launches on it (CUDA graphs cannot be
    # captured on the legacy default stream) and the step events are recorded on it
    stream = torch.cuda.Stream()
    layers = synth.make_network(CFG)
    eps = synth.load_eps(CFG)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ap_graphs = args.graphs
    ctx = Context(device=local, stream=stream.cuda_stream, node_capacity=args.node_capacity,
                  graphs=ap_graphs)
    net = ctx.load_network(layers)
    start = rank_start(rank)
    win = Window(ctx, net, layers, eps, start, args.window,
                 pool_size=args.window + 60 * (args.steps + args.warmup + 1) + 50)

    for _ in range(args.warmup):
        win.step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    # one untimed step with every kernel class timed: the per-class breakdown and
    # the dominant class; the timed steps then time that class alone (per-launch
    # events on every class would add their own overhead to the measured steps)
    ctx.profile(True)
    win.step()
    torch.cuda.synchronize()
    breakdown, _ = ctx.profile_read()
    dom_name = dominant(breakdown)[0]
    ctx.profile(True)
    ctx.profile_mask([dom_name])
    _, launches0 = ctx.profile_read()
    clocks = Clocks(local)
    clocks.start()
    nodes = 0
    ms = 0.0
    verdicts0 = dict(win.verdicts)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = win.step()
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        nodes += st["nodes_bounded"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats, launches1 = ctx.profile_read()
    ctx.profile(False)
    ctx.profile_mask(None)
    stats = {dom_name: stats[dom_name]}
    tot_ms, tot_nodes = reduce_timing(ms, nodes, device="cuda")
    value = tot_nodes / (tot_ms * 1e-3)

    # plain: one subproblem per launch on fresh properties (same kernels, no batching)
    plain = None
    if args.plain_nodes > 0:
        win2 = Window(ctx, net, layers, eps, start + 500_000, 8, pool_size=8 + args.plain_nodes)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        pn = 0
        e0.record(stream)
        while pn < args.plain_nodes:
            st = win2.ctx.bab_step(win2.active, max_nodes=1, steps=ADAM_STEPS)
            pn += st["nodes_bounded"]
            if st["nodes_bounded"] == 0:
                win2.admit()
        e1.record(stream)
        e1.synchronize()
        pms = e0.elapsed_time(e1)
        plain = {"value": pn / (pms * 1e-3), "unit": "nodes/s", "nodes": pn,
                 "properties": win2.next,
                 "form": "one subproblem per launch (max_nodes=1), same kernels, no graph"}

    # e2e: the same rolling-window workload through the public API, every step
    # uploading its newly admitted properties from host arrays and reading the
    # finished properties' verdicts back, timed on the host clock
    e2e = None
    if args.e2e_steps > 0:
        # a context of its own: the device-timed window still holds its nodes
        ectx = Context(device=local, stream=stream.cuda_stream, node_capacity=args.node_capacity)
        enet = ectx.load_network(layers)
        win3 = Window(ectx, enet, layers, eps, start + 700_000, args.window,
                      pool_size=args.window + 60 * (args.steps + args.warmup + 1) + 50,
                      preload=False)
        for _ in range(args.warmup):
            win3.step()
        torch.cuda.synchronize()
        h0, d0_ = win3.h2d, win3.d2h
        en, et = 0, 0.0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = win3.step()
            torch.cuda.synchronize()
            et += time.perf_counter() - t0
            en += st["nodes_bounded"]
        et_ms, en = reduce_timing(et * 1e3, en, device="cuda")
        e2e = {"value": en / (et_ms * 1e-3), "unit": "nodes/s",
               "h2d_bytes_per_step": (win3.h2d - h0) // args.steps,
               "d2h_bytes_per_step": (win3.d2h - d0_) // args.steps,
               "step": "one mnbab_bab_step over the 100-property rolling window; newly admitted "
                       "properties uploaded from host arrays and finished verdicts read back "
                       "inside the timed step (host clock)"}
        # cold solves: fresh properties from host arrays to verdicts
        cn, ct = 0, 0.0
        pools = [synth.make_properties(CFG, layers, n=16, eps=eps, start=start + 800_000 + 1000 * k)
                 for k in range(args.e2e_steps)]
        for k in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            props = []
            for pr in pools[k]:
                p = ectx.set_property(enet, pr.lo, pr.hi, pr.C, pr.d)
                ectx.set_budget(p, 32)
                props.append(p)
            while True:
                nb = ectx.bab_step(props, max_nodes=BATCH, steps=ADAM_STEPS)["nodes_bounded"]
                cn += nb
                if nb == 0:
                    break
            for p in props:
                ectx.verdict(p)
            torch.cuda.synchronize()
            ct += time.perf_counter() - t0
        e2e["cold_solve"] = {"value": cn / ct, "unit": "nodes/s", "solves": args.e2e_steps,
                             "solve": "16 fresh properties from host arrays (32-node budget "
                                      "each) to verdicts"}
        ectx.close()
    inter = None
    if args.inter_nodes > 0:
        inter = intermediate_run(local, stream, layers, eps, start + 600_000, args.inter_nodes,
                                 0 if (args.no_cpu_baseline or rank != 0) else 4)
    serving = None
    if world == 1 and (args.serve_requests is None or args.serve_requests > 0):
        sctx = Context(device=local, stream=stream.cuda_stream, node_capacity=SERVE_CAPACITY,
                       hbm_budget_bytes=SERVE_HBM)
        try:
            serving = serving_run(sctx, serving_nets(sctx), args.serve_requests or 24, args.serve_rate,
                                  seed=4, timeout_s=60.0, budget=BUDGET, plain_cap_s=15.0,
                                  stream=stream)
        finally:
            sctx.close()
    peaks, src = load_peaks()
    if "tf32_tflops" not in peaks:
        tf = measure_tf32()
        peaks["tf32_tflops"] = tf
        peaks["tf32_source"] = (f"measured in this run: cuBLAS TF32 GEMM 8192^3, best of 5 "
                                f"({tf:.1f} TFLOP/s)")
    roof = roofline(stats, peaks, src, kernels_sha(), layers=layers)
    mnc_big = None
    if world == 1 and args.mnc_big_props > 0:
        mnc_big = mnc_big_run(local, stream, args.mnc_big_props, args.mnc_big_steps,
                              args.mnc_big_groups, peaks,
                              src, kernels_sha())
    verdicts = None
    if world == 1 and args.verdicts:
        verdicts = {f"config{c}": verdicts_run(local, stream, int(c), full=False)
                    for c in args.verdicts.split(",")}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)
        cpu = {k: v for k, v in cpu.items() if not k.startswith("_")}
    if rank == 0:
        vd = {k: win.verdicts[k] - verdicts0.get(k, 0) for k in win.verdicts}
        out = {
            "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded He-normal net, blurred-uniform images; no dataset)",
            "config": {"workload": WORKLOAD, "l2": "flushed (256 MiB write) between timed steps",
                       "inputs": "every property uploaded to HBM before the timed region",
                       "parallelism": f"replicas x{world} (independent properties per rank)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches1 - launches0), "clocks": clk,
            "plain": plain,
            "batched_over_plain": (value / world / plain["value"]) if plain else None,
            "verdicts_in_timed_steps": {"verified": vd[1], "falsified": vd[-1], "unknown": vd[0]},
            "kernel_breakdown_ms": {k: round(v["ms"], 3) for k, v in breakdown.items() if v["ms"]},
            "kernel_breakdown_note": "one untimed step before the timed region, every class timed",
            "nodes_timed": tot_nodes,
            "serving": serving,
            "intermediate": inter,
            "conv_big_mnc": mnc_big,
            "verdicts_at_timeout": verdicts,
            "launches_before_timed": int(launches0),
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------------------
# Serving: a Poisson stream of verification requests over the networks whose
# radius has been calibrated, admitted into the running request loop as they
# arrive (continuous batching), against the plain per-request loop.
def serving_run(ctx, nets, n_req, rate, seed, timeout_s, budget, plain_cap_s, stream):
    """Serve one Poisson stream three ways on the same GPU:
    - ``stream``: batched request loop, requests submitted at their arrival
      time on the wall clock (continuous batching);
    - ``burst``: the same requests all submitted at once (saturated throughput);
    - ``plain``: one request at a time in arrival order, one subproblem per
      launch.  Its service times are measured on the GPU; the idle time
      before an arrival is skipped rather than slept, so its times to verdict
      are those of a FIFO single-server run of the same stream."""
    reqs = synth.poisson_stream(rate=rate, n=n_req, seed=seed, nets=tuple(sorted(nets)))
    host = []
    for r in reqs:
        cfg = r["cfg"]
        layers, net, eps = nets[cfg]
        spec = synth.CONFIGS[cfg]
        x0 = synth.make_image(r["input_seed"], spec["in_shape"]).reshape(-1)
        y = synth.net_forward(layers, x0)
        C, d = synth.property_rows(int(np.argmax(y)), y.shape[0])
        lo, hi = synth.input_box(x0, eps)
        host.append((r["arrival_s"], cfg, lo, hi, C, d))

    def submit(k):
        _, cfg, lo, hi, C, d = host[k]
        p = ctx.set_property(nets[cfg][1], lo, hi, C, d)
        ctx.set_budget(p, budget)
        return ctx.submit(p, timeout_s)

    def summary(ttv, verd, nodes, wall):
        ttv = np.asarray(ttv)
        cnt = {"verified": verd.count(1), "falsified": verd.count(-1), "unknown": verd.count(0)}
        return {"requests": len(ttv), "nodes": int(nodes), "wall_s": wall,
                "nodes_per_s": nodes / wall if wall > 0 else None,
                "time_to_verdict_p50_s": float(np.percentile(ttv, 50)) if len(ttv) else None,
                "time_to_verdict_p99_s": float(np.percentile(ttv, 99)) if len(ttv) else None,
                "verdicts": cnt}

    def run_batched(arrivals):
        torch_sync()
        t0 = time.perf_counter()
        pending = list(range(len(host)))
        tickets, t_sub = {}, {}
        nodes = 0
        while pending or any(not ctx.poll(t) for t in tickets.values()):
            now = time.perf_counter() - t0
            while pending and arrivals[pending[0]] <= now:
                k = pending.pop(0)
                tickets[k] = submit(k)
                t_sub[k] = time.perf_counter() - t0
            if not tickets or all(ctx.poll(t) for t in tickets.values()):
                if pending:
                    time.sleep(max(0.0, arrivals[pending[0]] - (time.perf_counter() - t0)))
                continue
            st = ctx.serve_step(BATCH, steps=ADAM_STEPS)
            nodes += st["step"]["nodes_bounded"]
        wall = time.perf_counter() - t0
        ttv, verd = [], []
        for k, t in tickets.items():
            r = ctx.request_result(t)
            ttv.append(t_sub[k] - arrivals[k] + r["total_s"])   # queueing before submission counts
            verd.append(r["verdict"])
        return summary(ttv, verd, nodes, wall)

    arr = [h[0] for h in host]
    out = {"requests": len(host), "rate_per_s": rate, "networks": sorted(nets),
           "timeout_s": timeout_s, "node_budget": budget,
           "stream": run_batched(arr),
           "burst": run_batched([0.0] * len(host))}
    # plain per-request loop, FIFO over the same arrivals
    v, busy, pn, ttv, verd, served = 0.0, 0.0, 0, [], [], 0
    for k in range(len(host)):
        if busy > plain_cap_s:
            break
        start = max(v, arr[k])
        left = arr[k] + timeout_s - start
        torch_sync()
        t1 = time.perf_counter()
        verdict = 0
        if left > 0:
            _, cfg, lo, hi, C, d = host[k]
            p = ctx.set_property(nets[cfg][1], lo, hi, C, d)
            ctx.set_budget(p, budget)
            while time.perf_counter() - t1 < left:
                st = ctx.bab_step([p], max_nodes=1, steps=ADAM_STEPS)
                pn += st["nodes_bounded"]
                if st["nodes_bounded"] == 0:
                    break
            verdict = ctx.verdict(p)[0]
        svc = time.perf_counter() - t1
        busy += svc
        v = start + svc
        ttv.append(v - arr[k])
        verd.append(verdict)
        served += 1
    plain = summary(ttv, verd, pn, busy)
    plain["form"] = "requests one at a time in arrival order, one subproblem per launch"
    plain["requests_of_stream"] = served
    out["plain"] = plain
    if plain["nodes_per_s"]:
        out["burst_nodes_per_s_over_plain"] = out["burst"]["nodes_per_s"] / plain["nodes_per_s"]
    return out


def torch_sync():
    import torch
    torch.cuda.synchronize()


def serving_nets(ctx):
    nets = {}
    for cfg in (1, 2, 3):
        try:
            eps = synth.load_eps(cfg)
        except (KeyError, OSError, ValueError):
            continue
        layers = synth.make_network(cfg)
        nets[cfg] = (layers, ctx.load_network(layers), eps)
    return nets


# ----------------------------------------------------------------------------
# Optimised intermediate bounds (Sec. 3.1, parameter sharing) of root nodes of
# the same workload: one mnbab_optimize_intermediate call over n_nodes roots.
def intermediate_run(local, stream, layers, eps, start, n_nodes, oracle_nodes):
    import torch
    from paper_2205_00263_gb300 import Context
    props = synth.make_properties(CFG, layers, n=n_nodes + 4, eps=eps, start=start)
    # each property also holds its root-bound slot and one root node per row
    ctx = Context(device=local, stream=stream.cuda_stream, node_capacity=4096)
    try:
        net = ctx.load_network(layers)
        ps = [ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d) for pr in props]
        nodes = [ctx.node_root(p, 0) for p in ps]  # starts every property (root bounds)
        # warm-up on 4 other roots (scratch allocation), every kernel class timed
        ctx.profile(True)
        ctx.optimize_intermediate(nodes[:4], steps=ADAM_STEPS)
        stats, _ = ctx.profile_read()
        ctx.profile(False)
        timed = nodes[4:]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        rows = ctx.optimize_intermediate(timed, steps=ADAM_STEPS)
        e1.record(stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
    finally:
        ctx.close()
    top = sorted(((k, v["ms"]) for k, v in stats.items()
                  if v["ms"] and not k.startswith(("phase_", "step_"))), key=lambda kv: -kv[1])
    out = {"nodes": len(timed), "rows": rows, "ms": ms, "wall_ms": 1e3 * wall,
           "nodes_per_s": len(timed) / (ms * 1e-3), "rows_per_s": rows / (ms * 1e-3),
           "steps": ADAM_STEPS,
           "form": "one call over root nodes (row 0) of fresh properties; layers 2..R, lower and "
                   "upper sets per node",
           "breakdown_warmup_ms": {k: round(v, 3) for k, v in top[:5]}}
    if oracle_nodes > 0:
        from oracle import bab, core
        t_or, rows_or = 0.0, 0
        for pr in props[4:4 + oracle_nodes]:
            net_o, lo_t, hi_t, l, u, S, m, dense = bab.prepare(layers, pr.C, pr.d, pr.lo, pr.hi)
            node = bab.root_node(net_o, 0, l, u, S, None)
            t1 = time.perf_counter()
            rows_or += core.optimize_intermediate(net_o, node, lo_t, hi_t,
                                                  core.AdamHP(steps=ADAM_STEPS))
            t_or += time.perf_counter() - t1
        # the block's CPU baseline: the FP64 oracle, as it stands, on a few of the roots
        out["cpu_baseline"] = {"value": oracle_nodes / t_or, "unit": "nodes/s",
                               "rows": rows_or, "nodes": oracle_nodes,
                               "cores": torch.get_num_threads(), "kind": "oracle"}
    return out


# ----------------------------------------------------------------------------
# Conv-big (3x32x32, seven ReLU layers) with k = 3 multi-neuron constraints from
# the library's generator: gamma terms, their gradients and ACS branching run in
# the timed BaB steps (256 subproblems per step).
MNC_BIG = ("conv_big_32: 3x32x32 -> conv32 3x3 -> conv32 4x4 s2 -> conv64 3x3 -> conv64 4x4 s2 -> "
           "FC512 -> FC512 -> FC10, k=3 multi-neuron constraints (library generator)")


def mnc_big_run(local, stream, n_props, steps, max_groups, peaks, src, ksha, capacity=4096,
                batch=256):
    import torch
    from paper_2205_00263_gb300 import Context
    layers2 = synth.make_network(2)
    props = synth.make_properties(2, layers2, n=n_props, eps=synth.load_eps(2), start=0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ctx = Context(device=local, stream=stream.cuda_stream, node_capacity=capacity,
                  max_mnc_rows=VERDICT_MNC_ROWS, hbm_budget_bytes=64 << 30)
    try:
        net = ctx.load_network(layers2)
        ps, rows = [], []
        t0 = time.perf_counter()
        for pr in props:
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            ctx.set_budget(p, BUDGET)
            rows.append(ctx.generate_mnc(p, max_groups))
            ps.append(p)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        ctx.bab_step(ps, max_nodes=batch, steps=ADAM_STEPS)   # warm-up (roots)
        ctx.profile(True)
        ctx.bab_step(ps, max_nodes=batch, steps=ADAM_STEPS)   # every class timed: breakdown
        torch.cuda.synchronize()
        breakdown, _ = ctx.profile_read()
        dom_name = dominant(breakdown)[0]
        ctx.profile(True)
        ctx.profile_mask([dom_name])
        nodes, ms, rebound = 0, 0.0, 0
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ctx.bab_step(ps, max_nodes=batch, steps=ADAM_STEPS)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            nodes += st["nodes_bounded"]
            rebound += st["rows_rebounded"]
        stats, _ = ctx.profile_read()
        ctx.profile(False)
        ctx.profile_mask(None)
        # the same steps after the autotuner picked the affine-step kernels
        t0 = time.perf_counter()
        recs = ctx.autotune(net, max_rows=4096)
        tune_s = time.perf_counter() - t0
        t_nodes, t_ms = 0, 0.0
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = ctx.bab_step(ps, max_nodes=batch, steps=ADAM_STEPS)
            e1.record(stream)
            e1.synchronize()
            t_ms += e0.elapsed_time(e1)
            t_nodes += st["nodes_bounded"]
        choices = {}
        for r in recs:
            choices[r["variant"]] = choices.get(r["variant"], 0) + 1
        tuned = {"value": t_nodes / (t_ms * 1e-3) if t_ms else None, "unit": "nodes/s",
                 "steps": steps, "nodes": t_nodes, "ms_per_step": t_ms / max(1, steps),
                 "autotune_s": tune_s, "records": len(recs), "choices": choices,
                 "note": "the next BaB steps of the same run after mnbab_autotune (other nodes "
                         "than the built-in steps above)"}
        verd = {"verified": 0, "falsified": 0, "unknown": 0}
        for p in ps:
            v, _, _ = ctx.verdict(p)
            verd["verified" if v == 1 else "falsified" if v == -1 else "unknown"] += 1
    finally:
        ctx.close()
    top = sorted(((k, v["ms"]) for k, v in breakdown.items()
                  if v["ms"] and not k.startswith(("phase_", "step_"))), key=lambda kv: -kv[1])
    return {"workload": MNC_BIG, "properties": n_props, "max_groups_per_layer": max_groups,
            "subproblems_per_step": batch, "node_capacity": capacity,
            "mnc_rows_per_property": sum(rows) / len(rows),
            "generate_s_per_property": gen_s / n_props,
            "value": nodes / (ms * 1e-3) if ms else None, "unit": "nodes/s",
            "steps": steps, "nodes": nodes, "ms_per_step": ms / max(1, steps),
            "rows_rebounded": rebound,
            "roofline": roofline({dom_name: stats[dom_name]}, peaks, src, ksha),
            "kernel_breakdown_ms": {k: round(v, 3) for k, v in top[:8]},
            "autotuned": tuned,
            "state_after_timed_steps": verd,
            "note": "constraint generation is outside the timed steps"}


# ----------------------------------------------------------------------------
# Verdicts at the timeout: the full method (alpha / beta / gamma with k = 3
# multi-neuron constraints from the library's generator, ACS branching, FIFO
# BaB) on the networks of configs 0, 2 and 3.  Config 0 runs in the plain form
# (one property at a time, one subproblem per launch, <= 256 nodes per
# property); configs 2 and 3 run a rolling window of at most 16 properties in
# the batched form (256 / 128 subproblems per step; a finished property's
# place goes to the next), each property with its own wall-clock timeout from
# its first step.  The node pool bounds the BaB: the per-property node budget
# is what the pool holds for the properties that run together (a bounded node
# frees its slot after its two children take theirs, so a property never holds
# more than rows + 1 + budget slots, plus one per node of the running step).
VERDICT_MNC_ROWS = 160_000   # constraint rows a property may hold (configs 2 and 3)
VERDICT_CFGS = {
    0: dict(workload="fc_small_784: 784 -> 100 -> 100 -> 10, k=3 multi-neuron constraints",
            props=16, full_props=16, timeout=0.0, full_timeout=0.0, batch=1, budget=256,
            capacity=2048, mnc_rows=1 << 16, hbm=16 << 30, plain=True, attack=(8, 20)),
    2: dict(workload=None, props=8, full_props=100, timeout=20.0,
            full_timeout=60.0, batch=256, budget=None, capacity=32768, mnc_rows=None,
            hbm=200 << 30, plain=False, window=16, attack=(8, 20)),
    3: dict(workload="resnet_32: 3x32x32 -> conv16 3x3 -> 2 basic blocks (32, 64 ch, s2, 1x1 "
                     "shortcuts) -> FC100 -> FC10, k=3 multi-neuron constraints",
            props=8, full_props=50, timeout=20.0, full_timeout=120.0, batch=128, budget=None,
            capacity=32768, mnc_rows=None, hbm=200 << 30, plain=False, window=16, attack=(8, 20)),
}


def verdicts_run(local, stream, cfg, full=False, max_groups=2000):
    import torch
    from paper_2205_00263_gb300 import Context
    spec = dict(VERDICT_CFGS[cfg])
    if cfg == 2:
        spec["workload"] = MNC_BIG
    n_props = spec["full_props"] if full else spec["props"]
    timeout = spec["full_timeout"] if full else spec["timeout"]
    layers = synth.make_network(cfg)
    props = synth.make_properties(cfg, layers, n=n_props, eps=synth.load_eps(cfg), start=0)
    mnc_rows = spec["mnc_rows"] or VERDICT_MNC_ROWS
    ctx = Context(device=local, stream=stream.cuda_stream, node_capacity=spec["capacity"],
                  max_mnc_rows=mnc_rows, hbm_budget_bytes=spec["hbm"])
    try:
        net = ctx.load_network(layers)
        ps, rows = [], []
        t0 = time.perf_counter()
        for pr in props:
            p = ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d)
            if timeout:
                ctx.set_timeout(p, timeout)
            if spec["attack"]:
                ctx.set_attack(p, spec["attack"][0], spec["attack"][1], seed=len(ps))
            rows.append(ctx.generate_mnc(p, max_groups))
            ps.append(p)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        # node budget: what the pool holds for the properties that run together
        # (every property's root nodes exist from its constraint generation on)
        roots = sum(pr.C.shape[0] + 1 for pr in props)
        together = 1 if spec["plain"] else min(n_props, spec["window"])
        budget = (spec["capacity"] - 16 - roots - spec["batch"]) // together
        if budget < 1:
            raise RuntimeError("node pool too small for the properties' roots")
        if spec["budget"]:
            budget = min(budget, spec["budget"])
        for p in ps:
            ctx.set_budget(p, budget)
        ttv, nodes, steps = [], 0, 0
        t0 = time.perf_counter()
        if spec["plain"]:
            for p in ps:
                while True:
                    st = ctx.bab_step([p], max_nodes=1, steps=ADAM_STEPS)
                    nodes += st["nodes_bounded"]
                    steps += 1
                    if ctx.queue_size(p) == 0:
                        break
                ttv.append(ctx.status(p)[2])
        else:
            waiting = list(ps)
            active = [waiting.pop(0) for _ in range(min(together, len(waiting)))]
            while active:
                st = ctx.bab_step(active, max_nodes=spec["batch"], steps=ADAM_STEPS)
                nodes += st["nodes_bounded"]
                steps += 1
                keep = []
                for p in active:
                    if ctx.queue_size(p) == 0:
                        ttv.append(ctx.status(p)[2])
                    else:
                        keep.append(p)
                while waiting and len(keep) < together:
                    keep.append(waiting.pop(0))
                active = keep
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        verd = {"verified": 0, "falsified": 0, "unknown": 0, "of_which_timed_out": 0}
        for p in ps:
            v, _, _ = ctx.verdict(p)
            verd["verified" if v == 1 else "falsified" if v == -1 else "unknown"] += 1
            verd["of_which_timed_out"] += int(ctx.status(p)[1])
    finally:
        ctx.close()
    ttv = np.sort(np.asarray(ttv))
    return {"workload": spec["workload"], "properties": n_props,
            "form": ("plain: one property at a time, one subproblem per launch" if spec["plain"]
                     else f"batched: rolling window of {together} properties, "
                          f"{spec['batch']} subproblems per step"),
            "timeout_s": timeout or None, "node_budget_per_property": budget,
            "max_groups_per_layer": max_groups, "mnc_rows_per_property": float(np.mean(rows)),
            "generate_s_per_property": gen_s / n_props,
            "pre_attack": f"{spec['attack'][0]} starts x {spec['attack'][1]} sign steps",
            "verdicts": verd,
            "nodes": nodes, "bab_steps": steps, "wall_s": wall,
            "nodes_per_s": nodes / wall if wall else None,
            "time_to_verdict_s": {"p50": float(np.percentile(ttv, 50)),
                                  "p99": float(np.percentile(ttv, 99))},
            "sample": "full specified size" if full else "bounded sample (see properties, timeout_s)"}


# ----------------------------------------------------------------------------
def cpu_baseline(seconds: float, start: int = 0):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    BaB on seeded properties of the same net until ~`seconds` of CPU work."""
    import torch
    from oracle import bab, core
    layers = synth.make_network(CFG)
    eps = synth.load_eps(CFG)
    nodes, t = 0, 0.0
    k = start
    while t < seconds:
        pr = synth.make_properties(CFG, layers, n=1, eps=eps, start=k)[0]
        k += 1
        t0 = time.perf_counter()
        r = bab.verify(layers, pr.C, pr.d, pr.lo, pr.hi, max_nodes=12,
                       hp=core.AdamHP(steps=ADAM_STEPS))
        t += time.perf_counter() - t0
        nodes += r.n_bounded
    return {"value": nodes / t, "unit": "nodes/s", "cores": torch.get_num_threads(),
            "kind": "oracle", "_nodes": nodes, "_seconds": t,
            "sample": f"{k - start} properties of the same net and radius, first <=12 FIFO nodes "
                      f"each (root bounding, DeepPoly pass, 20 Adam steps, ACS), {nodes} nodes "
                      f"in {t:.1f} s"}


def run_reference(args):
    rank, world, local = dist_info()
    if rank != 0:
        return
    per = []
    total_nodes, total_t = 0, 0.0
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(max(1.0, args.cpu_seconds / max(1, args.steps)), start=100 * s)
        if s >= args.warmup:
            total_nodes += cb["_nodes"]
            total_t += cb["_seconds"]
            per.append(cb["_seconds"])
    value = total_nodes / total_t
    import torch
    out = {"metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * total_t / max(1, args.steps), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD}, "impl": "reference",
           "cpu_baseline": {"value": value, "unit": "nodes/s", "kind": "oracle",
                            "cores": torch.get_num_threads(),
                            "sample": "per step: seeded properties, first <=12 FIFO nodes each"},
           "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gemm_tc(args):
    """Root bounding of conv_big_32 properties with the FC back-substitution and
    forward products forced onto the tcgen05 kernel (3xTF32: operands split into
    TF32 hi and lo parts, three MMAs per K step, FP32 accumulation in TMEM).  The
    FC512 rows give products of 2,048 rows x 4,096 x 512.  Reports the summed
    CUDA-event time and algorithmic flops of those GEMM launches."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    stream = torch.cuda.Stream()
    layers = synth.make_network(2)
    eps = synth.load_eps(2)
    props = synth.make_properties(2, layers, n=4, eps=eps)
    out = {}
    for path, label in ((2, "tcgen05_3xtf32"), (1, "simt_fp32")):
        ctx = Context(device=0, stream=stream.cuda_stream, node_capacity=256, gemm_path=path)
        net = ctx.load_network(layers)
        ps = [ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d) for pr in props]
        ctx.root_bounds(ps[0], 1)  # warm-up: first property's root bounds
        ps = [ctx.set_property(net, pr.lo, pr.hi, pr.C, pr.d) for pr in props]
        ctx.profile(True)
        for p in ps:
            ctx.root_bounds(p, 1)
        stats, _ = ctx.profile_read()
        ctx.profile(False)
        g = stats["backsub_fc_gemm"]
        out[label] = {"launches": g["launches"], "ms": g["ms"], "gflop": g["flops"] / 1e9,
                      "tflops": g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] else None}
        ctx.close()
    peaks, src = load_peaks()
    if "tf32_tflops" not in peaks:
        peaks["tf32_tflops"] = measure_tf32()
        peaks["tf32_source"] = "measured in this run: cuBLAS TF32 GEMM 8192^3, best of 5"
    out["peak_3xtf32_tflops"], out["peak_source"] = tf32x3_peak(peaks, src)
    t = out["tcgen05_3xtf32"]["tflops"]
    out["frac_of_3xtf32"] = t / out["peak_3xtf32_tflops"] if t else None
    out["workload"] = ("conv_big_32 root bounding, 4 properties: FC back-substitution GEMMs "
                       "(rows of FC512 and FC512 neurons, both sides)")
    print(json.dumps(out), flush=True)


def run_mnc_big(args):
    """The conv_big_32 arm alone (multi-neuron constraints from the library's
    generator, alpha / beta / gamma, ACS), e.g. for profiling on a small pool."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    stream = torch.cuda.Stream()
    peaks, src = load_peaks()
    cap = args.mnc_big_capacity
    out = mnc_big_run(0, stream, args.mnc_big_props, args.mnc_big_steps, args.mnc_big_groups,
                      peaks, src, kernels_sha(), capacity=cap, batch=min(256, cap // 4))
    print(json.dumps({"conv_big_mnc": out}), flush=True)


def run_serving(args):
    """Config 4: Poisson stream (rate 4/s, 400 requests, seed 4) over the
    calibrated networks of configs 1-3, 60 s timeout, continuous batching."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_00263_gb300 import Context
    stream = torch.cuda.Stream()
    ctx = Context(device=0, stream=stream.cuda_stream, node_capacity=SERVE_CAPACITY,
                  hbm_budget_bytes=SERVE_HBM)
    out = serving_run(ctx, serving_nets(ctx), args.serve_requests or 400, args.serve_rate, seed=4,
                      timeout_s=60.0, budget=BUDGET, plain_cap_s=120.0, stream=stream)
    out["metric"] = METRIC
    out["workload"] = ("serving: Poisson stream of verification requests over the calibrated "
                       "networks of configs 1-3, 60 s timeout, 64 GB HBM budget")
    print(json.dumps(out), flush=True)
    ctx.close()


def run_verdicts_full(args):
    """Verdicts at the specified sizes: configs 0 (16 properties, plain form), 2
    (100 properties, 60 s timeout each) and 3 (50 properties, 120 s each), the
    batched configurations with all properties at once."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    stream = torch.cuda.Stream()
    out = {f"config{c}": verdicts_run(0, stream, int(c), full=True)
           for c in (args.verdicts or "0,2,3").split(",")}
    print(json.dumps({"verdicts_at_timeout": out}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.verdicts_full:
        run_verdicts_full(a)
    elif a.gemm_tc:
        run_gemm_tc(a)
    elif a.serving:
        run_serving(a)
    elif a.mnc_big_only:
        run_mnc_big(a)
    else:
        run_ours(a)
