#!/usr/bin/env python
"""Benchmark of the generalized 2D correlation hot path on GB300.

Default workload: homo correlation, m = 256 perturbation steps, n = 32768
spectral variables, FP16 hi/lo split precision (32768^2 complex outputs,
8.6 GB of Phi and Psi per step).  A step is one corr2d_compute call: the
tcgen05 DFT kernel (reference, centering, sigma, transform), then the tcgen05
cross-spectrum kernel.  Prints one JSON line (rank 0).  Its roofline is that of the
cross-spectrum kernel against HBM (the measured copy bandwidth), with the tensor
roofline (its tcgen05 flops against the measured BF16 peak) beside it; the one with
the larger fraction, the binding one, leads.

The default run also times the comparison forms the metric names, on the same
inputs, L2 flush and CUDA-event timing ("forms" in the JSON line): the plain
FP32 GPU path and BF16 operands on the same problem, the upper-triangle and the
BF16 output, and the batched form (512 problems of uneven m, n1, n2) against one
call per problem and against the FP32 path per problem.  Their errors against the FP64 oracle,
on sampled outputs, come from the CPU-baseline leg, the one place the oracle
runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c4|c2|c3|c5] [--precision split|bf16|fp32]

Under torchrun the homo workloads (c4, c2) are split over the ranks by output
tiles (corr2d_compute_part: each GPU a balanced, contiguous part of the
mirrored tile list, written into its own buffer; strong scaling, no data-path
collective): the value is the problem's outputs divided by the slowest rank's
time.  The batched workload (c5) is split by problem (corr2d_plan_batch_part: a
cost-balanced share of the 512 problems per GPU, each rank one corr2d_batch call;
strong scaling, no collective).  The other workloads run one independent problem
per rank (weak scaling): all ranks' outputs divided by the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D-corr output elems/s & % HBM roofline, split-prec vs FP32 at 1e-5 rel err"
UNIT = "output elems/s"
L2_FLUSH_BYTES = 256 << 20
TOL = {"split": 1e-5, "fp32": 1e-5, "bf16": 1e-2}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c4", "c2", "c3", "c5"], default="c4")
    ap.add_argument("--precision", choices=["split", "bf16", "fp32"], default="split")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the comparison forms (FP32, BF16, upper triangle, batch)")
    ap.add_argument("--no-batch", action="store_true",
                    help="c5 only: one corr2d_compute call per problem instead of corr2d_batch")
    ap.add_argument("--upper-triangle", action="store_true",
                    help="homo workloads: store only the upper triangle (half the outputs)")
    ap.add_argument("--output-bf16", action="store_true",
                    help="c4/c2: store Phi and Psi as BF16 (half the output bytes)")
    ap.add_argument("--l2", choices=["clean", "dirty"], default="clean",
                    help="L2 flush before every step: write a 256 MB buffer, then (clean) read "
                         "another so that the flush's dirty lines are written back before the "
                         "step, or (dirty) leave them in L2")
    ap.add_argument("--n", type=int, default=0,
                    help="small profiling cases: c4 keeps the first N spectral variables, "
                         "c5 gives every stack N variables (same m mix)")
    ap.add_argument("--cpu-sample-n", type=int, default=0,
                    help="spectral variables of the oracle sample (0: sized to ~10-30 s)")
    return ap.parse_args()


# ---------------------------------------------------------------- workloads
def workload(name, precision, n_override=0):
    """(description dict, inputs) for a workload name."""
    import workloads as wl
    if name == "c4":
        y = wl.c4()
        if n_override and n_override < y.shape[1]:
            y = y[:, :n_override].copy()
        n = y.shape[1]
        return dict(workload=f"homo m=256 n={n} {precision}", m=256, n1=n, n2=n,
                    homo=True, alpha=0.0, precision=precision), (y, None)
    if name == "c2":
        y = wl.c2()
        return dict(workload=f"homo m=64 n=4096 {precision}", m=64, n1=4096, n2=4096, homo=True,
                    alpha=0.0, precision=precision), (y, None)
    if name == "c3":
        raw = wl.c3()
        return dict(workload=f"hetero m=128 n1=8192 n2=2048 alpha=0.5 {precision} "
                             f"(with preprocessing)", m=128, n1=8192, n2=2048, homo=False,
                    alpha=0.5, precision=precision), raw
    if n_override:
        spec = wl.c5_spec(n_fixed=n_override)
        return dict(workload=f"batched 512 problems m~U[8,200] every n={n_override} {precision}",
                    problems=len(spec.problems), outputs=spec.total_outputs,
                    precision=precision, alpha=0.0), spec
    spec = wl.c5_spec()
    return dict(workload=f"batched 512 problems m~U[8,200] n log-uniform [256,8192] {precision}",
                problems=len(spec.problems), outputs=spec.total_outputs, precision=precision,
                alpha=0.0), spec


def l2_text(mode):
    if mode == "clean":
        return ("flushed before every timed step outside the step's events: a 256 MB write, "
                "then a 256 MB read of another buffer, so that L2 holds no dirty lines of the "
                "flush when the step starts; each step writes >= 134 MB of output")
    return ("flushed before every timed step (256 MB write outside the step's events); each "
            "step writes >= 134 MB of output")


def config_for(desc, world, l2_mode, parallelism=None):
    return {**desc, "l2": l2_text(l2_mode),
            "parallelism": parallelism or f"weak: one independent problem per GPU x{world}"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region (log in a temp file)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"corr2d_clocks_gpu{gpu_index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            self._remove()
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        self._remove()
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}

    def _remove(self):
        try:
            os.unlink(self.path)
        except OSError:
            pass


# ---------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_tensor_peak():
    """Dense BF16 tensor throughput (TFLOP/s) of MEASURED_PEAKS.json, the burst figure;
    the split products are FP16 MMAs, whose nominal dense rate equals BF16's."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (bf16 burst)"
    return 1900.0, "fallback"


def tensor_flops(m, precision, pairs):
    """Tensor-core flops of the cross-spectrum over `pairs` output pairs: 8 K' per pair (the
    two real dot products of length 2 K'), three products each for the FP16 hi/lo split."""
    kp = (m - 1) // 2 + 1
    return 8.0 * kp * pairs * (3 if precision == "split" else 1)


def with_tensor_bound(hbm, flops, ms):
    """The HBM roofline `hbm` and the tensor one (flops per launch over `ms`): the binding
    bound (the larger fraction) leads, the other is kept under its own name."""
    peak, kind = measured_tensor_peak()
    ach = flops / (ms / 1e3) / 1e12
    ten = {"bound": "tensor", "achieved": round(ach, 1), "peak": peak, "unit": "TFLOP/s",
           "frac": round(ach / peak, 4), "peak_kind": kind, "algorithmic_flops_per_launch": flops}
    if ten["frac"] <= hbm["frac"]:
        return dict(hbm, tensor=ten)
    other = {k: v for k, v in hbm.items() if k not in ("traffic",)}
    return dict(ten, traffic=hbm.get("traffic"), hbm=other)


def xspec_traffic_per_launch(workload_name, precision, kernel="k_xspec_tc"):
    """DRAM bytes of one cross-spectrum launch from the committed ncu summary, if that
    summary was taken on the current kernel source (same sha256), else None."""
    src_name = {"k_xspec_pair": "k_xspec_pair.cu", "k_xspec_ta": "k_xspec_ta.cu"}.get(kernel,
                                                                                   "k_xspec.cu")
    src = os.path.join(ROOT, "paper_1808_00685_gb300", "csrc", src_name)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    tag = {"k_xspec_pair": "xspec_pair", "k_xspec_ta": "xspec_ta"}.get(kernel, "xspec")
    summ = os.path.join(ROOT, "profiles", f"{tag}_{workload_name}_{precision}.md")
    if not os.path.exists(summ):
        return None
    text = open(summ).read()
    m_sha = re.search(re.escape(src_name) + r" sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram bytes per full launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


def store_stream_gbs(device, gib=2, reps=5):
    """Write-only bandwidth of this GPU, measured live: a torch fill of a buffer far
    larger than L2 (a store-bound kernel can approach this, a copy-based peak is lower)."""
    import torch
    buf = torch.empty(gib << 28, dtype=torch.float32, device=device)
    for _ in range(2):
        buf.fill_(1.5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        buf.fill_(1.5)
    e1.record()
    torch.cuda.synchronize()
    gbs = buf.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
    del buf
    return round(gbs, 1)


def store_stream_same_size_gbs(device, nbytes, flush, reps=5):
    """Write-only bandwidth of a plain store stream of `nbytes` (a torch fill),
    each run after the same L2 flush as the timed steps: the ceiling a store-bound
    kernel of that output size can reach.  Near the L2 size (c2, c3: 134 MB) the
    first part of the stream is absorbed by L2 and the rest waits for write-back,
    so this is far below the large-buffer stream."""
    import torch
    buf = torch.empty(max(int(nbytes) // 4, 1), dtype=torch.float32, device=device)
    best = 1e30
    for k in range(reps + 1):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        buf.fill_(1.5)
        e1.record()
        e1.synchronize()
        if k > 0:
            best = min(best, e0.elapsed_time(e1))
    del buf
    return round(nbytes / (best / 1e3) / 1e9, 1)


def rowlen_elems(m, precision):
    planes = 2 if precision == "split" else 1
    g = 16 if planes == 2 else 32
    kp = ((m - 1) // 2 + 1 + g - 1) // g * g
    return kp // g * 64


def batch_bytes(spec, precision):
    """Algorithmic bytes of one cross-spectrum launch over a batch: Phi and Psi stored
    (8 B per output pair) and every problem's operand rows read once (n1 rows for a
    homo problem, whose two operands are one row set; n1 + n2 for a hetero one),
    the definition used for the single-problem workloads."""
    out = 0.0
    for p in spec.problems:
        rows = p.n1 if p.homo else p.n1 + p.n2
        out += 8.0 * p.n1 * p.n2 + 2.0 * rows * rowlen_elems(p.m, precision)
    return out


def gpu_numa_cpus(device_index):
    """(NUMA node, CPU list) of the host node the GPU hangs off, from sysfs; (None, None)
    where that is not known."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device_index)
        path = (f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:"
                f"{p.pci_device_id:02x}.0/numa_node")
        node = int(open(path).read().strip())
        if node < 0:
            return None, None
        text = open(f"/sys/devices/system/node/node{node}/cpulist").read().strip()
        cpus = set()
        for part in text.split(","):
            a, _, b = part.partition("-")
            cpus |= set(range(int(a), int(b or a) + 1))
        cpus &= set(os.sched_getaffinity(0))
        return node, (sorted(cpus) or None)
    except (OSError, ValueError, AttributeError, RuntimeError):
        return None, None


def link_bandwidth(h, d, stream, reps=3):
    """Best-of-reps pinned host<->device copy bandwidth (GB/s) of 1 GiB each way,
    with the buffers the end-to-end run uses."""
    import torch
    nb = min(1 << 30, h.numel() * h.element_size(), d.numel() * d.element_size())
    hb = h.view(-1).view(torch.uint8)[:nb]
    db = d.view(-1).view(torch.uint8)[:nb]
    res = {}
    with torch.cuda.stream(stream):
        for name, (dst, src) in (("h2d_gbs", (db, hb)), ("d2h_gbs", (hb, db))):
            dst.copy_(src, non_blocking=True)
            stream.synchronize()
            best = 1e30
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dst.copy_(src, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            res[name] = round(nb / (best / 1e3) / 1e9, 1)
    return res


def output_copy_ms(phi_h, psi_h, phi, psi, n, rows=1024):
    """Host time (ms) of copying both output maps device -> host the way the host-buffer
    entry point does: row slabs, Phi and Psi on two streams, into the same pinned buffers."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r0 in range(0, n, rows):
        with torch.cuda.stream(s1):
            phi_h[r0:r0 + rows].copy_(phi[r0:r0 + rows, :n], non_blocking=True)
        with torch.cuda.stream(s2):
            psi_h[r0:r0 + rows].copy_(psi[r0:r0 + rows, :n], non_blocking=True)
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, value, device):
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ---------------------------------------------------------------- timing
class Flusher:
    """L2 flush between steps: write a 256 MB buffer; in the clean mode also read a
    second one, so that the flush's dirty lines are written back before the step."""

    def __init__(self, device, mode):
        import torch
        self.mode = mode
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
        self.r = (torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
                  if mode == "clean" else None)

    def __call__(self):
        self.w.zero_()
        if self.r is not None:
            self.r.max()


def timed_steps(ctx, stream, step, flush, steps, warmup, per_call_timing=True):
    """Warm-up steps exactly like the timed ones, then `steps` timed steps, each
    bracketed by CUDA events on the stream the library launches on.  The timed steps
    carry no per-launch events: an event between the DFT and cross-spectrum launches
    costs several microseconds per step and serialises the two (the cross-spectrum
    launch would otherwise overlap the DFT's tail).  With `per_call_timing`, every
    timed step is followed by one more step of the same work, outside the timed
    events, in which the library records events around its two launches; those give
    the prep and cross-spectrum kernel times under the same clocks and power state as
    the timed steps beside them.  Returns the timed steps' times (ms), the kernel
    times and the profiled steps' times."""
    import torch

    def timed_step():
        flush()  # outside the step's events
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        return a, b

    def profiled_step():
        ctx.set_profiling(True)
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        p_ms, x_ms = ctx.timings()  # waits for this step's kernel events
        ctx.set_profiling(False)
        return a, b, p_ms, x_ms

    ctx.set_profiling(False)
    for _ in range(max(warmup, 0)):
        timed_step()
        if per_call_timing:
            profiled_step()
    torch.cuda.synchronize()
    ctx.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    ev, pev, prep_ms, xspec_ms = [], [], [], []
    for _ in range(steps):
        ev.append(timed_step())
        if per_call_timing:
            a, b, p_ms, x_ms = profiled_step()
            pev.append((a, b))
            prep_ms.append(p_ms)
            xspec_ms.append(x_ms)
    r1.record(stream)
    torch.cuda.synchronize()
    ctx.synchronize()  # raises on a device-side time-out
    return dict(step_ms=[a.elapsed_time(b) for a, b in ev], prep_ms=prep_ms, xspec_ms=xspec_ms,
                region_ms=r0.elapsed_time(r1),
                profiled_step_ms=[a.elapsed_time(b) for a, b in pev])


def sample_block(n, upper=False):
    """Sampled rows x columns of an n x n map where the errors are taken (first and
    last indices included).  For an upper-triangle output the rows come from the
    first half and the columns from the second, so that every entry has nu2 > nu1."""
    import workloads as wl
    if not upper:
        return wl.sample_rows(n, 256, seed=41), wl.sample_rows(n, 256, seed=42)
    h = n // 2
    return wl.sample_rows(h, 128, seed=43), h + wl.sample_rows(n - h, 128, seed=44)


def gather(phi, psi, rows, cols):
    """Phi/Psi at rows x cols, to host FP64 (numpy)."""
    import numpy as np
    import torch
    rt = torch.from_numpy(np.asarray(rows, np.int64)).to(phi.device)
    ct = torch.from_numpy(np.asarray(cols, np.int64)).to(phi.device)
    return (phi.index_select(0, rt).index_select(1, ct).double().cpu().numpy(),
            psi.index_select(0, rt).index_select(1, ct).double().cpu().numpy())


def error_of(got, want):
    """Relative Frobenius and max-abs errors of Phi and Psi against the oracle."""
    import numpy as np
    (gp, gq), (op, oq) = got, want
    big = max(float(np.abs(op).max()), float(np.abs(oq).max()), 1e-300)
    return {"rel_err_phi": float(np.linalg.norm(gp - op) / max(np.linalg.norm(op), 1e-300)),
            "rel_err_psi": float(np.linalg.norm(gq - oq) / max(np.linalg.norm(oq), 1e-300)),
            "max_abs_phi": float(np.abs(gp - op).max()), "max_abs_psi": float(np.abs(gq - oq).max()),
            "largest_magnitude": big}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(y, n_sample=0, alpha=0.0, target_s=15.0, single=False):
    """The FP64 oracle as it stands, all host threads, on the first n_sample
    spectral variables of the same stack (homo), and on one thread on a smaller
    sample (info["single_thread"]).  Returns (elems/s, info)."""
    import oracle
    threads = oracle.max_threads()
    m = y.shape[0]
    if n_sample <= 0:
        # the oracle costs a n (its DFT) + b n^2 (the correlation): calibrate
        # on two small samples, then size the measured run to ~target_s
        ts = []
        for n0 in (256, 1024):
            t0 = time.perf_counter()
            oracle.corr2d(y[:, :n0].copy(), alpha=alpha, nthreads=threads)
            ts.append(max(time.perf_counter() - t0, 1e-4))
        b = max((ts[1] / 1024 - ts[0] / 256) / (1024 - 256), 1e-15)
        a = max(ts[0] / 256 - b * 256, 0.0)
        n_est = (-a + math.sqrt(a * a + 4 * b * target_s)) / (2 * b)
        n_sample = int(min(y.shape[1], max(256, n_est)))
    ys = y[:, :n_sample].copy()
    t0 = time.perf_counter()
    oracle.corr2d(ys, alpha=alpha, nthreads=threads)
    dt = time.perf_counter() - t0
    info = dict(kind="oracle", cores=threads,
                sample=f"homo m={m}, first {n_sample} spectral variables of the same stack "
                       f"({n_sample * n_sample} outputs, {dt:.1f} s)", seconds=dt)
    if single:
        # one host thread too, on a sample sized for ~4 s (the cost grows as n^2)
        n1 = int(max(128, n_sample * math.sqrt(4.0 / max(dt, 1e-3)) / math.sqrt(threads)))
        n1 = min(n1, n_sample)
        t1 = time.perf_counter()
        oracle.corr2d(y[:, :n1].copy(), alpha=alpha, nthreads=1)
        dt1 = time.perf_counter() - t1
        info["single_thread"] = {"value": n1 * n1 / dt1, "cores": 1,
                                 "sample": f"homo m={m}, first {n1} spectral variables "
                                           f"({n1 * n1} outputs, {dt1:.1f} s)"}
    return n_sample * n_sample / dt, info


def oracle_at(y1, y2, rows, cols, alpha=0.0):
    """The oracle's Phi/Psi at rows x cols.  Reference, centering, sigma and DFT act on
    one spectral variable at a time, so correlating the sampled columns of the stacks
    gives exactly those entries (the oracle pin test_sampled_columns_give_those_entries)."""
    import numpy as np
    import oracle
    ys2 = y1 if y2 is None else y2
    phi, psi, _, _ = oracle.corr2d(np.ascontiguousarray(y1[:, rows]),
                                   np.ascontiguousarray(ys2[:, cols]), alpha=alpha,
                                   nthreads=oracle.max_threads())
    return phi, psi


def cpu_baseline_leg(args, y, alpha, checks):
    """The one place the oracle runs: its timing on a bounded sample of the workload
    (the CPU baseline) and its values at the sampled outputs of every timed form
    (checks: name -> (y1, y2, rows, cols, alpha, gpu values)), from which the forms'
    errors are computed.  Returns (cpu_baseline dict or None, errors by form)."""
    cpu = None
    if y is not None and not args.no_cpu_baseline:
        rate, info = cpu_oracle_rate(y, args.cpu_sample_n, alpha, single=True)
        cpu = {"value": rate, "unit": UNIT, **{k: v for k, v in info.items() if k != "seconds"}}
    errors = {}
    t0 = time.perf_counter()
    for name, entries in checks.items():
        worst = None
        for (y1, y2, rows, cols, a, got) in entries:
            e = error_of(got, oracle_at(y1, y2, rows, cols, a))
            if worst is None:
                worst = e
            else:  # worst problem of a batch, by relative error
                for k in e:
                    worst[k] = max(worst[k], e[k])
        if worst is not None:
            worst["sampled"] = (f"{len(entries)} problem(s), "
                                f"{sum(len(r) * len(c) for (_, _, r, c, _, _) in entries)} outputs")
            errors[name] = worst
    if cpu is not None and checks:
        cpu["checks_s"] = round(time.perf_counter() - t0, 2)
    return cpu, errors


# ---------------------------------------------------------------- forms
def run_forms(args, ctx, stream, flush, y, yd, phi, psi, ldo, rows, cols, checks):
    """Comparison forms of the metric on the same inputs, flush and timing: c4 in FP32,
    with BF16 operands, upper-triangle output and BF16 output; the batch of 512 problems
    batched, per problem and per problem in FP32.  Sampled GPU outputs go into `checks`."""
    import torch
    import paper_1808_00685_gb300 as pkg
    import workloads as wl
    forms = {}
    m, n = y.shape
    peak_fp32 = ctx.fp32_peak_tflops()
    peak, _ = measured_peaks()

    def c4_form(name, out=None, **kw):
        o = out or (phi, psi)

        def step():
            ctx.compute(yd, out=o, **kw)
        t = timed_steps(ctx, stream, step, flush, args.steps, args.warmup)
        ms = statistics.mean(t["step_ms"])
        xms = statistics.mean(t["xspec_ms"])
        upper = kw.get("upper_triangle", False)
        outs = n * (n + 1) / 2 if upper else n * n
        d = {"workload": f"homo m={m} n={n} {kw.get('precision', 'split')}"
                         + (" upper triangle" if upper else "")
                         + (" BF16 output" if kw.get("output_bf16") else ""),
             "ms_per_step": round(ms, 4), "value": n * n / (ms / 1e3),
             "kernel_ms": round(xms, 4), "prep_ms": round(statistics.mean(t["prep_ms"]), 4),
             "steps": args.steps}
        prec = kw.get("precision", "split")
        if prec == "fp32":
            kp1 = (m - 1) // 2 + 1
            ach = 8.0 * kp1 * (n * (n + 1) / 2) / (xms / 1e3) / 1e12  # unique pairs of a homo map
            d["roofline"] = {"bound": "alu", "achieved": round(ach, 2), "peak": round(peak_fp32, 1),
                             "unit": "TFLOP/s", "frac": round(ach / peak_fp32, 4),
                             "peak_kind": "measured: FP32 FMA probe kernel (corr2d_measure_fp32_peak)"}
        else:
            xb = (4.0 if kw.get("output_bf16") else 8.0) * outs + 1.0 * n * rowlen_elems(m, prec) * 2
            ach = xb / (xms / 1e3) / 1e9
            d["roofline"] = with_tensor_bound(
                {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                 "frac": round(ach / peak, 4), "algorithmic_bytes_per_launch": xb},
                tensor_flops(m, prec, n * (n + 1) / 2), xms)
        r, c = sample_block(n, upper)
        checks[name] = [(y, None, r, c, 0.0, gather(o[0], o[1], r, c))]
        return d

    forms["fp32"] = c4_form("fp32", precision="fp32")
    forms["bf16"] = c4_form("bf16", precision="bf16")
    forms["upper_triangle"] = c4_form("upper_triangle", precision="split", upper_triangle=True)
    # Phi and Psi stored as BF16 (the FP32 values rounded to nearest): half the output bytes
    b16 = pkg.Context.alloc_out(n, n, yd.device, bf16=True)[:2]
    forms["bf16_output"] = c4_form("bf16_output", out=b16, precision="split", output_bf16=True)
    del b16

    # the batched form: 512 problems, m ~ U{8..200}, n log-uniform [256, 8192]
    spec = wl.c5_spec()
    ins = wl.batch_inputs(spec)
    probs = []
    for (y1, y2), p in zip(ins, spec.problems):
        d1 = torch.from_numpy(y1).to(yd.device)
        d2 = None if y2 is None else torch.from_numpy(y2).to(yd.device)
        ph, ps, _ = pkg.Context.alloc_out(p.n1, p.n2, yd.device)
        probs.append((d1, d2, ph, ps))
    outputs = spec.total_outputs
    samp = [(wl.sample_rows(p.n1, 4, seed=9000 + i), wl.sample_rows(p.n2, 48, seed=19000 + i))
            for i, p in enumerate(spec.problems)]

    def c5_checks():
        out = []
        for (y1, y2), (_, _, ph, ps), (r, c) in zip(ins, probs, samp):
            out.append((y1, y2, r, c, 0.0, gather(ph, ps, r, c)))
        return out

    def c5_form(name, step, per_call):
        t = timed_steps(ctx, stream, step, flush, args.steps, args.warmup, per_call)
        ms = statistics.mean(t["step_ms"])
        d = {"workload": f"batched {len(probs)} problems m~U[8,200] n log-uniform [256,8192] "
                         + name, "ms_per_step": round(ms, 4), "value": outputs / (ms / 1e3),
             "steps": args.steps}
        if per_call:
            xms = statistics.mean(t["xspec_ms"])
            d["kernel_ms"] = round(xms, 4)
            d["prep_ms"] = round(statistics.mean(t["prep_ms"]), 4)
            xb = batch_bytes(spec, "split")
            ach = xb / (xms / 1e3) / 1e9
            fl = sum(tensor_flops(p.m, "split", p.n1 * (p.n1 + 1) / 2 if p.homo else p.n1 * p.n2)
                     for p in spec.problems)
            d["roofline"] = with_tensor_bound(
                {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                 "frac": round(ach / peak, 4), "algorithmic_bytes_per_launch": xb}, fl, xms)
        checks[name] = c5_checks()
        return d

    plan = ctx.batch_plan(probs, precision="split")
    forms["c5_batch"] = c5_form("c5_batch", plan.run, True)

    def per_problem(prec):
        def step():
            for d1, d2, ph, ps in probs:
                ctx.compute(d1, d2, precision=prec, out=(ph, ps))
        return step
    forms["c5_per_problem"] = c5_form("c5_per_problem", per_problem("split"), False)
    forms["c5_fp32_per_problem"] = c5_form("c5_fp32_per_problem", per_problem("fp32"), False)
    del probs, plan
    torch.cuda.empty_cache()
    return forms, peak_fp32


# ---------------------------------------------------------------- our arm
def run_ours(args, world, rank, local, pg):
    import numpy as np
    import torch

    import paper_1808_00685_gb300 as pkg
    import workloads as wl

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    desc, inputs = workload(args.workload, args.precision, args.n)
    ctx = pkg.Context(local, stream)
    flush = Flusher(device, args.l2)
    launches_per_step = 2
    per_call_timing = True  # the step is one library call: its kernel events time it
    upper = args.upper_triangle and args.workload in ("c4", "c2")
    obf = args.output_bf16 and args.workload in ("c4", "c2") and args.precision != "fp32"
    strong = world > 1 and args.workload in ("c4", "c2") and args.precision != "fp32"
    scaling, parallelism = "weak", None

    if args.workload in ("c4", "c2"):
        y, _ = inputs
        yd = torch.from_numpy(y).to(device)
        m, n = y.shape
        phi, psi, ldo = pkg.Context.alloc_out(n, n, device, bf16=obf)
        outputs = n * n
        # Phi and Psi stored (the upper triangle only: n (n + 1) / 2 pairs), the homo
        # problem's one operand row set read once
        stored = n * (n + 1) / 2 if upper else n * n
        pairs = n * (n + 1) / 2  # the unique pairs of a homo map: the tensor-core work
        if strong:
            # this rank's part of the mirrored tile list: its blocks and mirrored blocks
            tiles = pkg.corr2d_plan_part(n, n, True, 0, rank, world)
            stored = pairs = 0.0
            for ti, tj in tiles:
                h = min(128, n - 128 * ti)
                area = h * min(128, n - 128 * tj)
                stored += area * (1 if (upper or ti == tj) else 2)
                pairs += h * (h + 1) / 2 if ti == tj else area
            scaling = "strong"
            parallelism = (f"strong: one problem split by output tiles over {world} GPUs "
                           f"(corr2d_compute_part, balanced parts of the mirrored tile list; "
                           f"this rank {len(tiles)} tiles), no collective")

            def step():
                ctx.compute_part(yd, None, rank, world, precision=args.precision,
                                 upper_triangle=upper, out=(phi, psi), output_bf16=obf)
        else:
            def step():
                ctx.compute(yd, precision=args.precision, out=(phi, psi), upper_triangle=upper,
                            output_bf16=obf)
        xbytes = (4.0 if obf else 8.0) * stored + 1.0 * n * rowlen_elems(m, args.precision) * 2
        tflops = tensor_flops(m, args.precision, pairs)
        if upper:
            desc["workload"] += " upper triangle"
            desc["upper_triangle"] = True
        if obf:
            desc["workload"] += " BF16 output"
            desc["output_bf16"] = True
    elif args.workload == "c3":
        raw = inputs
        x1, y1r = torch.from_numpy(raw.x1).to(device), torch.from_numpy(raw.y1).to(device)
        x2, y2r = torch.from_numpy(raw.x2).to(device), torch.from_numpy(raw.y2).to(device)
        n1, n2 = raw.n1_out, raw.n2_out
        phi, psi, ldo = pkg.Context.alloc_out(n1, n2, device)
        outputs = n1 * n2

        def step():
            a, _ = ctx.preprocess(x1, y1r, n1)
            b, _ = ctx.preprocess(x2, y2r, n2)
            ctx.compute(a, b, precision=args.precision, alpha=raw.alpha, out=(phi, psi))
        launches_per_step = 4  # 2 x resampling (axis check inside), DFT, cross-spectrum
        xbytes = 8.0 * n1 * n2 + 2.0 * (n1 + n2) * rowlen_elems(128, args.precision)
        tflops = tensor_flops(128, args.precision, n1 * n2)
        y = raw.y1
    else:
        spec = inputs
        outputs = spec.total_outputs
        if world > 1 and not (args.no_batch or args.precision == "fp32"):
            # one batch over several GPUs: each rank runs corr2d_batch on its cost-balanced
            # share of the problems (strong scaling, no data-path collective)
            shapes = [(p.m, p.n1, p.n2, p.homo) for p in spec.problems]
            sel = pkg.plan_batch_part(shapes, rank, world)
            if not sel:
                raise SystemExit(f"rank {rank} of {world}: no problems in its part")
            strong = True
            scaling = "strong"
            parallelism = (f"strong: the batch split by problem over {world} GPUs "
                           f"(corr2d_plan_batch_part, cost-balanced; this rank {len(sel)} of "
                           f"{len(spec.problems)} problems), no collective")
            spec = wl.BatchSpec(problems=[spec.problems[i] for i in sel])
        ins = wl.batch_inputs(spec)
        probs = []
        for (y1, y2), p in zip(ins, spec.problems):
            d1 = torch.from_numpy(y1).to(device)
            d2 = None if y2 is None else torch.from_numpy(y2).to(device)
            ph, ps, _ = pkg.Context.alloc_out(p.n1, p.n2, device)
            probs.append((d1, d2, ph, ps))
        if args.no_batch or args.precision == "fp32":
            # one library call per problem (the FP32 path has no batched form)
            launches_per_step = sum(2 if y2 is None else 3 if args.precision == "fp32" else 2
                                    for (_, y2), _p in zip(ins, spec.problems))
            per_call_timing = False

            def step():
                for d1, d2, ph, ps in probs:
                    ctx.compute(d1, d2, precision=args.precision, out=(ph, ps))
        else:
            plan = ctx.batch_plan(probs, precision=args.precision)

            def step():
                plan.run()
        xbytes = batch_bytes(spec, args.precision)
        tflops = sum(tensor_flops(p.m, args.precision,
                                  p.n1 * (p.n1 + 1) / 2 if p.homo else p.n1 * p.n2)
                     for p in spec.problems)
        desc["batched"] = not (args.no_batch or args.precision == "fp32")
        y = None

    # The clock sampler starts (and settles) before the warm-up, so that the GPU
    # is not left idle between the warm-up and the timed steps.
    sampler = ClockSampler(local)
    sampler.start()
    try:
        barrier(pg)
        t = timed_steps(ctx, stream, step, flush, args.steps, args.warmup, per_call_timing)
        barrier(pg)
    except BaseException:
        sampler.stop()  # no nvidia-smi left running
        raise
    clocks = sampler.stop()
    kind, pair_clusters = ctx.kernel_info()
    kernel = {pkg.XSPEC_TC: "k_xspec_tc", pkg.XSPEC_TC_PAIR: "k_xspec_pair",
              pkg.XSPEC_TC_TA: "k_xspec_ta", pkg.XSPEC_FP32: "k_xspec_simt"}.get(kind, "none")
    ms = statistics.mean(t["step_ms"])
    ms_max = reduce_max(pg, ms, device)
    value = (1 if strong else world) * outputs / (ms_max / 1e3)

    peak, peak_kind = measured_peaks()
    # several calls per step: the per-kernel events cover the last call only,
    # so the whole step time stands in for the kernel time
    x_mean = statistics.mean(t["xspec_ms"]) if per_call_timing else ms
    achieved = xbytes / (x_mean / 1e3) / 1e9
    # the committed capture is of a whole launch with FP32 outputs: a rank's part, the
    # upper triangle and BF16 outputs are other launches
    traffic = (None if (strong or upper or obf)
               else xspec_traffic_per_launch(args.workload, args.precision, kernel))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kernel,
                "grid": (f"{pair_clusters} CTA pairs" if kernel == "k_xspec_pair" else None),
                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": xbytes,
                "kernel_ms": round(x_mean, 4),
                "prep_ms": round(statistics.mean(t["prep_ms"]), 4) if t["prep_ms"] else None,
                "kernel_timing": ("per-launch CUDA events in a profiled step of the same "
                                  "work after each timed step, outside its events"
                                  if per_call_timing else
                                  "whole step (several launches per step)"),
                "profiled_ms_per_step": (round(statistics.mean(t["profiled_step_ms"]), 4)
                                         if t["profiled_step_ms"] else None)}
    if args.precision != "fp32":
        # second denominator: the write-only stream (measured after the timed region)
        st = store_stream_gbs(device)
        roofline.update({"store_stream_gbs": st, "frac_of_store_stream": round(achieved / st, 4)})
        if outputs * 8 < (2 << 30):
            # output near the L2 size: the same-size store stream is the fair ceiling
            ss = store_stream_same_size_gbs(device, 8.0 * outputs, flush)
            roofline.update({"store_stream_same_size_gbs": ss,
                             "frac_of_same_size_store_stream": round(achieved / ss, 4)})
        # the tensor roofline beside it; where it binds (the upper triangle: half the stores
        # for the same products) it leads and the HBM figures move under "hbm"
        tpeak, tkind = measured_tensor_peak()
        tach = tflops / (x_mean / 1e3) / 1e12
        ten = {"bound": "tensor", "achieved": round(tach, 1), "peak": tpeak, "unit": "TFLOP/s",
               "frac": round(tach / tpeak, 4), "peak_kind": tkind,
               "algorithmic_flops_per_launch": tflops}
        if ten["frac"] > roofline["frac"]:
            moved = ("bound", "achieved", "peak", "unit", "frac", "peak_kind",
                     "algorithmic_bytes_per_launch", "store_stream_gbs", "frac_of_store_stream",
                     "store_stream_same_size_gbs", "frac_of_same_size_store_stream")
            roofline["hbm"] = {k: roofline.pop(k) for k in moved if k in roofline}
            roofline.update(ten)
        else:
            roofline["tensor"] = ten
    if args.precision == "fp32":
        fp32_peak = ctx.fp32_peak_tflops()
        kp1 = (desc.get("m", 2) - 1) // 2 + 1
        n_ = desc.get("n1", 0)
        # 8 flops per output and frequency, unique outputs of a homo problem
        flops = 8.0 * kp1 * (n_ * (n_ + 1) / 2 if desc.get("homo") else outputs)
        ach = flops / (x_mean / 1e3) / 1e12
        roofline.update({"bound": "alu", "achieved": round(ach, 2), "peak": round(fp32_peak, 1),
                         "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                         "peak_kind": "measured: FP32 FMA probe kernel (corr2d_measure_fp32_peak)"})

    # sampled outputs of the main run, for its error against the oracle
    checks = {}
    rows = cols = None
    if args.workload in ("c4", "c2") and rank == 0 and not strong:
        rows, cols = sample_block(n, upper)
        checks["main"] = [(y, None, rows, cols, 0.0, gather(phi, psi, rows, cols))]

    forms = None
    if (not args.no_forms and args.workload == "c4" and args.precision == "split" and not upper
            and not obf and world == 1 and not args.n):
        sampler2 = ClockSampler(local)
        sampler2.start()
        try:
            forms, _ = run_forms(args, ctx, stream, flush, y, yd, phi, psi, ldo, rows, cols,
                                 checks)
        finally:
            forms_clocks = sampler2.stop()
        forms["clocks"] = forms_clocks

    # end to end through the host-buffer entry point (pinned host memory placed on
    # the GPU's NUMA node when sysfs names it)
    e2e = None
    if not args.no_e2e and args.workload in ("c4", "c2") and not strong:
        node, cpus = gpu_numa_cpus(local)
        saved = os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
        try:
            y_h = torch.from_numpy(y).pin_memory()
            phi_h = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
            psi_h = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        finally:
            os.sched_setaffinity(0, saved)
        ctx.compute_host(y_h, precision=args.precision, out=(phi_h, psi_h))  # warm-up
        # each step is followed by a plain copy of the same outputs in the same pattern,
        # so that the copy bound is measured under the same host conditions
        times, copies = [], []
        for _ in range(max(args.e2e_steps, 1)):
            t0 = time.perf_counter()
            ctx.compute_host(y_h, precision=args.precision, out=(phi_h, psi_h))
            times.append(time.perf_counter() - t0)
            copies.append(output_copy_ms(phi_h, psi_h, phi, psi, n))
        e2e_s = reduce_max(pg, statistics.mean(times), device)
        link = link_bandwidth(phi_h, phi, stream)
        h2d_b, d2h_b = int(y.nbytes), int(2 * n * n * 4)
        out_ms = statistics.median(copies)
        link_ms = h2d_b / (link["h2d_gbs"] * 1e9) * 1e3 + out_ms
        e2e = {"value": world * outputs / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
               "api": "corr2d_compute_host", "ms_per_step": round(e2e_s * 1e3, 2),
               "ms_each_step": [round(t * 1e3, 2) for t in times],
               "link": {**link, "numa_node": node,
                        "pinned_on": "GPU's NUMA node" if cpus else "default placement",
                        "output_copy_ms": round(out_ms, 2),
                        "output_copy_gbs": round(d2h_b / (out_ms / 1e3) / 1e9, 1),
                        "copy_bound_ms": round(link_ms, 2),
                        "frac_of_copy_bound": round(link_ms / (e2e_s * 1e3), 4)}}
        del phi_h, psi_h, y_h

    ctx.close()
    cpu = None
    errors = {}
    if rank == 0 and world == 1:
        cpu, errors = cpu_baseline_leg(args, y, desc.get("alpha", 0.0), checks)
    if forms is not None:
        for name, e in errors.items():
            if name in forms:
                forms[name]["error"] = e
                tol = TOL["bf16" if name in ("bf16", "bf16_output") else "split"]
                forms[name]["within_tol"] = bool(e["rel_err_phi"] <= tol and e["rel_err_psi"] <= tol)
        x_ms = roofline["kernel_ms"]
        forms["speedup"] = {
            "split_vs_fp32_c4_step": round(forms["fp32"]["ms_per_step"] / ms_max, 2),
            "split_vs_fp32_c4_kernel": round(forms["fp32"]["kernel_ms"] / x_ms, 2),
            "batch_vs_per_problem_c5": round(forms["c5_per_problem"]["ms_per_step"] /
                                             forms["c5_batch"]["ms_per_step"], 2),
            "batch_vs_fp32_per_problem_c5": round(forms["c5_fp32_per_problem"]["ms_per_step"] /
                                                  forms["c5_batch"]["ms_per_step"], 2)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True,
        "scaling": scaling, "vs_baseline": None,
        "dtype": {"split": "f16 hi/lo split, f32 accumulate (double-float f32 centering)",
                  "bf16": "bf16, f32 accumulate (double-float f32 centering)",
                  "fp32": "f32 (f64 centering)"}[args.precision],
        "data": "synthetic (seeded band spectra; the paper's datasets are not available)",
        "config": config_for(desc, world, args.l2, parallelism),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        # the timed region holds each timed step and, with kernel timing, its profiled step
        "gpu_launches": launches_per_step * args.steps * (2 if per_call_timing else 1),
        "region_ms": round(t["region_ms"], 3),
    }
    if "main" in errors:
        line["error"] = errors["main"]
    if forms is not None:
        line["forms"] = forms
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    if rank != 0:
        return
    desc, inputs = workload(args.workload if args.workload != "c5" else "c4", args.precision)
    if args.workload in ("c4", "c2"):
        y = inputs[0]
    elif args.workload == "c3":
        y = inputs.y1
    else:
        y = inputs[0]
    rates = []
    n_s = args.cpu_sample_n or 0
    info = None
    ms = []
    target = max(2.0, min(15.0, 150.0 / max(args.steps, 1)))
    for _ in range(max(args.steps, 1)):
        rate, info = cpu_oracle_rate(y, n_s, desc.get("alpha", 0.0), target)
        n_s = int(re.search(r"first (\d+)", info["sample"]).group(1))
        rates.append(rate)
        ms.append(info["seconds"] * 1e3)
    value = statistics.mean(rates)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(ms), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded band spectra; the paper's datasets are not available)",
        "config": config_for(desc, world, args.l2), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": info["kind"],
                         "cores": info["cores"], "sample": info["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        # each step is one bounded oracle sample; keep the whole run to a few minutes
        if args.cpu_sample_n <= 0:
            args.cpu_sample_n = 0
        run_reference(args, world, rank)
        return
    world, rank, local, pg = dist_setup(args)
    try:
        run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
