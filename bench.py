#!/usr/bin/env python
"""Benchmark: free-space Poisson solve throughput (grid cells solved / s).

One step = one full solve (five passes) of the default workload, the largest
single-GPU configuration: a 512^3-cell FP32 field (seeded lognormal random
field with a k^-3 spectrum plus a uniform ball of radius 40 cells), unit
spacing, G = 1, padded to 1024^3.  Inputs are resident in HBM before timing
(and larger than L2); L2 is also flushed (256 MiB write) between steps
outside the timed events.  Each rank solves its own independent field (weak
scaling, no data-path collective).

Prints ONE JSON line on rank 0.  `--impl reference` times the FP64 CPU
oracle (FFT-convolution route, its kernel transformed once as a plan would)
on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid cells solved/sec and % of HBM roofline at stated rel-L2 vs FP64 oracle"
UNIT = "cells/s"
PASS_NAMES = ["x_fwd", "y_fwd", "z_conv", "y_inv", "x_inv"]
KERNEL_NAMES = ["k_x_fwd", "k_y_fwd", "k_z_conv", "k_y_inv", "k_x_inv"]
TOL_REL_L2 = 1e-6

WORKLOADS = {
    "blobs32": dict(n=32, desc="32^3 cells, 4 seeded Gaussian blobs (widths 2-5 cells, amplitudes "
                    "U[0.5,2]) on a zero background, unit spacing, G=1, zero-padded to 64^3; "
                    "accuracy against the direct pair sum"),
    "plummer256": dict(n=256, desc="256^3 cells FP32, 64 seeded Plummer spheres + 1% uniform "
                       "background, unit spacing, G=1, zero-padded to 512^3"),
    "lognormal512": dict(n=512, desc="512^3 cells FP32, seeded lognormal field (sigma 1.5, "
                         "k^-3 spectrum) + uniform ball r=40, zero-padded to 1024^3"),
    "plummer384x8": dict(n=384, fields=8, desc="8 fields of 384^3 cells, 16 seeded Plummer "
                         "spheres each + 1% uniform background, zero-padded to 768^3 "
                         "(radix-3 sizes), solved one after another with one plan"),
    "batch96": dict(n=None, desc="96 FP32 fields, edges from {64,96,128,192,256,384}, half "
                    "cubic / half 2:1, 4-16 seeded Gaussian blobs each, one graph launch per "
                    "batch (persistent kernel or per-field kernels, whichever is faster)"),
    "nested128x8": dict(n=128, fields=8, desc="8 nested-grid levels of 128^3 FP32 cells (spacing "
                        "halving per level, 1 .. 2^-7), 16 seeded Plummer spheres each + 1% background; "
                        "value: device-resident batched solve; e2e: host-staged levels with transfers "
                        "overlapped (poisson_solve_host_levels, pinned)"),
}


def make_density(name, seed):
    import workloads
    n = WORKLOADS[name]["n"]
    if name == "blobs32":
        rho, _ = workloads.gaussian_blobs(n, count=4, seed=seed)
        return rho  # FP64 workload: no cast here
    if name == "plummer256":
        rho, _ = workloads.plummer_spheres(n, count=64, seed=seed)
    elif name == "plummer384x8":
        rho, _ = workloads.plummer_spheres(n, count=16, seed=seed)
    else:
        rho, _ = workloads.lognormal_field(n, seed=seed)
    return rho.astype(np.float32)


def pass_bytes(nx, ny, nz, rsize=4):  # rsize: bytes per real value
    """Algorithmic HBM bytes of each pass (read + write, octant Ghat)."""
    c = 2 * rsize
    cells = nx * ny * nz
    w1 = (nx + 1) * ny * nz * c
    w2 = (nx + 1) * 2 * ny * nz * c
    g = (nx + 1) * (ny + 1) * (nz + 1) * rsize
    return [cells * rsize + w1, w1 + w2, 2 * w2 + g, w2 + w1, w1 + cells * rsize]


# the sources the pass kernels (five passes, tensor-core z pass) are built
# from: a profile's counters stay valid while these are unchanged
KERNEL_SOURCES = ("fft_core.cuh", "fft_pk.cuh", "passes.cuh", "passes_pk.cuh", "configs.cuh", "tma.cuh", "tc_dft.cuh", "internal.h",
                  "greens_layout.h",
                  "twiddles.cu", "passes_f32_row.cu", "passes_f32_y.cu", "passes_f32_z.cu", "passes_f64.cu",
                  "passes_tc.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_02294_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """dram bytes/launch from a committed ncu summary, if it was taken on the
    current kernel sources (profiles/*.md lines 'traffic: <kernel> <workload>
    <bytes> source=<hash>')."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    cur = source_hash()
    pat = re.compile(r"^traffic:\s+(\S+)\s+(\S+)\s+(\d+)\s+source=(\w+)", re.M)
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        for m in pat.finditer(open(os.path.join(pdir, fn)).read()):
            if m.group(1) == kernel and m.group(2) == workload and m.group(4) == cur:
                return int(m.group(3))
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20", "-i", str(self.gpu_id)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def started(self):
        """True once nvidia-smi has written its first sample."""
        try:
            self.fh.flush()
            return self.proc is None or os.path.getsize(self.path) > 0
        except Exception:
            return True

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=sorted(reasons), samples=len(rows))
        return out


_ORACLE_CACHE = {}


def cpu_oracle_time(rho32, reps, min_seconds):
    """Time the FP64 oracle (FFT-convolution route, all host cores).  The
    kernel's transform depends only on the grid and is computed once before
    the timed solves, as a plan would; each timed solve is the forward real
    FFT of the padded density, the multiply and the inverse FFT.  The last
    input's result is kept, so that another precision of the same field
    reuses it as its accuracy reference when reps = 0 is asked."""
    import oracle
    key = (rho32.shape, hashlib.sha256(np.ascontiguousarray(rho32).tobytes()).hexdigest())
    if reps == 0 and key in _ORACLE_CACHE:
        return list(_ORACLE_CACHE[key][0]), _ORACLE_CACHE[key][1]
    reps = max(reps, 1)
    rho = rho32.astype(np.float64)
    Kh = oracle.kernel_rfft(rho.shape, workers=-1)
    times = []
    out = None
    t_start = time.perf_counter()
    while len(times) < reps or (time.perf_counter() - t_start) < min_seconds:
        t0 = time.perf_counter()
        out = oracle.solve_fft_with(rho, Kh, workers=-1)
        times.append(time.perf_counter() - t0)
        if len(times) >= 20:
            break
    _ORACLE_CACHE.clear()
    _ORACLE_CACHE[key] = (times, out)
    return times, out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = args.workload
    n = WORKLOADS[wl]["n"]
    rho32 = make_density(wl, args.seed)
    import oracle
    rho = rho32.astype(np.float64)
    Kh = oracle.kernel_rfft(rho.shape, workers=-1)  # once, as a plan would
    for _ in range(args.warmup):
        oracle.solve_fft_with(rho, Kh, workers=-1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.solve_fft_with(rho, Kh, workers=-1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * n ** 3 / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl, "description": WORKLOADS[wl]["desc"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "full %d^3 field per step, oracle FFT-convolution route "
                                   "(scipy.fft FP64, workers=all cores; the kernel's transform "
                                   "computed once before the steps)" % n},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def max_over_ranks(value, world, device=None):
    """Largest `value` over all ranks (the job's wall time is the slowest
    rank's); identity on one rank.  Works with any torch.distributed backend
    (NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, cells_per_rank, steps, max_seconds):
    """Whole-job throughput: every rank solves its own field each step, so
    the job solves world * cells_per_rank cells per step."""
    return world * cells_per_rank * steps / max_seconds


def field_seed(base_seed, rank, nfields, field):
    """Seed of field `field` of `rank`: every rank's fields are distinct."""
    return base_seed + rank * nfields + field


def execution_desc(mode, launches):
    if mode == 0:
        return "one kernel per pass (%d launches per solve)" % launches
    if mode in (1, 2):
        return "one persistent dataflow kernel per solve (fused mode %d)" % mode
    return ("x passes whole, y/z/y passes in column bands on %d streams (banded mode %d, %d launches "
            "per solve)" % (4 if mode == 3 else 8, mode, launches))


def library_baselines(plan, rho, n, steps, flush, stream):
    """Baselines timed on the same GPU and input:
    (a) this library's plain FP32 pipeline (poisson_solve_unfused: the
    padded grid materialised, full per-axis FFTs with the library's own line
    transforms, separate multiply and crop) -- the yardstick for what the
    pruned, fused passes buy;
    (b) cuFFT (through torch.fft) 3-D R2C/C2R with separate pad, multiply
    and crop kernels;
    (c) cuFFT per axis: pad, per-axis forward FFTs, multiply, per-axis
    inverse FFTs, crop.
    (b) and (c) use this plan's transformed Green's function (expanded from
    its octant), so all three compute the same Phi."""
    import torch
    M = 2 * n
    octant = torch.from_numpy(plan.greens_octant()).to(device=rho.device, dtype=rho.dtype)
    fold = torch.arange(M, device=rho.device)
    fold = torch.minimum(fold, M - fold)
    gfull = octant[fold][:, fold][:, :, : n + 1].contiguous()  # rfft layout [kz][ky][kx]
    pad = torch.zeros((M, M, M), device=rho.device, dtype=rho.dtype)

    def cufft_3d():
        pad.zero_()
        pad[:n, :n, :n] = rho
        X = torch.fft.rfftn(pad)
        X *= gfull
        y = torch.fft.irfftn(X, s=(M, M, M), norm="forward")
        return y[:n, :n, :n].contiguous()

    def plain_per_axis():
        pad.zero_()
        pad[:n, :n, :n] = rho
        X = torch.fft.rfft(pad, dim=2)
        X = torch.fft.fft(X, dim=1)
        X = torch.fft.fft(X, dim=0)
        X *= gfull
        X = torch.fft.ifft(X, dim=0, norm="forward")
        X = torch.fft.ifft(X, dim=1, norm="forward")
        y = torch.fft.irfft(X, n=M, dim=2, norm="forward")
        return y[:n, :n, :n].contiguous()

    own = torch.empty_like(rho)

    def plain_own():
        return plan.solve_unfused(rho, out=own, stream=stream)

    out = {}
    for name, fn in (("plain_own_unfused", plain_own), ("cufft_r2c_3d", cufft_3d),
                     ("cufft_per_axis_unfused", plain_per_axis)):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in ts)
        out[name] = {"ms": ms, "cells_per_s": n ** 3 / (ms / 1e3), "result": res}
    return out


def host_transfer_experiment():
    """The paper's host-staging measurement (a 128^3 array moved host ->
    device, pinned vs pageable; 1 ms vs 3 ms on its A100 nodes) repeated on
    this GPU's host link, for an FP64 array."""
    import torch
    n = 128
    res = {"bytes": n ** 3 * 8}
    dev = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    for name, pin in (("pinned", True), ("pageable", False)):
        h = torch.randn((n, n, n), dtype=torch.float64)
        if pin:
            h = h.pin_memory()
        for _ in range(3):
            dev.copy_(h, non_blocking=pin)
        torch.cuda.synchronize()
        ts = []
        for _ in range(20):
            t0 = time.perf_counter()
            dev.copy_(h, non_blocking=pin)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        res[name + "_ms"] = 1e3 * statistics.median(ts)
    return res


BATCH_MODES = ["persistent kernel (k_batched)", "per-field launches in one graph, autotuned variants",
               "per-field launches in one graph, untuned variants"]


def batch_launches(plans, mode):
    """Kernel launches of one batched solve: one persistent kernel (mode 0);
    per field, the launches one solve with the plan's variants makes,
    counted from a captured solve (mode 1: a column pass on a persistent
    TMA variant adds a plain launch for its Nyquist-column tiles), or five
    (mode 2: the untuned variants)."""
    if mode == 0:
        return 1
    if mode == 2:
        return 5 * len(plans)
    return sum(p.launch_count() for p in plans)


def run_batch(args):
    """Batched uneven solve: one persistent kernel per batch (graph replay)."""
    import torch

    import paper_2409_02294_gb300 as pg
    import workloads

    torch.cuda.set_device(0)
    shapes = workloads.batch_shapes(96, seed=args.seed)
    dens = workloads.batch_densities(shapes, seed=args.seed)
    # autotuned per shape (a shape that repeats reuses the first plan's tuning)
    plans = [pg.Plan(s[2], s[1], s[0], flags=pg.abi.FLAG_AUTOTUNE) for s in shapes]
    rhos = [torch.from_numpy(d).cuda() for d in dens]
    phis = [torch.empty_like(r) for r in rhos]
    cells = sum(int(np.prod(sh)) for sh in shapes)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pg.solve_batched(plans, rhos, phis, stream)  # the first call picks the faster mode
    torch.cuda.synchronize()
    assert plans[0].sync_status() == 0
    chosen = pg.batch_mode(plans)

    def timed(mode):
        pg.batch_mode(plans, mode)
        for _ in range(2):
            pg.solve_batched(plans, rhos, phis, stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for e0, e1 in evs:
            e0.record(stream)
            pg.solve_batched(plans, rhos, phis, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        return sorted(e0.elapsed_time(e1) for e0, e1 in evs)

    others = {m: timed(m) for m in (0, 1, 2) if m != chosen}
    lat = timed(chosen)
    total_ms = sum(lat)
    # the same fields solved one after another with the single-field passes
    seq = []
    for _ in range(max(3, min(args.steps, 10))):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p, r, o in zip(plans, rhos, phis):
            p.solve(r, out=o)
        e1.record(stream)
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    # accuracy: batched output vs the single-field solve for every field, and
    # vs the FP64 oracle for one field of each distinct shape (up to 12)
    pg.solve_batched(plans, rhos, phis, stream)
    worst = 0.0
    for p, r, o in zip(plans, rhos, phis):
        ref = p.solve(r)
        worst = max(worst, float((o.double() - ref.double()).norm() / ref.double().norm()))
    acc = {"max_rel_l2_vs_single_field_solve": worst}
    if not args.no_cpu_baseline:
        import oracle
        seen, l2s, mxs = set(), [], []
        for s, d, o in zip(shapes, dens, phis):
            if s in seen or len(seen) >= 12:
                continue
            seen.add(s)
            ref = oracle.solve_fft(d.astype(np.float64))
            out = o.double().cpu().numpy()
            l2s.append(float(np.linalg.norm(out - ref) / np.linalg.norm(ref)))
            mxs.append(float(np.abs(out - ref).max() / np.abs(ref).max()))
        acc.update({"rel_l2": max(l2s), "max_rel": max(mxs), "tolerance_rel_l2": TOL_REL_L2,
                    "reference": "FP64 oracle, full field, one field of each of %d distinct shapes "
                                 "(worst of them)" % len(seen)})
    pb = 0
    for s in shapes:
        pb += sum(pass_bytes(s[2], s[1], s[0]))
    peak, peak_kind = peaks()
    mean_s = total_ms / len(lat) / 1e3
    achieved = pb / mean_s / 1e9
    line = {
        "metric": METRIC, "value": cells / mean_s, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / len(lat),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batch96", "description": WORKLOADS["batch96"]["desc"],
                   "fields": len(shapes), "cells": cells,
                   "l2": "inputs (3.1 GB) larger than L2"},
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "min": lat[0], "max": lat[-1]},
        "batch_mode": {"chosen": BATCH_MODES[chosen],
                       "other_modes_p50_ms": {BATCH_MODES[m]: v[len(v) // 2] for m, v in others.items()}},
        "sequential_single_field_ms": statistics.median(seq),
        "roofline": {"bound": "hbm", "kernel": "k_batched" if chosen == 0 else "all kernels of the batch graph",
                     "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes": pb, "peak_source": peak_kind},
        "accuracy": acc,
        "gpu_launches": args.steps * batch_launches(plans, chosen),
    }
    for p in plans:
        p.close()
    return emit(line, args)


def run_levels(args):
    """Nested-grid levels: independent 128^3 fields with halving spacing,
    solved from device memory (batched) and from host memory with the
    transfers overlapped with the solves."""
    import torch

    import paper_2409_02294_gb300 as pg
    import workloads

    torch.cuda.set_device(0)
    wl = "nested128x8"
    n, nl = WORKLOADS[wl]["n"], WORKLOADS[wl]["fields"]
    plans = [pg.Plan(n, n, n, h=2.0 ** -l, flags=pg.abi.FLAG_AUTOTUNE if l == 0 else 0) for l in range(nl)]
    for p in plans[1:]:  # same grid size: reuse the variants tuned on level 0
        for i, v in enumerate(plans[0].info()["variant"]):
            p.set_variant(i, v)
        p.set_variant(5, plans[0].info()["fused"])
    dens = [workloads.plummer_spheres(n, count=16, seed=args.seed + l)[0].astype(np.float32) for l in range(nl)]
    rhos = [torch.from_numpy(d).cuda() for d in dens]
    phis = [torch.empty_like(r) for r in rhos]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    cells = nl * n ** 3
    for _ in range(max(3, args.warmup)):
        pg.solve_batched(plans, rhos, phis, stream)
    torch.cuda.synchronize()
    lat = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pg.solve_batched(plans, rhos, phis, stream)
        e1.record(stream)
        lat.append((e0, e1))
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) for a, b in lat)
    ms = statistics.median(lat)
    # cpu_baseline leg: the oracle timed on one level on the host cores; its
    # result is also the accuracy reference for that level
    cpu = acc = None
    if not args.no_cpu_baseline:
        import oracle
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            ref = oracle.solve_fft(dens[3].astype(np.float64), h=2.0 ** -3)
            ts.append(time.perf_counter() - t0)
        cpu = {"value": n ** 3 / statistics.median(ts), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one 128^3 level (level 3), oracle FFT-convolution route (scipy.fft FP64, all host "
                         "cores), 3 solves, median"}
        out = phis[3].double().cpu().numpy()
        acc = {"rel_l2": float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
               "max_rel": float(np.abs(out - ref).max() / np.abs(ref).max()),
               "tolerance_rel_l2": TOL_REL_L2, "reference": "FP64 oracle, full field (level 3)"}
    # host-staged: overlapped pipeline vs one poisson_solve_host per level
    hin = [torch.from_numpy(d).pin_memory() for d in dens]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    for _ in range(3):
        pg.solve_host_levels(plans, hin, hout, stream)
    k = max(5, min(args.steps, 30))
    t0 = time.perf_counter()
    for _ in range(k):
        pg.solve_host_levels(plans, hin, hout, stream)
    t_ov = (time.perf_counter() - t0) / k
    t0 = time.perf_counter()
    for _ in range(k):
        for p, a, b in zip(plans, hin, hout):
            p.solve_host(a, b, stream)
    t_seq = (time.perf_counter() - t0) / k
    same = all(torch.equal(hout[i], phis[i].cpu()) for i in range(nl))
    pb = sum(pass_bytes(n, n, n)) * nl
    peak, peak_kind = peaks()
    achieved = pb / (ms / 1e3) / 1e9
    launches = sum(p.launch_count() for p in plans) if pg.batch_mode(plans) == 1 else 1
    line = {
        "metric": METRIC, "value": cells / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl, "description": WORKLOADS[wl]["desc"], "levels": nl, "cells": cells,
                   "l2": "flushed between steps (256 MiB write, outside the timed events)"},
        "latency_ms": {"p50": ms, "min": lat[0], "max": lat[-1]},
        "roofline": {"bound": "hbm", "kernel": "all kernels of the batch graph", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes": pb, "peak_source": peak_kind},
        "accuracy": acc,
        "cpu_baseline": cpu,
        "e2e": {"value": cells / t_ov, "unit": UNIT, "h2d_bytes_per_step": cells * 4,
                "d2h_bytes_per_step": cells * 4, "steps": k, "host_memory": "pinned",
                "sequential_host_solves_value": cells / t_seq,
                "overlap_speedup": t_seq / t_ov, "equal_to_device_solve": same},
        "gpu_launches": launches * args.steps,
    }
    for p in plans:
        p.close()
    return emit(line, args)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2409_02294_gb300 as pg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()

    wl = args.workload
    n = WORKLOADS[wl]["n"]
    nf = WORKLOADS[wl].get("fields", 1)
    rdt = np.float64 if args.precision == "fp64" else np.float32
    rhos32 = [make_density(wl, field_seed(args.seed, rank, nf, i)).astype(rdt) for i in range(nf)]
    rho32 = rhos32[0]
    rhos = [torch.from_numpy(r).to(dev) for r in rhos32]
    phis = [torch.empty_like(r) for r in rhos]
    rho, phi = rhos[0], phis[0]
    if args.variants:
        # fixed kernel variants (x fwd, y fwd, z, y inv, x inv, execution mode),
        # no autotuning: for profiling one known configuration
        plan = pg.Plan(n, n, n, precision=args.precision)
        for i, v in enumerate(int(x) for x in args.variants.split(",")):
            plan.set_variant(i, v)
    else:
        plan = pg.Plan(n, n, n, precision=args.precision, flags=pg.abi.FLAG_AUTOTUNE)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    fused = plan.info()["fused"]
    launches = plan.launch_count()  # kernel launches per solve, counted from a captured graph

    def step(evs=None, per_pass=False):
        for f in range(nf):
            if evs is not None and f == 0:
                evs[0].record(stream)
            if fused and not per_pass:
                plan.solve(rhos[f], out=phis[f], stream=stream)
                if evs is not None:
                    evs[f * 5 + 5].record(stream)
                continue
            for i in range(5):
                plan.solve_pass(i, rhos[f], phis[f], stream)
                if evs is not None:
                    evs[f * 5 + i + 1].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    events = [[torch.cuda.Event(enable_timing=True) for _ in range(5 * nf + 1)] for _ in range(args.steps)]
    props = torch.cuda.get_device_properties(dev)
    gpu_id = "GPU-" + str(props.uuid) if hasattr(props, "uuid") else str(dev.index)
    sampler = ClockSampler(gpu_id)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    # keep the GPU busy with untimed solves until the sampler reports, so that
    # its samples cover the whole timed region
    t_wait = time.perf_counter()
    while not sampler.started() and time.perf_counter() - t_wait < 5.0:
        flush.zero_()
        step()
        torch.cuda.synchronize()
    barrier()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        step(events[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clocks = sampler.stop()

    step_ms = [ev[0].elapsed_time(ev[5 * nf]) for ev in events]
    if fused:
        # per-pass breakdown of the five-launch mode, measured after the timed
        # region, for the roofline of each kernel
        pev = [[torch.cuda.Event(enable_timing=True) for _ in range(5 * nf + 1)]
               for _ in range(min(args.steps, 50))]
        for ev in pev:
            flush.zero_()
            step(ev, per_pass=True)
        torch.cuda.synchronize()
    else:
        pev = events
    pass_ms = [sum(ev[f * 5 + i].elapsed_time(ev[f * 5 + i + 1]) for ev in pev for f in range(nf))
               / (len(pev) * nf) for i in range(5)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    cells = n ** 3 * nf
    value = weak_scaling_value(world, cells, args.steps, total_ms / 1e3)

    # accuracy of this run's output against the FP64 oracle, and the oracle
    # timed on the host cores (rank 0, N = 1 only)
    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, ref = cpu_oracle_time(rho32, reps=getattr(args, "cpu_reps", 2),
                                     min_seconds=getattr(args, "cpu_min_seconds", 8.0) if nf == 1 else 0.0)
        if wl == "blobs32":
            import oracle
            ref = oracle.solve_direct(rho32.astype(np.float64))  # the exact pair sum
        out = phi.double().cpu().numpy()
        acc = {"rel_l2": float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
               "max_rel": float(np.abs(out - ref).max() / np.abs(ref).max()),
               "tolerance_rel_l2": {"fp64": 1e-12, "fp32": TOL_REL_L2, "tc_fp16x2": TOL_REL_L2,
                                    "tc_bf16x2": 1e-5}[args.precision],
               "reference": ("FP64 oracle direct pair sum" if wl == "blobs32" else "FP64 oracle, full field")
               + (" (field 0)" if nf > 1 else "")}
        cpu = {"value": n ** 3 / statistics.median(times), "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "full %d^3 field, oracle FFT-convolution route (scipy.fft FP64, all "
                         "host cores; kernel transform computed once beforehand), %d solves, "
                         "median" % (n, len(times))}

    # library baselines on the same GPU, same input
    libs = None
    host_xfer = None
    if rank == 0 and world == 1 and not args.no_baselines:
        # timed on field 0; for a batch of equal fields the whole batch takes nf times that
        lb = library_baselines(plan, rho, n, min(args.steps, 20), flush, stream)
        ours = phi.double()
        libs = {}
        for k, v in lb.items():
            r = v.pop("result").double()
            if nf > 1:
                v["ms_all_fields"] = v["ms"] * nf
                v["note"] = "ms is per field (field 0); the batch of %d fields takes ms_all_fields" % nf
            v["rel_l2_vs_this_solve"] = float((r - ours).norm() / ours.norm())
            if acc is not None:
                v["rel_l2_vs_oracle"] = float(np.linalg.norm(r.cpu().numpy() - ref) / np.linalg.norm(ref))
            libs[k] = v
        host_xfer = host_transfer_experiment()

    # end to end through the C-ABI host-buffer calls: every step's H2D of rho
    # and D2H of phi are inside the timed region.  The K steps go through one
    # poisson_solve_host_levels call (each step's transfers overlap the
    # neighbouring steps' solves); one synchronous poisson_solve_host per step
    # is reported beside it.
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(rhos32[0]).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        ksteps = max(3, min(args.steps, 50))
        lv = ([plan] * ksteps, [host_in] * ksteps, [host_out] * ksteps)
        for _ in range(2):
            pg.solve_host_levels(*lv, stream=stream)
            plan.solve_host(host_in, host_out, stream)
        barrier()
        t0 = time.perf_counter()
        pg.solve_host_levels(*lv, stream=stream)
        te = time.perf_counter() - t0
        te = max_over_ranks(te, world, dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            plan.solve_host(host_in, host_out, stream)
        ts = time.perf_counter() - t0
        ts = max_over_ranks(ts, world, dev)
        e2e = {"value": weak_scaling_value(world, n ** 3, ksteps, te), "unit": UNIT,
               "h2d_bytes_per_step": rho32.nbytes, "d2h_bytes_per_step": rho32.nbytes,
               "steps": ksteps, "host_memory": "pinned",
               "host_path": "poisson_solve_host_levels over the steps' fields (transfers overlapped)",
               "synchronous_per_step_value": weak_scaling_value(world, n ** 3, ksteps, ts)}
        if rank == 0 and world == 1:
            pg_in = torch.from_numpy(rhos32[0].copy())
            pg_out = torch.empty_like(pg_in)
            plan.solve_host(pg_in, pg_out, stream)
            t0 = time.perf_counter()
            for _ in range(max(3, ksteps // 5)):
                plan.solve_host(pg_in, pg_out, stream)
            tp = (time.perf_counter() - t0) / max(3, ksteps // 5)
            e2e["pageable_value"] = n ** 3 / tp

    dom = int(np.argmax(pass_ms))
    kernel_names = list(KERNEL_NAMES)
    if args.precision in ("tc_fp16x2", "tc_bf16x2"):
        kernel_names[2] = "k_z_conv_tc"
    pb = pass_bytes(n, n, n, 8 if args.precision == "fp64" else 4)
    peak, peak_kind = peaks()
    if fused:
        # the solve is one kernel (fused modes) or overlapping kernels on
        # several streams (banded modes): the roofline is the whole solve's
        dom_name = "k_fused" if fused in (1, 2) else "all kernels of the banded solve"
        dom_bytes = sum(pb)
        achieved = dom_bytes * nf / (total_ms / args.steps / 1e3) / 1e9
    else:
        dom_name = kernel_names[dom]
        dom_bytes = pb[dom]
        achieved = pb[dom] / (pass_ms[dom] / 1e3) / 1e9
    traffic = profiled_traffic(dom_name, wl)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32"}.get(args.precision, "f32+%s" % args.precision[3:]),
            "data": "synthetic",
            "config": {"workload": wl, "description": WORKLOADS[wl]["desc"], "precision": args.precision,
                       "l2": "flushed between steps (256 MiB write, outside the timed events)",
                       "parallelism": "independent field per GPU" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
                         if peak_kind == "measured" else "fallback 6800 GB/s",
                         "traffic": traffic, "algorithmic_bytes": dom_bytes},
            "execution": execution_desc(fused, launches),
            "passes" if not fused else "five_launch_breakdown":
                {PASS_NAMES[i]: {"ms": pass_ms[i], "GBps": pb[i] / (pass_ms[i] / 1e3) / 1e9,
                                       "frac": pb[i] / (pass_ms[i] / 1e3) / 1e9 / peak}
                       for i in range(5)},
            "solve_roofline_frac": sum(pb) * nf / (total_ms / args.steps / 1e3) / 1e9 / peak,
            "accuracy": acc,
            "library_baselines_same_gpu": libs,
            "host_transfer_128cube_fp64": host_xfer,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches * nf * args.steps,
            "kernel_variants": plan.info()["variant"],
            "clocks": clocks,
            "wall_s_timed": t_wall,
        }
    plan.close()
    del rhos, phis, rho, phi, flush
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    if world == 1 and args.configs:
        line["configs"] = secondary_configs(args)
    return emit(line, args)


# The other configurations of the benchmark, measured in the same run after
# the headline line (one GPU): the 32^3 FP64 direct-sum check, 256^3 Plummer,
# the 96-field uneven batch, 8 x 384^3 Plummer in FP32 and both
# compensated tensor-core precisions, and the nested-grid levels.
SECONDARY = [("blobs32", "fp64"), ("plummer256", "fp32"), ("batch96", "fp32"), ("plummer384x8", "fp32"),
             ("plummer384x8", "tc_fp16x2"), ("plummer384x8", "tc_bf16x2"), ("nested128x8", "fp32")]
DROP_KEYS = ("metric", "unit", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data",
             "library_baselines_same_gpu", "host_transfer_128cube_fp64", "e2e", "kernel_variants")


def secondary_configs(args):
    import copy
    import gc

    import torch
    out = {}
    for wl, prec in SECONDARY:
        a = copy.copy(args)
        a.workload, a.precision = wl, prec
        a.steps, a.warmup = max(5, min(args.steps, 20)), 3
        a.no_e2e, a.no_baselines, a.variants, a.configs, a.quiet = True, True, "", False, True
        # the oracle here gives the accuracy reference (computed once per field)
        a.cpu_reps, a.cpu_min_seconds = 0, 0.0
        key = wl if prec == "fp32" else "%s_%s" % (wl, prec)
        t0 = time.perf_counter()
        try:
            line = RUNNERS.get(wl, run_ours)(a)
            out[key] = {k: v for k, v in line.items() if k not in DROP_KEYS}
        except Exception as exc:  # report, keep the headline line
            out[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
        out[key]["wall_s"] = time.perf_counter() - t0
        gc.collect()
        torch.cuda.empty_cache()
    return out


def emit(line, args):
    if getattr(args, "quiet", False):
        return line
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="lognormal512")
    ap.add_argument("--seed", type=int, default=2409)
    ap.add_argument("--precision", choices=["fp64", "fp32", "tc_fp16x2", "tc_bf16x2"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--variants", default="",
                    help="comma list of kernel variants per pass (and execution mode): skip autotuning")
    ap.add_argument("--grid", default="",
                    help="NXxNYxNZ: time the passes of one plan on this grid (seeded normal density), "
                         "for profiling a kernel on a smaller case")
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="measure only the headline workload (by default the other configurations are "
                         "measured after it and reported under 'configs')")
    args = ap.parse_args()
    args.quiet = False
    if args.workload != "lognormal512" or args.variants:
        args.configs = False
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.grid:
        return run_grid(args)
    return RUNNERS.get(args.workload, run_ours)(args)


def run_grid(args):
    """One plan on an arbitrary grid (--grid NXxNYxNZ) with a seeded
    standard-normal density: per-pass CUDA-event times and HBM fractions of
    the five passes.  For profiling a pass kernel of a given transform length
    on a grid smaller than the benchmark's (e.g. the 512-long z columns on
    256 x 256 x 512)."""
    import torch

    import paper_2409_02294_gb300 as pg
    nx, ny, nz = (int(v) for v in args.grid.lower().split("x"))
    torch.cuda.set_device(0)
    rng = np.random.default_rng(args.seed)
    rho = torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
    phi = torch.empty_like(rho)
    if args.variants:
        plan = pg.Plan(nx, ny, nz)
        for i, v in enumerate(int(x) for x in args.variants.split(",")):
            plan.set_variant(i, v)
    else:
        plan = pg.Plan(nx, ny, nz, flags=pg.abi.FLAG_AUTOTUNE)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flush.zero_()
        for i in range(5):
            plan.solve_pass(i, rho, phi, stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    for ev in evs:
        flush.zero_()
        ev[0].record(stream)
        for i in range(5):
            plan.solve_pass(i, rho, phi, stream)
            ev[i + 1].record(stream)
    torch.cuda.synchronize()
    pass_ms = [statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in evs) for i in range(5)]
    step_ms = statistics.mean(ev[0].elapsed_time(ev[5]) for ev in evs)
    pb = pass_bytes(nx, ny, nz)
    peak, _ = peaks()
    line = {"metric": METRIC, "value": nx * ny * nz / (step_ms / 1e3), "unit": UNIT, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grid %dx%dx%d (seeded normal density)" % (nx, ny, nz)},
            "passes": {PASS_NAMES[i]: {"ms": pass_ms[i], "frac": pb[i] / (pass_ms[i] / 1e3) / 1e9 / peak}
                       for i in range(5)},
            "kernel_variants": plan.info()["variant"]}
    plan.close()
    return emit(line, args)


RUNNERS = {"batch96": run_batch, "nested128x8": run_levels}

if __name__ == "__main__":
    sys.exit(main())
