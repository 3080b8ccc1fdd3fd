"""Benchmark: batched product-convolution apply on one GB300 per rank.

Workload (the throughput figure's configuration): 512x512 box, regular 16x16
sample grid (r = 256), rotated anisotropic Gaussian with smooth random
sigma1, sigma2 in [2, 8] and angle in [0, pi), R = 24, 128^2 patch FFTs, 64
right-hand sides of iid N(0,1) (synthetic, seeded).  One step = one
pc_apply_batched of the 64 vectors: gather . w, FFTs, spectral products,
inverse FFTs and the ordered overlap-add, all in libpc's kernels.

Metric: right-hand sides per second (higher is better).  ``value`` times the
step with x and y resident in HBM (L2 flushed between steps by writing a
256 MB buffer outside the timed window); ``e2e`` times the same call with the
inputs copied from pinned host memory and the result copied back inside the
timed window.  ``plain_gpu`` is the plain per-vector path (gather, cuFFT,
product, cuFFT, overlap-add) on the same operator.

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (a bounded random sample of output pixels per step, scaled to
right-hand sides per second).

Multi-GPU: the operator and the batch are replicated (weak scaling, no
collective on the data path); value = all ranks' right-hand sides / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "product-convolution RHS/s"
WORKLOAD = "fp32_512"
# description, kernel name and the sources whose hash keys the profiled DRAM traffic
WORKLOADS = {
    "fp32_512": ("512x512 regular 16x16 grid (r=256), anisotropic Gaussian R=24, 128^2 patch FFTs, 64 RHS",
                 "fft2d_kernel<float,128>", ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_overlap.cuh"]),
    "fp64_64": ("FP64 64x64 regular 4x4 grid (r=16), isotropic Gaussian R=12, 64^2 patch FFTs, 1 RHS "
                "(the correctness configuration: latency-bound)", "fft2d_kernel<double,64>",
                ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_overlap.cuh"]),
    "fp32_128c": ("128^3 regular 8x8x8 grid (r=512), axis-aligned Gaussian R=12, 64^3 patch FFTs, 32 RHS",
                  "fft3d_kernel<false,2>", ["pc_fft3d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_cluster.cuh"]),
    "bf16x3_128c": ("128^3 regular 8x8x8 grid (r=512), axis-aligned Gaussian R=12, 64^3 patches: plane FFTs in "
                    "FP32, first-axis DFTs as split-BF16 tensor-core GEMMs, 32 RHS",
                    "tc3d_axis0_kernel", ["pc_tc3d.cu", "pc_tc.cuh", "pc_ptx.cuh"]),
    "bf16x3_128c_adjoint": ("adjoint apply (Eq. adjoint_random_z) of the 128^3 regular 8x8x8 grid (r=512) operator, "
                            "axis-aligned Gaussian R=12, 64^3 patches: plane FFTs in FP32, first-axis correlation as "
                            "split-BF16 tensor-core GEMMs, 32 RHS", "tc3d_axis0_adj_kernel",
                            ["pc_tc3d.cu", "pc_tc.cuh", "pc_ptx.cuh"]),
    "fp32_128c_adjoint": ("adjoint apply (Eq. adjoint_random_z) of the 128^3 regular 8x8x8 grid (r=512) operator, "
                          "axis-aligned Gaussian R=12, 64^3 patch FFTs, 32 RHS", "fft3d_kernel<true,1>",
                          ["pc_fft3d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_cluster.cuh"]),
    "fp32_512_adjoint": ("adjoint apply (Eq. adjoint_random_z) of the 512x512 regular 16x16 grid (r=256) "
                         "operator, anisotropic Gaussian R=24, 128^2 patch FFTs, 64 RHS",
                         "fft2d_kernel<float,128,true>", ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh",
                                                          "pc_overlap.cuh"]),
    "fp32_512_estimator": ("randomized error estimator (Section 2.6) on the 512x512 regular 16x16 grid operator: "
                           "A~* of 64 probes, then per-cell FP64 norms of A~*Z - A*Z over the 225 leaf cells",
                           "fft2d_kernel<float,128,true>", ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh",
                                                            "pc_overlap.cuh"]),
    "fp32_512_block": ("block apply A~[T,S] (Section 3.3) of the 512x512 regular 16x16 grid operator: "
                       "T = [128,255]^2, S = [256,383]x[128,255] (adjacent 128^2 boxes, an H-matrix near-field "
                       "block), 64 RHS", "fft2d_kernel<float,128>",
                       ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_overlap.cuh"]),
    "fp32_512_blocks": ("the 100 near-field blocks A~[T_i,S_j] (Section 3.3) of the 512x512 regular 16x16 grid "
                        "operator for a 4x4 partition into 128^2 boxes (every pair of boxes that touch, itself "
                        "included), 64 RHS per block, one plan in two launches", "fft2d_kernel<float,128>",
                        ["pc_fft2d.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_overlap.cuh"]),
    "adaptive_1024": ("1024x1024 adaptive quadtree (r=1579), heavy-tailed R=64, per-patch FFT sizes "
                      "(128^2 with 2x2 kernel sub-windows, 256^2) chosen by the work model, 32 RHS",
                      "fft2d_parts<float,128|256>",
                      ["pc_fft2d.cu", "pc_fft2d_big.cu", "pc_fftcore.cuh", "pc_ptx.cuh", "pc_overlap.cuh"]),
}
# launch-shape arguments of a workload's operator (the rest take the defaults)
WORKLOAD_TUNING = {"adaptive_1024": {"per_patch": True}}
# workload name -> (operator configuration, precision)
WORKLOAD_OPERATOR = {"fp64_64": ("fp64_64", "fp64"), "fp32_512": ("fp32_512", "fp32"), "fp32_512_adjoint": ("fp32_512", "fp32"),
                     "fp32_512_estimator": ("fp32_512", "fp32"), "fp32_512_block": ("fp32_512", "fp32"),
                     "fp32_512_blocks": ("fp32_512", "fp32"),
                     "fp32_128c": ("fp32_128c", "fp32"), "bf16x3_128c": ("fp32_128c", "bf16x3"),
                     "fp32_128c_adjoint": ("fp32_128c", "fp32"), "bf16x3_128c_adjoint": ("fp32_128c", "bf16x3"),
                     "adaptive_1024": ("adaptive_1024", "fp32")}


# closed boxes (lo, hi) of the block workload: targets T, sources S
BLOCK_T = ((128, 128), (255, 255))
BLOCK_S = ((256, 128), (383, 255))


def near_field_blocks(n=512, box=128):
    """(T, S) pairs of a partition of [0, n)^2 into box x box squares: every
    ordered pair of squares that touch (itself included)."""
    m = n // box
    out = []
    for i0 in range(m):
        for i1 in range(m):
            for j0 in range(max(0, i0 - 1), min(m, i0 + 2)):
                for j1 in range(max(0, i1 - 1), min(m, i1 + 2)):
                    out.append((((i0 * box, i1 * box), (i0 * box + box - 1, i1 * box + box - 1)),
                                ((j0 * box, j1 * box), (j0 * box + box - 1, j1 * box + box - 1))))
    return out


def block_algorithmic_flops(lo, hi, R, nrhs, block=None):
    """Nominal FLOPs of a block apply: over the terms k whose bbox(U_k) meets
    S and whose reach bbox(U_k) (+) [-R, R]^2 meets T, 5 L log2 L + 3 L with
    L = prod_a (|S cap bbox(U_k)|_a + 2R), the linear-convolution extent of
    the translated term (Section 3.3)."""
    (tlo, thi), (slo, shi) = block if block is not None else (BLOCK_T, BLOCK_S)
    flops = 0.0
    terms = 0
    for a, b in zip(lo, hi):
        ca = [max(int(a[i]), slo[i]) for i in range(2)]
        cb = [min(int(b[i]), shi[i]) for i in range(2)]
        if any(cb[i] < ca[i] for i in range(2)):
            continue
        if any(cb[i] + R < tlo[i] or ca[i] - R > thi[i] for i in range(2)):
            continue
        L = float(np.prod([cb[i] - ca[i] + 1 + 2 * R for i in range(2)]))
        flops += 5.0 * L * math.log2(L) + 3.0 * L
        terms += 1
    return flops * nrhs, terms


def kernel_sources_hash(names):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1805_06018_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch from profiles/<kernel>_<workload>.md (an ncu
    capture), or None when the kernel sources changed since the capture."""
    desc, kname, srcs = WORKLOADS[workload]
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kname.split("<")[0], workload))
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_sources_sha256_16") != kernel_sources_hash(srcs):
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def algorithmic_work(shape, lo, hi, R, nrhs, spectra_bytes, elem=4):
    """FLOPs and HBM bytes per apply of the workload, by the nominal formula
    sum_k 5 L_k log2 L_k + 3 L_k with L_k = prod_a (n_a + 2R) (the exact
    linear-convolution extent of patch k), and x + y + spectra bytes."""
    flops = 0.0
    for a, b in zip(lo, hi):
        L = float(np.prod([(bb - aa + 1) + 2 * R for aa, bb in zip(a, b)]))
        flops += 5.0 * L * math.log2(L) + 3.0 * L
    N = int(np.prod(shape))
    return flops * nrhs, 2.0 * N * elem * nrhs + spectra_bytes


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 4 + i and r[4 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world):
    """The slowest rank's value, on every rank (one process: x itself).  The
    reduction runs on the process group's own device: CUDA for NCCL, the
    host for gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def cpu_oracle_rate(wl, x, seconds, seed=0, adjoint=False, keep=None):
    """Time the oracle on random output pixels until `seconds` have passed;
    returns (RHS/s-equivalent, pixels, threads, elapsed).  If `keep` is a
    dict it receives the last call's "points" and oracle "values" [B][n]."""
    from oracle import PCOracle
    orc = PCOracle.from_workload(wl)
    fn = orc.apply_adjoint if adjoint else orc.apply
    rng = np.random.default_rng(seed)
    done = 0
    t0 = time.perf_counter()
    chunk = min(512, wl.n)
    while time.perf_counter() - t0 < seconds:
        pts = rng.choice(wl.n, chunk, replace=False)
        out = fn(x, points=pts)
        if keep is not None:
            keep["points"], keep["values"] = pts, out
        done += chunk
        chunk = min(chunk * 2, 65536, wl.n)   # large calls: each also transposes the whole input batch
    el = time.perf_counter() - t0
    return wl.nrhs * (done / wl.n) / el, done, os.cpu_count(), el


def sampled_error(y, points, values):
    """Largest relative l2 error over the right-hand sides of the device
    result y [B][*box] at the oracle's sampled output pixels (FP64 values
    [B][len(points)])."""
    import torch
    idx = torch.as_tensor(np.asarray(points, dtype=np.int64), device=y.device)
    got = y.reshape(y.shape[0], -1).index_select(1, idx).double().cpu().numpy()
    ref = np.asarray(values, dtype=np.float64).reshape(got.shape)
    den = np.maximum(np.linalg.norm(ref, axis=1), np.finfo(np.float64).tiny)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / den))


def workload_config(wl, desc, world, fft):
    """The `config` dict of a bench line; both arms print the same one."""
    return {"workload": desc, "global_batch": wl.nrhs * world, "per_gpu_batch": wl.nrhs, "grid": list(wl.shape),
            "radius": wl.radius, "fft": fft, "parallelism": "replicas%d" % world,
            "l2": "flushed between steps (256 MB write)"}


def run_reference_block(args, wl):
    """Reference arm of the block workload: the oracle's translated block
    apply, one right-hand side per step (a bounded sample of the 64)."""
    import workloads
    from oracle import PCOracle
    from oracle.block import apply_block_translated
    (tlo, thi), (slo, shi) = BLOCK_T, BLOCK_S
    sS = tuple(b - a + 1 for a, b in zip(slo, shi))
    x = workloads.rhs(wl.rhs_seed, wl.nrhs, sS)
    orc = PCOracle.from_workload(wl)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        apply_block_translated(orc, tlo, thi, slo, shi, x[i % wl.nrhs:i % wl.nrhs + 1])
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload][0],
                                            "global_batch": wl.nrhs, "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                             "sample": "1 of the %d RHS per step through the translated block apply" % wl.nrhs},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    import workloads
    from workloads import configs
    from oracle import build as obuild
    obuild.build()
    wl = configs.get(WORKLOAD_OPERATOR[args.workload][0])
    if args.workload.endswith("_block") or args.workload.endswith("_blocks"):
        return run_reference_block(args, wl)
    # the FP32 right-hand sides, promoted to the oracle's FP64 before timing
    x = workloads.rhs(wl.rhs_seed, wl.nrhs, wl.shape).astype(np.float64)
    from oracle import PCOracle
    orc = PCOracle.from_workload(wl)
    fn = orc.apply_adjoint if args.workload.endswith("_adjoint") else orc.apply
    rng = np.random.default_rng(1)
    # each step is one oracle call on random output pixels.  A call also lays
    # out the whole input batch (a fixed cost that a full apply pays once), so
    # steps are as large as the run allows: the warm-up steps size the sample
    # so that a step takes about 120 s / (K + W) (0.5 s to 30 s), which keeps
    # the whole run near two minutes whatever the workload's cost per pixel
    target = min(30.0, max(0.5, 120.0 / (args.steps + args.warmup)))
    per_step = min(2048, wl.n)
    times = []
    for i in range(args.warmup + args.steps):
        pts = rng.choice(wl.n, per_step, replace=False)
        t0 = time.perf_counter()
        fn(x, points=pts)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
        elif dt > 0:
            per_step = int(min(wl.n, max(min(2048, wl.n), per_step * target / dt)))
    tot = sum(times)
    value = args.steps * wl.nrhs * (per_step / wl.n) / tot
    sample = ("%d random output pixels x %d RHS per step (of %d pixels), one oracle call each, which also "
              "transposes the whole input batch" % (per_step, wl.nrhs, wl.n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(wl, WORKLOADS[args.workload][0], world, wl.fft),
            "cpu_baseline": {"value": value, "unit": "RHS/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def block_oracle_rate(wl, xS, seconds):
    """The oracle's translated block apply (Section 3.3) on whole right-hand
    sides until `seconds` have passed; returns (RHS/s, RHS done, elapsed)."""
    from oracle import PCOracle
    from oracle.block import apply_block_translated
    orc = PCOracle.from_workload(wl)
    (tlo, thi), (slo, shi) = BLOCK_T, BLOCK_S
    done = 0
    t0 = time.perf_counter()
    while done < len(xS) and (done == 0 or time.perf_counter() - t0 < seconds):
        apply_block_translated(orc, tlo, thi, slo, shi, xS[done:done + 1])
        done += 1
    el = time.perf_counter() - t0
    return done / el, done, el


def run_block(args, rank, world):
    """One step = pc_block_apply of the workload's 64 right-hand sides on
    S, giving them on T; the plan is made once, before the timed region."""
    import torch
    import workloads
    from workloads import configs
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import build as libbuild

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    libbuild.build()
    wl = configs.get("fp32_512", **({"nrhs": args.nrhs} if args.nrhs > 0 else {}))
    desc, kname, _ = WORKLOADS[args.workload]
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    phi = workloads.impulse_windows(wl.shape, pts, wl.kernel)
    ctx = pcg.Context(torch.cuda.current_device())
    op = pcg.Operator(ctx, wl.shape, wl.cells, wl.radius, phi, precision="fp32")
    (tlo, thi), (slo, shi) = BLOCK_T, BLOCK_S
    plan = pcg.BlockPlan(op, tlo, thi, slo, shi)
    terms, tiles = plan.info()
    sS = tuple(b - a + 1 for a, b in zip(slo, shi))
    sT = tuple(b - a + 1 for a, b in zip(tlo, thi))
    nS, nT = int(np.prod(sS)), int(np.prod(sT))
    x_host = workloads.rhs(wl.rhs_seed, wl.nrhs, sS)
    x = torch.from_numpy(x_host).cuda()
    y = torch.empty((wl.nrhs,) + sT, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step():
        plan.pc_block_apply(wl.nrhs, x.data_ptr(), nS, y.data_ptr(), nT, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
    plan.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    tot_ms = float(step_ms.sum())
    if world > 1:
        dist.barrier()
    tot_ms = max_over_ranks(tot_ms, world)
    value = aggregate_rate(args.steps * wl.nrhs, world, tot_ms / 1e3)

    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty(y.shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(xh, non_blocking=True)
        step()
        yh.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = aggregate_rate(e2e_steps * wl.nrhs, world, e2e_s)

    lo, hi = pcg.pc_neighbourhood_boxes(wl.shape, wl.cells)
    flops, nominal_terms = block_algorithmic_flops(lo, hi, wl.radius, wl.nrhs)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    step_mean = float(step_ms.mean())
    achieved = flops / (step_mean / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc, "global_batch": wl.nrhs * world, "per_gpu_batch": wl.nrhs,
                       "grid": list(wl.shape), "radius": wl.radius, "T": [list(tlo), list(thi)],
                       "S": [list(slo), list(shi)], "terms": terms, "tiles": tiles,
                       "parallelism": "replicas%d" % world, "l2": "flushed between steps (256 MB write)"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "per": "block apply of %d RHS" % wl.nrhs},
            "e2e": {"value": e2e_value, "unit": "RHS/s", "h2d_bytes_per_step": int(x_host.nbytes),
                    "d2h_bytes_per_step": int(yh.numel() * 4)},
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": profiled_traffic(args.workload), "kernel": kname,
                         "kernel_ms": step_mean, "timed": "zero fill + patch kernel (events around the call)",
                         "algorithmic_flop_per_launch": flops, "nominal_terms": nominal_terms,
                         "peak_basis": "FP32 FMA pipe: SMs x 128 lanes x 2 x %.0f MHz" % sm_max},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        rate, done, el = block_oracle_rate(wl, x_host, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                                "sample": "%d of the %d RHS through the translated block apply in %.1f s"
                                          % (done, wl.nrhs, el)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    op.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_blocks(args, rank, world):
    """One step = pc_block_apply_many of the 100 near-field blocks, 64 RHS
    each; value counts block right-hand sides per second.  The same blocks
    as 100 single-block plans, one after another, are timed beside it."""
    import torch
    import workloads
    from workloads import configs
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import build as libbuild

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    libbuild.build()
    wl = configs.get("fp32_512", **({"nrhs": args.nrhs} if args.nrhs > 0 else {}))
    desc, kname, _ = WORKLOADS[args.workload]
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    phi = workloads.impulse_windows(wl.shape, pts, wl.kernel)
    ctx = pcg.Context(torch.cuda.current_device())
    op = pcg.Operator(ctx, wl.shape, wl.cells, wl.radius, phi, precision="fp32")
    blocks = near_field_blocks()
    nb = len(blocks)
    plan = pcg.BlockPlan(op, [b[0][0] for b in blocks], [b[0][1] for b in blocks], [b[1][0] for b in blocks],
                         [b[1][1] for b in blocks])
    terms, tiles = plan.info()
    nS = [int(np.prod(sh)) for sh in plan.s_shapes]
    nT = [int(np.prod(sh)) for sh in plan.t_shapes]
    xh = [workloads.rhs(wl.rhs_seed + i, wl.nrhs, sh) for i, sh in enumerate(plan.s_shapes)]
    xs = [torch.from_numpy(a).cuda() for a in xh]
    ys = [torch.empty((wl.nrhs,) + sh, dtype=torch.float32, device="cuda") for sh in plan.t_shapes]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    xp, yp = [x.data_ptr() for x in xs], [y.data_ptr() for y in ys]

    def step():
        plan.pc_block_apply_many(wl.nrhs, xp, nS, yp, nT, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.check()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
        torch.cuda.synchronize()
    plan.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    tot_ms = float(step_ms.sum())
    if world > 1:
        dist.barrier()
    tot_ms = max_over_ranks(tot_ms, world)
    value = aggregate_rate(args.steps * wl.nrhs * nb, world, tot_ms / 1e3)
    # the same blocks as separate single-block plans
    singles = [pcg.BlockPlan(op, *b[0], *b[1]) for b in blocks]
    for pl, x, y, a, c in zip(singles, xp, yp, nS, nT):
        pl.pc_block_apply(wl.nrhs, x, a, y, c, sp)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sep = []
    for _ in range(max(3, min(args.steps // 10, 10))):
        flush.fill_(1.0)
        s0.record(stream)
        for pl, x, y, a, c in zip(singles, xp, yp, nS, nT):
            pl.pc_block_apply(wl.nrhs, x, a, y, c, sp)
        s1.record(stream)
        torch.cuda.synchronize()
        sep.append(s0.elapsed_time(s1))
    for pl in singles:
        pl.close()
    # end to end with host buffers (pinned), copies in the timed region
    xph = [torch.from_numpy(a).pin_memory() for a in xh]
    yph = [torch.empty(y.shape, dtype=torch.float32).pin_memory() for y in ys]
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for x, h in zip(xs, xph):
            x.copy_(h, non_blocking=True)
        step()
        for y, h in zip(ys, yph):
            h.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e2e_value = aggregate_rate(e2e_steps * wl.nrhs * nb, world, max_over_ranks(time.perf_counter() - t0, world))
    lo, hi = pcg.pc_neighbourhood_boxes(wl.shape, wl.cells)
    flops = 0.0
    nominal = 0
    for b in blocks:
        f, t_ = block_algorithmic_flops(lo, hi, wl.radius, wl.nrhs, block=b)
        flops += f
        nominal += t_
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    step_mean = float(step_ms.mean())
    achieved = flops / (step_mean / 1e3) / 1e12
    rounds = (nb + 63) // 64
    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "blocks": nb, "counted": "block right-hand sides (blocks x RHS)",
                       "global_batch": wl.nrhs * world, "per_gpu_batch": wl.nrhs, "grid": list(wl.shape),
                       "radius": wl.radius, "terms": terms, "tiles": tiles, "parallelism": "replicas%d" % world,
                       "l2": "inputs (400 MB) larger than L2, and flushed between steps (256 MB write)"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "per": "%d blocks x %d RHS" % (nb, wl.nrhs)},
            "separate_single_block_plans": {"value": nb * wl.nrhs / (np.mean(sep) / 1e3), "unit": "RHS/s",
                                            "ms": float(np.mean(sep)), "kernels": 2 * nb},
            "e2e": {"value": e2e_value, "unit": "RHS/s",
                    "h2d_bytes_per_step": int(sum(a.nbytes for a in xh)),
                    "d2h_bytes_per_step": int(sum(y.numel() * 4 for y in ys))},
            "gpu_launches": 2 * rounds * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": profiled_traffic(args.workload), "kernel": kname,
                         "kernel_ms": step_mean,
                         "timed": "%d rounds of zero fill + patch kernel (events around the call)" % rounds,
                         "algorithmic_flop_per_launch": flops / rounds, "nominal_terms": nominal,
                         "peak_basis": "FP32 FMA pipe: SMs x 128 lanes x 2 x %.0f MHz" % sm_max},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        from oracle import PCOracle
        from oracle.block import apply_block_translated
        orc = PCOracle.from_workload(wl)
        done = 0
        t0 = time.perf_counter()
        while done == 0 or time.perf_counter() - t0 < args.cpu_seconds:
            (tlo, thi), (slo, shi) = blocks[done % nb]
            apply_block_translated(orc, tlo, thi, slo, shi, xh[done % nb][:1])
            done += 1
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / el, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                                "sample": "%d block right-hand sides through the translated block apply in %.1f s"
                                          % (done, el)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    op.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def serve_operators(pcg, ctx, with_3d=True, autotune=False):
    """The served operator mix: 2D 256^2 (9x9 grid), 512^2 (the benchmark
    operator), 1024^2 (adaptive quadtree, heavy-tailed, R = 64) and 2048^2
    (65x65 grid), FP32 with 128^2 patch FFTs; and 3D 64^3 ... 160^3 in FP32
    and BF16x3.  autotune: every operator's launch shape from the library's
    autotuner (a NULL pc_tuning) instead."""
    import workloads
    from workloads import configs
    wls = []
    for L, n in ((256, 9), (2048, 65)):
        shape = (L, L)
        kern = workloads.GaussianAniso2D(workloads.SmoothField(shape, 2.0, 8.0, 5000 + L),
                                         workloads.SmoothField(shape, 2.0, 8.0, 5001 + L),
                                         workloads.SmoothField(shape, 0.0, math.pi, 5002 + L), 24)
        wls.append(("gaussian_%d" % L, shape, workloads.regular_grid(shape, (n, n)), kern, 24))
    c2 = configs.fp32_512()
    wls.insert(1, ("gaussian_512", c2.shape, c2.cells, c2.kernel, c2.radius))
    c3 = configs.adaptive_1024()
    wls.insert(2, ("adaptive_1024", c3.shape, c3.cells, c3.kernel, c3.radius))
    ops = []
    for name, shape, cells, kern, R in wls:
        pts = pcg.pc_sample_points(shape, cells)
        # regular grids: 128^2 patch FFTs, batched with the other requests; the
        # adaptive operator: per-patch FFT sizes (its requests then run through its own apply)
        tune = {"autotune": True} if autotune else WORKLOAD_TUNING.get(name, {"fft_size": 128})
        ops.append((name, pcg.Operator(ctx, shape, cells, R, workloads.impulse_windows(shape, pts, kern),
                                       precision="fp32", **tune)))
    if with_3d:
        # 3D: 64^3 (5^3 grid), 96^3 (7^3), 128^3 (8^3, the 3D workload), 160^3
        # (10^3); axis-aligned Gaussian, sigma in [1.5, 5], R = 12, 64^3 patches;
        # each in FP32 and in the BF16x3 (tensor-core) mode
        for L, n in ((64, 5), (96, 7), (128, 8), (160, 10)):
            shape = (L, L, L)
            s3 = [workloads.SmoothField(shape, 1.5, 5.0, 4000 + 1 + i) for i in range(3)]
            kern = workloads.GaussianAxis3D(s3[0], s3[1], s3[2], 12)
            cells = workloads.regular_grid(shape, (n, n, n))
            pts = pcg.pc_sample_points(shape, cells)
            phi = workloads.impulse_windows(shape, pts, kern)
            for prec in ("fp32", "bf16x3"):
                ops.append(("gaussian3d_%d_%s" % (L, prec), pcg.Operator(ctx, shape, cells, 12, phi, precision=prec,
                                                                         autotune=autotune)))
    return ops


def serve_measure(pcg, ctx, ops, n_requests, rng, levels=(0.5, 0.8, 0.95), rhs_max=64, sat_requests=None,
                  plain=True):
    """Serving measurement over `ops` [(name, operator)]: requests pick an
    operator uniformly and U[1, rhs_max] right-hand sides; a saturated run
    (all submitted at once), then Poisson arrivals at each load level (a
    fraction of the saturated RHS/s) with n_requests requests each, 120 GB
    budget.  Returns the stats and, if `plain`, the plain per-vector path's
    RHS/s on the saturated request set (2D requests)."""
    import torch
    import workloads
    by_shape = {}
    for i, (_, op) in enumerate(ops):
        if op.shape not in by_shape:
            by_shape[op.shape] = torch.from_numpy(workloads.rhs(7000 + i, rhs_max, op.shape)).cuda()
    pools = [by_shape[op.shape] for _, op in ops]

    def make_requests(n):
        return [(int(rng.integers(0, len(ops))), int(rng.integers(1, rhs_max + 1))) for _ in range(n)]

    # per operator, a bounded pool of rhs_max-RHS output buffers (48 GB shared
    # by the operators); a request takes one and returns it on completion
    ybufs = []
    for o, (_, op) in enumerate(ops):
        per = rhs_max * op.N * 4
        ybufs.append([torch.empty_like(pools[o]) for _ in range(max(4, min(64, (48 << 30) // len(ops) // per)))])

    def run(reqs, rate):
        srv = pcg.Server(ctx, budget_bytes=120 << 30, max_inflight=512, streams=2, max_requests_per_launch=32)
        free = [list(range(len(b))) for b in ybufs]
        torch.cuda.synchronize()
        gaps = rng.exponential(1.0 / rate, len(reqs)) if rate else np.zeros(len(reqs))
        t0 = time.perf_counter()
        due = t0
        pending = {}

        def reap():
            for t in [t for t in pending if srv.poll(t) is not None]:
                o, b = pending.pop(t)
                free[o].append(b)

        for (o, k), g in zip(reqs, gaps):
            due += g
            while time.perf_counter() < due or not free[o]:
                reap()
            b = free[o].pop()
            pending[srv.submit(ops[o][1], pools[o][:k], ybufs[o][b][:k])] = (o, b)
        while pending:
            reap()
        st = srv.stats()
        srv.close()
        return st

    run(make_requests(16), None)   # warm-up
    sat_reqs = make_requests(sat_requests or max(32, n_requests // 2))
    sat = run(sat_reqs, None)
    mean_rhs = (1 + rhs_max) / 2.0
    loads = []
    for f in levels:
        reqs = make_requests(n_requests)
        st = run(reqs, f * sat["rhs_per_s"] / mean_rhs)
        loads.append({"load": f, "requests": st["completed"], "rhs_per_s": st["rhs_per_s"],
                      "p50_ms": 1e3 * st["p50_latency_s"], "p99_ms": 1e3 * st["p99_latency_s"],
                      "launches": st["launches"], "peak_budget_bytes": st["peak_bytes"]})
    out = {"saturated": {"requests": sat["completed"], "rhs_per_s": sat["rhs_per_s"],
                         "p50_ms": 1e3 * sat["p50_latency_s"], "p99_ms": 1e3 * sat["p99_latency_s"],
                         "launches": sat["launches"]},
           "loads": loads, "requests_after_warmup": sat["completed"] + sum(lv["requests"] for lv in loads)}
    if plain:
        # the plain per-vector path on the saturated request set, one request
        # after another (operators with per-patch shapes have no plain path:
        # their requests are left out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rhs = 0
        for o, k in sat_reqs:
            if ops[o][1].info()["num_parts"] > 1:
                continue
            y = torch.empty_like(pools[o][:k])
            ops[o][1].apply_plain(pools[o][:k], y)
            rhs += k
        torch.cuda.synchronize()
        out["plain_gpu_rhs_per_s"] = rhs / (time.perf_counter() - t0)
    return out


def run_serve(args):
    """Serving: Poisson arrivals of requests (operator uniform over the mix,
    RHS uniform in [1, 64]) at 50/80/95 % of the saturated rate, 120 GB budget."""
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import build as libbuild
    libbuild.build()
    ctx = pcg.Context(0)
    t0 = time.time()
    ops = serve_operators(pcg, ctx, with_3d=not args.serve_2d, autotune=not args.serve_fixed_shapes)
    build_s = time.time() - t0
    m = serve_measure(pcg, ctx, ops, args.serve_requests, np.random.default_rng(17))
    line = {"metric": "served product-convolution RHS/s; p50/p99 latency", "mode": "serve",
            "value": m["saturated"]["rhs_per_s"], "unit": "RHS/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "saturated": m["saturated"], "loads": m["loads"],
            "plain_gpu_rhs_per_s": m.get("plain_gpu_rhs_per_s"),
            "config": {"operators": [n for n, _ in ops], "rhs_per_request": "U[1,64]", "budget_bytes": 120 << 30,
                       "shapes": {n: {k: op.info()[k] for k in ("fft_size", "window_split", "tile", "ctas_per_sm",
                                                                "num_parts", "autotuned", "tuned_candidates")}
                                  for n, op in ops},
                       "shapes_from": "the library's autotuner (NULL pc_tuning)" if not args.serve_fixed_shapes else
                                      "fixed: 128^2 patch FFTs, per-patch shapes for the adaptive operator",
                       "operator_build_s": round(build_s, 1),
                       "arrivals": "Poisson at 50/80/95% of the saturated rate",
                       "modes": "2D FP32" if args.serve_2d else "2D FP32; 3D FP32 and BF16x3 (tensor-core first axis)",
                       "requests_after_warmup": m["requests_after_warmup"],
                       "plain_gpu": "the saturated request set, one request after another, without "
                                    "requests of per-patch operators (no plain path)"}}
    print(json.dumps(line), flush=True)


def roofline_of(pcg, wl, info, precision, kms, workload):
    """Roofline of the dominant kernel of one apply: nominal FLOPs (or, for the
    tensor-core stage, executed MMA FLOPs) over its event-timed duration
    (kms: per-step kernel ms, or per-step [stage0, stage1, stage2] ms for the
    BF16x3 split path), against the FP32 FMA pipe, the FP64 rate or the
    measured BF16 peak.  Returns (roofline, roofline_tensor or None, kernel
    name, kernel ms)."""
    import torch
    staged = precision == "bf16x3"
    kname = WORKLOADS[workload][1]
    if info.get("num_parts", 1) > 1 and not kname.startswith("fft2d_parts"):
        kname = "fft2d_parts<%d per-patch launch shapes>" % info["num_parts"]
    lo, hi = pcg.pc_neighbourhood_boxes(wl.shape, wl.cells)
    flops, bytes_ = algorithmic_work(wl.shape, lo, hi, wl.radius, wl.nrhs, info["spectra_bytes"],
                                     elem=8 if precision == "fp64" else 4)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    roof_tensor = None
    if staged:
        # three kernels per chunk; nominal flops split by transform axis:
        # phase 1 = forward axes 1, 2; tensor stage = axis 0 forward + inverse
        # + product; phase 3 = inverse axes 1, 2.  Executed tensor-core flops
        # count the MMAs the tensor stage issues (3 split products per step).
        adj = workload.endswith("_adjoint")
        stage_names = ["fft3d_phase1_kernel", "tc3d_axis0_adj_kernel" if adj else "tc3d_axis0_kernel",
                       "fft3d_phase3_kernel"]
        st_ms = np.mean(np.array(kms), axis=0)
        npairs = (wl.nrhs + 1) // 2
        f_stage = [0.0, 0.0, 0.0]
        mma_flops = 0.0
        assert info["num_tiles"] == len(lo), "one tile per patch expected"
        for a, b in zip(lo, hi):
            n = [bb - aa + 1 for aa, bb in zip(a, b)]
            Ls = [v + 2 * wl.radius for v in n]
            L = float(np.prod(Ls))
            f_stage[0] += 2.5 * L * (math.log2(Ls[1]) + math.log2(Ls[2]))
            f_stage[1] += 5.0 * L * math.log2(Ls[0]) + 3.0 * L
            f_stage[2] += 2.5 * L * (math.log2(Ls[1]) + math.log2(Ls[2]))
            # GEMM 1 over the n0 input planes (adjoint: the L0 output-box planes), GEMM 2 over 2 P
            rows_in = Ls[0] if adj else n[0]
            mma_flops += npairs * 32 * 3 * ((2 * rows_in + 15) // 16 + 8) * 2.0 * 128 * 128 * 16
        f_stage = [f * wl.nrhs for f in f_stage]
        bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
        tc_ach = mma_flops / (st_ms[1] / 1e3) / 1e12
        roof_tensor = {"bound": "tensor", "kernel": stage_names[1], "kernel_ms": float(st_ms[1]),
                       "executed_mma_flop_per_apply": mma_flops, "achieved": tc_ach, "peak": bf16_peak,
                       "unit": "TFLOP/s", "frac": tc_ach / bf16_peak,
                       "peak_basis": "measured cuBLAS bf16 GEMM (burst)",
                       "nominal_fft_tflops": f_stage[1] / (st_ms[1] / 1e3) / 1e12,
                       "stage_ms": {nm: float(t) for nm, t in zip(stage_names, st_ms)}}
        dom = int(np.argmax(st_ms))
        kname = stage_names[dom]
        kern_ms = float(st_ms[dom])
        if dom == 1:
            achieved, peak, bound, basis = tc_ach, bf16_peak, "tensor", roof_tensor["peak_basis"]
            work = mma_flops
        else:
            achieved = f_stage[dom] / (kern_ms / 1e3) / 1e12
            peak, bound = fp32_peak, "alu"
            basis = "FP32 FMA pipe: SMs x 128 lanes x 2 x %.0f MHz" % sm_max
            work = f_stage[dom]
    elif precision == "fp64":
        kern_ms = float(np.mean(kms))
        achieved, peak, bound, work = flops / (kern_ms / 1e3) / 1e12, 1.25, "alu", flops
        basis = "nominal GB300 FP64 rate, 1.25 TFLOP/s (no measured FP64 peak)"
    else:
        kern_ms = float(np.mean(kms))
        achieved, peak, bound, work = flops / (kern_ms / 1e3) / 1e12, fp32_peak, "alu", flops
        basis = "FP32 FMA pipe: SMs x 128 lanes x 2 x %.0f MHz" % sm_max
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kname, "kernel_ms": kern_ms, "algorithmic_flop_per_launch": work,
            "algorithmic_bytes_per_launch": bytes_, "peak_basis": basis}
    return roof, roof_tensor, kname, kern_ms


def suite_apply(pcg, ctx, name, steps, warmup, flush, plain_steps=2, accuracy_points=2048):
    """One sub-workload of the default run: its batched apply timed on the
    device (L2 flushed between steps), its result against the FP64 oracle at
    sampled output points, its roofline, and the plain per-vector path on the
    same operator where it applies.  Returns the entry and the operator."""
    import torch
    import workloads
    from workloads import configs
    from oracle import PCOracle
    cfg_name, precision = WORKLOAD_OPERATOR[name]
    wl = configs.get(cfg_name)
    desc = WORKLOADS[name][0]
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    op = pcg.Operator(ctx, wl.shape, wl.cells, wl.radius, workloads.impulse_windows(wl.shape, pts, wl.kernel),
                      precision=precision, **WORKLOAD_TUNING.get(name, {}))
    info = op.info()
    x_host = workloads.rhs(wl.rhs_seed, wl.nrhs, wl.shape)
    x = torch.from_numpy(x_host).cuda()
    if precision == "fp64":
        x = x.double()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    staged = precision == "bf16x3"
    for _ in range(warmup):
        op.pc_apply_batched(wl.nrhs, x.data_ptr(), wl.n, y.data_ptr(), wl.n, stream.cuda_stream)
    torch.cuda.synchronize()
    op.check()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kms = []
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        op.pc_apply_batched(wl.nrhs, x.data_ptr(), wl.n, y.data_ptr(), wl.n, stream.cuda_stream)
        ev[i][1].record(stream)
        kms.append([op.stage_ms(k) for k in range(3)] if staged else op.kernel_ms())
    torch.cuda.synchronize()
    op.check()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    entry = {"config": desc, "value": wl.nrhs * steps / (step_ms.sum() / 1e3), "unit": "RHS/s",
             "ms_per_step": float(step_ms.mean()), "steps": steps, "warmup": warmup,
             "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                            "per": "apply of %d RHS" % wl.nrhs},
             "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "f32+bf16x3"}[precision],
             "fft": info["fft_size"], "tile": info["tile"], "num_tiles": info["num_tiles"],
             "num_colors": info["num_colors"], "window_split": info["window_split"], "num_parts": info["num_parts"]}
    # accuracy: the oracle (FP64, direct sums) at sampled output points, all RHS
    rng = np.random.default_rng(5)
    npts = min(wl.n, accuracy_points)
    sel = np.sort(rng.choice(wl.n, npts, replace=False))
    orc = PCOracle.from_workload(wl)
    t0 = time.perf_counter()
    ref = orc.apply(x_host.astype(np.float64), points=sel)
    entry["accuracy"] = {"rel_l2_vs_fp64_oracle": sampled_error(y, sel, ref), "points": int(npts), "rhs": wl.nrhs,
                         "per": "max over right-hand sides", "oracle_s": time.perf_counter() - t0}
    roof, roof_tensor, kname, _ = roofline_of(pcg, wl, info, precision, kms, name)
    roof["traffic"] = profiled_traffic(name) if kname == WORKLOADS[name][1] else None
    entry["roofline"] = roof
    if roof_tensor is not None:
        entry["roofline_tensor"] = roof_tensor
    if precision != "fp64" and plain_steps > 0:
        yp = torch.empty_like(x)
        op.pc_apply_plain(wl.nrhs, x.data_ptr(), wl.n, yp.data_ptr(), wl.n, stream.cuda_stream)
        torch.cuda.synchronize()
        pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(plain_steps)]
        for a, b in pe:
            flush.fill_(1.0)
            a.record(stream)
            op.pc_apply_plain(wl.nrhs, x.data_ptr(), wl.n, yp.data_ptr(), wl.n, stream.cuda_stream)
            b.record(stream)
        torch.cuda.synchronize()
        pms = [a.elapsed_time(b) for a, b in pe]
        entry["plain_gpu"] = {"value": wl.nrhs / (np.mean(pms) / 1e3), "unit": "RHS/s", "ms_per_apply": float(np.mean(pms)),
                              "accuracy_rel_l2_vs_fp64_oracle": sampled_error(yp, sel, ref),
                              "path": "per vector: gather, cuFFT R2C, product, cuFFT C2R, overlap-add (FP32)"}
        del yp
    del x, y
    return entry, op


def suite(pcg, ctx, args):
    """The other configurations, measured on the same run: the FP64 64^2
    correctness workload, the 3D 128^3 workload in FP32 and with the
    tensor-core first axis (BF16x3), the adaptive 1024^2 workload (batched,
    and as 256 served requests of U[1,32] right-hand sides), and serving of
    the 2D operator mix with Poisson arrivals."""
    import torch
    import workloads
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    plan = [("fp64_64", 30, 3), ("fp32_128c", 8, 3), ("bf16x3_128c", 8, 3), ("adaptive_1024", 8, 3)]
    for name, steps, warm in plan:
        try:
            entry, op = suite_apply(pcg, ctx, name, steps, warm, flush,
                                    plain_steps=0 if name == "adaptive_1024" else 2,
                                    accuracy_points=512 if name.endswith("128c") else 2048)
            if name == "adaptive_1024":
                # the adaptive workload as written: 256 requests of U[1,32] RHS through the server
                m = serve_measure(pcg, ctx, [("adaptive_1024", op)], 256, np.random.default_rng(31), levels=(),
                                  rhs_max=32, sat_requests=256, plain=False)
                entry["served_256_requests"] = dict(m["saturated"], rhs_per_request="U[1,32]",
                                                    arrivals="all 256 submitted at once")
            op.close()
            out[name] = entry
        except Exception as e:   # a report, never a reason to lose the line
            out[name] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
        torch.cuda.empty_cache()
    del flush
    if args.suite_serve_requests > 0:
        try:
            t0 = time.time()
            ops = serve_operators(pcg, ctx, with_3d=False, autotune=not args.serve_fixed_shapes)
            build_s = time.time() - t0
            m = serve_measure(pcg, ctx, ops, args.suite_serve_requests, np.random.default_rng(17))
            m["config"] = {"operators": [n for n, _ in ops], "rhs_per_request": "U[1,64]", "budget_bytes": 120 << 30,
                           "shapes": {n: {k: op.info()[k] for k in ("fft_size", "window_split", "tile", "ctas_per_sm",
                                                                    "num_parts", "autotuned", "tuned_candidates")}
                                      for n, op in ops},
                           "shapes_from": "the library's autotuner (NULL pc_tuning)" if not args.serve_fixed_shapes
                                          else "fixed: 128^2 patch FFTs, per-patch shapes for the adaptive operator",
                           "operator_build_s": round(build_s, 1),
                           "arrivals": "Poisson at 50/80/95% of the saturated rate",
                           "plain_gpu": "the saturated request set, one request after another, "
                                        "without the per-patch operator's requests (no plain path)"}
            out["serving_2d_mix"] = m
            for _, op in ops:
                op.close()
        except Exception as e:
            out["serving_2d_mix"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--serve", action="store_true", help="serving benchmark instead of the batched apply")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-2d", action="store_true", help="serve the 2D operators of the mix only")
    ap.add_argument("--serve-fixed-shapes", action="store_true",
                    help="serve operators with fixed launch shapes (128^2 patch FFTs, per-patch shapes for the "
                         "adaptive operator) instead of the shapes the library's autotuner chooses")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--nrhs", type=int, default=0,
                    help="override the workload's batch (smaller cases for profiler captures)")
    ap.add_argument("--no-suite", action="store_true",
                    help="skip the other configurations that the default run adds under 'workloads'")
    ap.add_argument("--suite-serve-requests", type=int, default=2000,
                    help="requests per load level of the default run's serving measurement (0: skip it)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.serve:
        return run_serve(args)
    if args.workload.endswith("_block"):
        return run_block(args, rank, world)
    if args.workload.endswith("_blocks"):
        return run_blocks(args, rank, world)

    import torch
    import torch.distributed as dist
    import workloads
    from workloads import configs
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import build as libbuild

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(pcg.binding.LIB_PATH):
        libbuild.build()
    if world > 1:
        dist.barrier()

    cfg_name, precision = WORKLOAD_OPERATOR[args.workload]
    wl = configs.get(cfg_name, **({"nrhs": args.nrhs} if args.nrhs > 0 else {}))
    desc, kname, ksrcs = WORKLOADS[args.workload]
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    phi = workloads.impulse_windows(wl.shape, pts, wl.kernel)
    ctx = pcg.Context(local)
    op = pcg.Operator(ctx, wl.shape, wl.cells, wl.radius, phi, precision=precision,
                      **WORKLOAD_TUNING.get(args.workload, {}))
    staged = precision == "bf16x3"
    info = op.info()
    x_host = workloads.rhs(wl.rhs_seed, wl.nrhs, wl.shape)
    if precision == "fp64":
        x_host = x_host.astype(np.float64)
    x = torch.from_numpy(x_host).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    N = wl.n

    apply_fn = op.pc_apply_adjoint_batched if args.workload.endswith("_adjoint") else op.pc_apply_batched
    estimator = args.workload.endswith("_estimator")
    if estimator:
        # Y = A* Z stands in as a second seeded array: the work does not depend on its values
        y_true = torch.from_numpy(workloads.rhs(wl.rhs_seed + 1, wl.nrhs, wl.shape)).cuda()

    def step():
        if estimator:
            op.estimate_cell_errors(x, y_true, len(wl.cells), stream=stream)
        else:
            apply_fn(wl.nrhs, x.data_ptr(), N, y.data_ptr(), N, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    op.check()

    # ---- device-resident timing
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
            kms.append([op.stage_ms(k) for k in range(3)] if staged else op.kernel_ms())
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    op.check()
    launches_per_step = int(op.launches())
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    tot_ms = float(step_ms.sum())
    tot_ms = max_over_ranks(tot_ms, world)
    value = aggregate_rate(args.steps * wl.nrhs, world, tot_ms / 1e3)

    # ---- end to end through the public API with host buffers
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    is_adj = args.workload.endswith("_adjoint")
    if not estimator:
        # pc_apply_host: pinned host buffers in and out, copies pipelined with the kernels
        op.pc_apply_host(wl.nrhs, xh.data_ptr(), N, yh.data_ptr(), N, is_adj, 0, sp)
        torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        if estimator:
            x.copy_(xh, non_blocking=True)
            step()   # the estimator returns its per-cell result on the host itself
        else:
            op.pc_apply_host(wl.nrhs, xh.data_ptr(), N, yh.data_ptr(), N, is_adj, 0, sp)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e_value = aggregate_rate(e2e_steps * wl.nrhs, world, e2e_s)

    # ---- plain per-vector path on the same operator
    plain = None
    adjoint = args.workload.endswith("_adjoint") or estimator
    if not args.no_plain and wl.ndim == 2 and not adjoint and precision == "fp32":
        yp = torch.empty_like(x)
        op.pc_apply_plain(wl.nrhs, x.data_ptr(), N, yp.data_ptr(), N, sp)
        torch.cuda.synchronize()
        pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        psteps = max(3, min(args.steps // 10, 20))
        pms = []
        for _ in range(psteps):
            flush.fill_(1.0)
            pe0.record(stream)
            op.pc_apply_plain(wl.nrhs, x.data_ptr(), N, yp.data_ptr(), N, sp)
            pe1.record(stream)
            torch.cuda.synchronize()
            pms.append(pe0.elapsed_time(pe1))
        rel = float(torch.max(torch.linalg.vector_norm((yp - y).reshape(wl.nrhs, -1), dim=1) /
                              torch.linalg.vector_norm(y.reshape(wl.nrhs, -1), dim=1)).item())
        plain = {"value": wl.nrhs / (np.mean(pms) / 1e3), "unit": "RHS/s", "p50_ms": float(np.median(pms)),
                 "max_rel_l2_vs_fused": rel, "kernels_per_step": op.launches()}
        step()  # leave the operator's last launch = the fused path

    # ---- roofline of the fused kernel (FP32 ALU bound)
    roof, roof_tensor, kname, kern_ms = roofline_of(pcg, wl, info, precision, kms, args.workload)
    roof["traffic"] = profiled_traffic(args.workload) if kname == WORKLOADS[args.workload][1] else None

    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32",
            "data": "synthetic",
            "config": workload_config(wl, desc, world, info["fft_size"]),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "per": "apply of %d RHS" % wl.nrhs},
            "plain_gpu": plain,
            "e2e": {"value": e2e_value, "unit": "RHS/s", "h2d_bytes_per_step": int(x_host.nbytes),
                    "d2h_bytes_per_step": 8 * len(wl.cells) if estimator else int(x_host.nbytes),
                    "call": "pc_estimate_cell_errors after a host-to-device copy of Z" if estimator else
                    "pc_apply_host (pinned host x, y; chunked copies overlapped with the kernels)"},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof,
            "clocks": clk.summary()}
    if roof_tensor is not None:
        line["roofline_tensor"] = roof_tensor
        line["dtype"] = "f32+bf16x3"
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        kept = {}
        rate, pix, cores, el = cpu_oracle_rate(wl, x_host, args.cpu_seconds, adjoint=adjoint, keep=kept)
        line["cpu_baseline"] = {"value": rate, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                                "sample": "%d random output pixels x %d RHS in %.1f s" % (pix, wl.nrhs, el)}
        if not estimator and kept:
            # the timed result against the FP64 oracle at the last sample's pixels
            try:
                err = sampled_error(y, kept["points"], kept["values"])
                line["accuracy"] = {"rel_l2_vs_fp64_oracle": err, "pixels": int(len(kept["points"])),
                                    "rhs": wl.nrhs, "per": "max over right-hand sides"}
            except Exception as e:   # a report, never a reason to lose the line
                line["accuracy"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    if rank == 0 and world == 1 and args.workload == WORKLOAD and not args.no_suite:
        op.close()
        op = None
        del x, y, flush
        torch.cuda.empty_cache()
        line["workloads"] = suite(pcg, ctx, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if op is not None:
        op.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
