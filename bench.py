#!/usr/bin/env python
"""Benchmark: Myrtle-5 32x32 NNGP kernel entries/s and PCG iterations/s on GB300.

Workload (the headline configuration): Myrtle-5 stage pattern (2, 1, 0),
sigma_w^2 = 2, sigma_b^2 = 0, 2048 train + 512 test 32x32x3 images (N(0,1)
noise blurred by a 3x3 box filter, standardised per channel), 10 random
classes (one-hot minus 0.1).  One step is the whole hot path: per-image
self-variances, the train-train kernel block (upper triangle, 2,098,176
unique entries), the test-train block (1,048,576 entries), and the Jacobi
PCG ridge solve of the train block (10 right-hand sides, lambda = 1e-4 tr(K)/N,
relative residual 1e-6 with FP64 refinement).  value = unique kernel entries
per second of the whole step.

Also reported: the fused kernel alone (roofline, plain ALU bound), the plain
layer-wise FP32 / FP64 forms on sample tiles at equal accuracy, PCG
iterations/s mixed vs plain FP64, the end-to-end number through host buffers,
and the CPU oracle on the host cores.

--impl reference times the float64 CPU oracle (the only reference this
method has) on the same workload and metric, on a bounded sample per step.
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Myrtle-5 32x32 kernel entries/s and PCG iters/s: mixed vs plain at rel err<=1e-5"
CONVS = (2, 1, 0)
SW2, SB2 = 2.0, 0.0
REL_LAMBDA = 1e-4
CONFIGS = {
    "headline": dict(n_train=2048, n_test=512, hw=32, n_classes=10),
    "small": dict(n_train=64, n_test=16, hw=32, n_classes=10),
    # a small 64x64 case (profiling the tiled form on a short launch)
    "small64": dict(n_train=16, n_test=8, hw=64, n_classes=10),
}
FP32_LANES_PER_SM = 128  # the derived fallback when no probe file exists
PEAKS_PROBE = os.path.join(ROOT, "profiles", "peaks_probe.json")


def algorithmic_ops_per_entry(hw: int, convs=CONVS, C: int = 3) -> float:
    """FP32 operations per kernel entry by the method's own arithmetic.

    Per pixel pair of a stage and per layer: conv stencil 9 adds + 1 FMA for
    scale and bias = 10; arc-cosine map 25 (scaling products 2, clamp 2,
    1 - c^2 1, sqrt 1, range reduction 2, degree-6 arcsine polynomial 8,
    select 2, assembly 4, output scale 1, stencil-free); seed channel
    contraction C FMAs; 2x2 pool or global average 1 add."""
    ops = 0.0
    n_stages_eff = 1 + (convs[1] > 0 if len(convs) > 1 else 0) + (
        (convs[1] > 0 and convs[2] > 0) if len(convs) > 2 else 0)
    for s in range(n_stages_eff):
        pairs = (hw >> s) ** 4
        per = 0.0
        if s == 0:
            per += C
        per += convs[s] * (10 + 25)
        per += 1  # pool scatter or global average
        ops += pairs * per
    return ops


# --------------------------------------------------------------------------
# CPU oracle legs (spawned workers; the oracle is test infrastructure, run
# here only as the cpu_baseline / reference arm)
# --------------------------------------------------------------------------

def _oracle_worker(args):
    seed, n_pairs, hw = args
    import numpy as np
    import torch

    torch.set_num_threads(1)
    sys.path.insert(0, ROOT)
    import oracle

    import nkdata

    x = torch.tensor(nkdata.standardise(nkdata.images(n_pairs + 1, hw, 3, seed, blur=True))[0]
                     .astype(np.float32).astype(np.float64))
    arch = oracle.Arch(CONVS)
    qs = [oracle.myrtle_self_q(arch, SW2, SB2, x[i]) for i in range(n_pairs + 1)]
    t0 = time.perf_counter()
    for k in range(n_pairs):
        oracle.myrtle_layers_pair(arch, SW2, SB2, x[k], x[k + 1], qs[k], qs[k + 1])
    return time.perf_counter() - t0


def cpu_pcg_rate(n: int = 2048, r: int = 10, d: int = 3072):
    """The oracle's textbook Jacobi PCG (float64 numpy, BLAS threads as numpy
    starts them) on a kernel matrix the oracle computes itself: the depth-3
    FC ReLU NNGP (sigma_w^2 = 2, sigma_b^2 = 0.01) of n random rows of
    dimension d; r right-hand sides, lambda = 1e-4 tr(K)/n, tol 1e-6.  Only
    the solve is timed.  The CPU counterpart of the PCG iterations/s."""
    import numpy as np

    import nkdata
    import oracle

    X = nkdata.fc_rows(n, d, seed=nkdata.SEED_TRAIN).astype(np.float64)
    K = oracle.fc_nngp(X, X, 2.0, 0.01, depth=3).numpy()
    lam = 1e-4 * float(np.trace(K)) / n
    Y = nkdata.labels(n, r)
    total_its, solves, relmax = 0, 0, 0.0
    t0 = time.perf_counter()
    while solves == 0 or time.perf_counter() - t0 < 1.0:  # repeated solves, about a second
        _, iters, rel = oracle.pcg(K, Y, lam, precond="jacobi", tol=1e-6, maxit=20000)
        total_its += int(iters)
        solves += 1
        relmax = max(relmax, float(np.max(rel)))
    dt = time.perf_counter() - t0
    return {"iters_per_s": total_its / dt, "iters": total_its // solves, "solves": solves, "seconds": dt,
            "relres": relmax, "kind": "oracle",
            "sample": f"Jacobi PCG, {r} right-hand sides, N = {n} (FC3 NNGP of {n} random rows of dimension "
                      f"{d}, float64 numpy), tol 1e-6, solved {solves} times"}


def cpu_baseline_line(rate: float, pairs: int, seconds: float, cores: int, pairs_per_process: int,
                      workload_entries: int) -> dict:
    """The cpu_baseline object: the oracle's all-core rate on the bounded
    sample, per core, and the time the whole workload would take at that rate
    (extrapolated, not measured)."""
    return {"value": rate, "unit": "entries/s", "cores": cores, "kind": "oracle",
            "per_core": rate / cores, "workload_extrapolated_s": workload_entries / rate,
            "sample": f"{pairs} Myrtle-5 32x32 pixel-pair recursions ({pairs_per_process} per process, "
                      f"{cores} spawned processes x 1 thread, float64 torch CPU); self-variances "
                      f"precomputed outside the timed loop; {seconds:.1f} s"}


def cpu_oracle_rate(n_workers: int, pairs_per_worker: int, hw: int, seed0: int = 100):
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_workers) as pool:
        t0 = time.perf_counter()
        times = pool.map(_oracle_worker, [(seed0 + w, pairs_per_worker, hw) for w in range(n_workers)])
        wall = time.perf_counter() - t0
    pairs = n_workers * pairs_per_worker
    # self-variances are computed outside the timed loop: they are O(N) per
    # image, negligible against the O(N^2) entries of a full job
    return pairs / max(times), pairs, max(times), wall


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (a replicated job takes as long as its
    slowest replica); x itself without a process group."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, units_per_replica: float, seconds: float) -> float:
    """Whole-job units per second: each of the `world` replicas processes the
    same workload (weak scaling, no data-path exchange)."""
    return world * units_per_replica / seconds


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


TRAFFIC_HEADLINE = os.path.join(ROOT, "profiles", "k_myrtle_tiled_traffic_headline.json")


def headline_traffic(config_name: str, variant: int):
    """DRAM bytes of the tiled kernel's two launches of a headline step, from
    the ncu capture recorded in profiles/ (dram__bytes_read + write), while
    the kernel's source files hash as they did at the capture; None
    otherwise (another kernel, another workload, or changed sources)."""
    import hashlib

    if variant != 3 or config_name != "headline":
        return None, "no capture of this kernel and workload"
    try:
        with open(TRAFFIC_HEADLINE) as f:
            rec = json.load(f)
        h = hashlib.sha256()
        for rel in rec["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as g:
                h.update(g.read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None, "the kernel's sources changed since the capture"
        return float(rec["bytes_per_step"]), ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the step's two "
                                              "launches (profiles/k_myrtle_tiled_traffic_headline.json); the kernel "
                                              "is ALU-bound, this is about 9 GB/s of DRAM traffic")
    except Exception as e:
        return None, f"no traffic record ({type(e).__name__})"


def load_probe() -> dict:
    """Rates measured by `bench.py --probe-peaks` on this GPU type (nk_probe),
    stored per SM and cycle so that they scale with the clock a run saw."""
    try:
        with open(PEAKS_PROBE) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak(sm_count: int, clock_mhz: float) -> tuple:
    """FP32 lane-operations per second at this clock: the probed FMA issue
    rate per SM and cycle when a probe file exists, else the unit count."""
    pr = load_probe()
    per = pr.get("fp32_fma_per_sm_per_cycle")
    if per:
        return (sm_count * per * clock_mhz * 1e6 / 1e12,
                f"probed: {per:.1f} FP32 lane-FMAs per SM per cycle (nk_probe, {pr.get('gpu', '?')}) x "
                f"{sm_count} SMs x {clock_mhz:.0f} MHz")
    return (sm_count * FP32_LANES_PER_SM * clock_mhz * 1e6 / 1e12,
            f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x {clock_mhz:.0f} MHz (FP32 ops/s)")


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args, rank, world, dist):
    import numpy as np
    import torch

    import nkdata
    from paper_2303_05420_gb300.api import Handle

    cfg = CONFIGS[args.config]
    n_tr, n_te, hw = cfg["n_train"], cfg["n_test"], cfg["hw"]

    # CPU oracle baseline first: its spawn pool starts before any CUDA call
    cpu = None
    cpu_pcg = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        rate, pairs, tmax, wall = cpu_oracle_rate(cores, args.cpu_pairs, hw)
        cpu = cpu_baseline_line(rate, pairs, tmax, cores, args.cpu_pairs, n_tr * (n_tr + 1) // 2 + n_te * n_tr)
        cpu_pcg = cpu_pcg_rate()

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    prob = nkdata.image_problem(n_tr, n_te, hw, n_classes=cfg["n_classes"], blur=True)
    Xh = torch.tensor(np.concatenate([prob.x_train, prob.x_test]).astype(np.float32)).pin_memory()
    Yh = torch.tensor(prob.y_train).pin_memory()
    X = Xh.to(dev)
    Y = Yh.to(dev)
    h = Handle()
    # autotune the fused kernel's launch shape for this workload (setup, untimed)
    if args.fused_variant is None:
        variant = h.autotune(CONVS, SW2, SB2, hw, hw, 3)
    else:
        variant = args.fused_variant
        h.autotune_set(CONVS, SW2, SB2, hw, hw, variant)
    Ktr = torch.empty((n_tr, n_tr), dtype=torch.float32, device=dev)
    Kte = torch.empty((n_te, n_tr), dtype=torch.float32, device=dev)
    A = torch.empty((n_tr, Y.shape[1]), dtype=torch.float64, device=dev)
    entries = n_tr * (n_tr + 1) // 2 + n_te * n_tr
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(Xd, Yd, marks=None):
        if marks is not None:
            marks[0].record(stream)
        q = h.self_diag(Xd, CONVS, SW2, SB2)
        if marks is not None:
            marks[1].record(stream)
        h.block(Xd, q, Xd, q, CONVS, SW2, SB2, prec="mixed", a_range=(0, n_tr), b_range=(0, n_tr),
                symmetric=True, out=Ktr)
        h.block(Xd, q, Xd, q, CONVS, SW2, SB2, prec="mixed", a_range=(n_tr, n_tr + n_te),
                b_range=(0, n_tr), out=Kte)
        if marks is not None:
            marks[2].record(stream)
        _, its, rel = h.pcg_solve(Ktr, Yd, -REL_LAMBDA, precond="jacobi", prec="mixed", tol=1e-6,
                                  maxit=20000, A=A)
        if marks is not None:
            marks[3].record(stream)
        return its, rel

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(X, Y)
    h.sync_status()

    sampler = ClockSampler(dev.index)
    step_ms, sd_ms, blk_ms, pcg_ms, iters, rels = [], [], [], [], [], []
    launches0 = h.launch_count()
    sampler.start()
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        marks = [ev() for _ in range(4)]
        its, rel = step(X, Y, marks)
        torch.cuda.synchronize()
        step_ms.append(marks[0].elapsed_time(marks[3]))
        sd_ms.append(marks[0].elapsed_time(marks[1]))
        blk_ms.append(marks[1].elapsed_time(marks[2]))
        pcg_ms.append(marks[2].elapsed_time(marks[3]))
        iters.append(its)
        rels.append(max(rel))
    barrier()
    clocks = sampler.stop()
    launches = h.launch_count() - launches0
    h.sync_status()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = replica_throughput(world, entries * args.steps, total_ms / 1e3)

    # ---- end to end through host buffers (H2D inputs, D2H solution + test block)
    Ah = torch.empty_like(A, device="cpu").pin_memory()
    Kteh = torch.empty_like(Kte, device="cpu").pin_memory()
    e2e_ms = []
    for k in range(max(1, args.e2e_steps)):
        flush.zero_()
        barrier()
        a, b = ev(), ev()
        a.record(stream)
        Xd = Xh.to(dev, non_blocking=True)
        Yd = Yh.to(dev, non_blocking=True)
        step(Xd, Yd)
        Ah.copy_(A, non_blocking=True)
        Kteh.copy_(Kte, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_val = replica_throughput(world, entries, max_over_ranks(statistics.mean(e2e_ms), dist, dev) / 1e3)

    # ---- kernel-only roofline of the fused Myrtle kernel
    ops_entry = algorithmic_ops_per_entry(hw)
    blk_s = statistics.mean(blk_ms) / 1e3
    # the block interval holds the two fused launches (for the tiled form each
    # after its workspace clear, about 50 MB here)
    achieved_tops = ops_entry * entries / blk_s / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    run_clock = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak_tops, peak_source = fp32_peak(sm_count, run_clock)
    traffic, traffic_src = headline_traffic(args.config, variant)

    # ---- plain layer-wise forms on sample tiles, at equal accuracy
    extra = {}
    if not args.skip_plain:
        q = h.self_diag(X, CONVS, SW2, SB2)
        # rows [0, tile) against columns [tile, 2 tile): both inside the
        # n_tr + n_te images (the small profiling configs have 80)
        tile = min(64, n_tr, (n_tr + n_te) // 2)
        res = {}
        for prec, t in [("mixed", tile), ("plain_fp32", tile), ("plain_fp64", min(16, n_tr))]:
            out = torch.empty((t, t), dtype=torch.float64 if prec == "plain_fp64" else torch.float32,
                              device=dev)
            # the same pairs for every form: rows [0, t), columns [tile, tile + t)
            h.block(X, q, X, q, CONVS, SW2, SB2, prec=prec, a_range=(0, t), b_range=(tile, tile + t),
                    out=out)
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            h.block(X, q, X, q, CONVS, SW2, SB2, prec=prec, a_range=(0, t), b_range=(tile, tile + t),
                    out=out)
            b.record(stream)
            torch.cuda.synchronize()
            res[prec] = (t * t / (a.elapsed_time(b) / 1e3), out.double().cpu())
        k16 = res["plain_fp64"][1]
        extra["plain_fp32_entries_per_s"] = res["plain_fp32"][0]
        extra["plain_fp64_entries_per_s"] = res["plain_fp64"][0]
        extra["mixed_tile_entries_per_s"] = res["mixed"][0]
        extra["mixed_over_plain_fp32"] = res["mixed"][0] / res["plain_fp32"][0]
        extra["maxrel_mixed_vs_plain_fp64"] = float(((res["mixed"][1][:16, :16] - k16).abs() / k16.abs()).max())
        extra["maxrel_plain_fp32_vs_plain_fp64"] = float(((res["plain_fp32"][1][:16, :16] - k16).abs()
                                                          / k16.abs()).max())
        extra["plain_tiles"] = f"{tile}x{tile} (fp32, mixed), 16x16 (fp64) train pairs"
        # NTK (layer-wise FP32) on the same tile
        h.block_ntk(X, q, X, q, CONVS, SW2, SB2, prec="plain_fp32", a_range=(0, tile), b_range=(tile, 2 * tile))
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        Kn, Tn = h.block_ntk(X, q, X, q, CONVS, SW2, SB2, prec="plain_fp32", a_range=(0, tile),
                             b_range=(tile, 2 * tile))
        b.record(stream)
        torch.cuda.synchronize()
        extra["ntk_plain_fp32_entries_per_s"] = tile * tile / (a.elapsed_time(b) / 1e3)
        # fused NTK (the tiled row stream carrying Theta beside K): the same
        # tile for accuracy against the layer-wise form, a symmetric
        # 256-image block for the rate
        Km, Tm = h.block_ntk(X, q, X, q, CONVS, SW2, SB2, prec="mixed", a_range=(0, tile),
                             b_range=(tile, 2 * tile))
        nsym = min(256, n_tr)
        h.block_ntk(X, q, X, q, CONVS, SW2, SB2, prec="mixed", a_range=(0, nsym), b_range=(0, nsym), symmetric=True)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        h.block_ntk(X, q, X, q, CONVS, SW2, SB2, prec="mixed", a_range=(0, nsym), b_range=(0, nsym), symmetric=True)
        b.record(stream)
        torch.cuda.synchronize()
        h.sync_status()
        extra["ntk_mixed_entries_per_s"] = nsym * (nsym + 1) / 2 / (a.elapsed_time(b) / 1e3)
        extra["ntk_mixed_over_plain_fp32"] = extra["ntk_mixed_entries_per_s"] / extra["ntk_plain_fp32_entries_per_s"]
        extra["ntk_mixed_workload"] = f"myrtle5_(2,1,0)_32x32_ntk_symmetric{nsym}_mixed_tiled"
        # Myrtle-10 (3,3,3) on the same images: NNGP and NTK in the three-stage tiled form
        c10, sb10 = (3, 3, 3), 0.01
        q10 = h.self_diag(X, c10, SW2, sb10)
        for key, fn in (("myrtle10_mixed_entries_per_s",
                         lambda: h.block(X, q10, X, q10, c10, SW2, sb10, prec="mixed", a_range=(0, nsym),
                                         b_range=(0, nsym), symmetric=True)),
                        ("ntk10_mixed_entries_per_s",
                         lambda: h.block_ntk(X, q10, X, q10, c10, SW2, sb10, prec="mixed", a_range=(0, nsym),
                                             b_range=(0, nsym), symmetric=True))):
            fn()
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            extra[key] = nsym * (nsym + 1) / 2 / (a.elapsed_time(b) / 1e3)
        h.sync_status()
        extra["myrtle10_workload"] = f"myrtle10_(3,3,3)_32x32_symmetric{nsym}_sb2_0.01_mixed_tiled"
        # the 64x64 problem of the mixed-resolution workload in the layer-wise
        # FP32 form, on a 16 x 16 sample of pairs (the fused form: queue leg)
        x64 = nkdata.standardise(nkdata.images(32, 64, 3, nkdata.SEED_TRAIN, blur=True))[0]
        X64 = torch.tensor(x64.astype(np.float32), device=dev)
        q64 = h.self_diag(X64, CONVS, SW2, SB2)
        h.block(X64, q64, X64, q64, CONVS, SW2, SB2, prec="plain_fp32", a_range=(0, 2), b_range=(16, 18))
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        h.block(X64, q64, X64, q64, CONVS, SW2, SB2, prec="plain_fp32", a_range=(0, 16), b_range=(16, 32))
        b.record(stream)
        torch.cuda.synchronize()
        r64 = 256 / (a.elapsed_time(b) / 1e3)
        extra["plain_fp32_64x64_entries_per_s"] = r64
        extra["plain_fp32_64x64_blocks_s_extrapolated"] = (512 * 513 // 2 + 128 * 512) / r64
        extra["ntk_over_nngp_mean"] = float((Tn.double() / Kn.double()).mean())
        extra["ntk_maxrel_mixed_vs_plain_fp32"] = float(((Tm.double() - Tn.double()).abs() / Tn.double().abs()).max())
        # PCG: mixed vs plain FP64 on the same train block, with the Jacobi
        # preconditioner of the configuration and with the paper's pivoted
        # Cholesky one (rank 100)
        h.pcg_set_rank(100)
        for pc, prec in [("jacobi", "mixed"), ("jacobi", "plain_fp64"), ("pivchol", "mixed"),
                         ("pivchol", "plain_fp64")]:
            a, b = ev(), ev()
            a.record(stream)
            _, its, rel = h.pcg_solve(Ktr, Y, -REL_LAMBDA, precond=pc, prec=prec, tol=1e-6,
                                      maxit=20000, A=A, allow_not_converged=True)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            key = f"pcg_{prec}" if pc == "jacobi" else f"pcg_pivchol100_{prec}"
            extra[f"{key}_iters"] = its
            extra[f"{key}_ms"] = ms
            extra[f"{key}_iters_per_s"] = its / (ms / 1e3)
            extra[f"{key}_relres"] = max(rel)
    lam_used = h.last_lambda()
    if not args.skip_plain:
        extra.update(config1_leg(h, dev))
        extra.update(erf_leg(h, dev))
        extra.update(cv8_leg(h, dev))
    if not args.skip_grad:
        extra.update(grad_leg(h, dev, args.grad_support, args.grad_targets))
    if not args.skip_queue:
        extra.update(queue_leg(h, dev))
    if not args.skip_fc:
        extra.update(fc_leg(h, dev, load_peaks(), args.fc_train, args.fc_test))

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"myrtle5_(2,1,0)_{hw}x{hw}_train{n_tr}_test{n_te}_pcg10rhs",
                   "entries_per_step": entries, "parallelism": f"replicas{world}",
                   "precision": "FP64 self-variances, FP32 on-chip recursion, FP64 combine; "
                                "PCG FP32 matvec + FP64 scalars + FP64 refinement",
                   "l2": "256 MB buffer written between timed steps"},
        "pcg_iters_per_s": statistics.mean(iters) / (statistics.mean(pcg_ms) / 1e3),
        "pcg_l2": pcg_l2_roofline(n_tr, statistics.mean(iters), statistics.mean(pcg_ms) / 1e3),
        "pcg_iters": iters[-1],
        "pcg_relres": rels[-1],
        "lambda": lam_used,
        "breakdown_ms": {"self_diag": statistics.mean(sd_ms), "blocks": statistics.mean(blk_ms),
                         "pcg": statistics.mean(pcg_ms)},
        "kernel_only_entries_per_s": entries / blk_s,
        "fused_variant": variant,
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "TFLOP/s",
                     "frac": achieved_tops / peak_tops, "traffic": traffic, "traffic_source": traffic_src,
                     "kernel": "k_myrtle_tiled" if variant == 3 else "k_myrtle_fused",
                     "peak_source": peak_source, "ops_per_entry": ops_entry},
        "e2e": {"value": e2e_val, "unit": "entries/s",
                "h2d_bytes_per_step": Xh.numel() * 4 + Yh.numel() * 8,
                "d2h_bytes_per_step": Ah.numel() * 8 + Kteh.numel() * 4},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "cpu_pcg_baseline": cpu_pcg,
    }
    line.update(extra)
    # the figures the metric compares, last in the line (a truncated tail of
    # the output keeps them)
    keys = ["mixed_over_plain_fp32", "plain_fp32_entries_per_s", "plain_fp64_entries_per_s", "pcg_iters_per_s",
            "pcg_mixed_iters_per_s", "pcg_plain_fp64_iters_per_s", "fc3_gram_ms", "grad_backward_s",
            "queue_graph_ms", "erf_entries_per_s", "cv8_entries_per_s", "config1_entries_per_s", "ntk_mixed_entries_per_s", "ntk10_mixed_entries_per_s"]
    line["summary"] = {"value": value, "e2e": e2e_val, "roofline_frac": achieved_tops / peak_tops,
                       **{k: line.get(k) for k in keys if k in line}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def pcg_l2_roofline(n: int, iters: float, seconds: float) -> dict:
    """The headline solve's K (n^2 FP32, 16 MB at n = 2048) stays in L2: K
    bytes per CG iteration x iterations / solve time (refinement sweeps
    included), against the probed L2 read bandwidth."""
    gbs = 4.0 * n * n * iters / seconds / 1e9
    peak = load_probe().get("l2_read_GBs")
    return {"bound": "l2", "achieved": gbs, "unit": "GB/s", "peak": peak, "frac": gbs / peak if peak else None,
            "note": "K bytes per iteration / whole-solve time against the probed L2 read bandwidth; the "
                    "iteration is latency-bound at this size (four dependent launches)"}


def adjoint_layerwise_bytes(convs, hw: int, esize: int = 4, input_sides: int = 2) -> int:
    """Bytes the layer-fused adjoint (nk_block_backward, FP32) moves through
    HBM per image pair (E_s = (hw / 2^s)^4 elements at stage s).  Forward:
    the first layer writes its pre-activation (the input covariance is formed
    on load), every later layer reads the previous one (mapped on load) and
    writes its own, each pool reads the previous stage's last tensor and
    writes the pooled one, the readout reads the last.  Reverse, per layer:
    the stored pre-activation, the incoming gradient (none for the readout's
    constant, the next stage's tensor through the pool adjoint, else this
    stage's) and the outgoing gradient, plus the q-term partial sums (two
    H^2 W buffers written and read); the input adjoints read the last
    gradient once per image set that needs a gradient (input_sides, 2 or 1).
    Stage patterns without empty middle stages."""
    last = max(s for s, n in enumerate(convs) if n > 0)
    E = [(hw >> s) ** 4 for s in range(last + 1)]
    Wd = [hw >> s for s in range(last + 1)]
    tot = 0
    first = True
    for s in range(last + 1):
        if s > 0:
            tot += E[s - 1] + E[s]
        for _ in range(convs[s]):
            tot += E[s] if first else 2 * E[s]
            first = False
    tot += E[last]
    const = True
    for s in range(last, -1, -1):
        for k in range(convs[s] - 1, -1, -1):
            tot += 2 * E[s] + 4 * E[s] // Wd[s]
            if const:
                const = False
            elif k == convs[s] - 1:
                tot += E[s + 1]
            else:
                tot += E[s]
    tot += input_sides * E[0]
    return esize * tot


def adjoint_roofline(seconds: float, pairs_two: int, pairs_one: int, peaks: dict, convs=(3, 3, 3),
                     hw: int = 32) -> dict:
    """Achieved HBM bandwidth of the layer-wise adjoint under the traffic
    model above (pairs_two pairs with both input gradients, pairs_one with
    one), against the measured copy bandwidth."""
    per_pair = adjoint_layerwise_bytes(convs, hw)
    tot = per_pair * pairs_two + adjoint_layerwise_bytes(convs, hw, input_sides=1) * pairs_one
    gbs = tot / seconds / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "bytes_per_pair": per_pair, "traffic": None,
            "note": "layer-fused traffic model (adjoint_layerwise_bytes) x pairs / backward time, against the "
                    "measured copy bandwidth; the passes are issue-bound, not bandwidth-bound"}


def grad_leg(h, dev, n_sup=100, n_tgt=2048):
    """Myrtle-10 kernel-ridge support-set loss, 100 support x 2048 target
    32x32 images (same generator; n_sup, n_tgt shrink it for profiling),
    sigma_w^2 = 2, sigma_b^2 = 0.01: forward
    blocks K_ss (upper triangle) and K_ts by the fused kernel, loss in torch,
    gradients w.r.t. the support pixels, sigma_w^2 and sigma_b^2 by the FP32
    layer-wise adjoint.  A small untimed warm-up (4 x 8) and an untimed pass of
    the loss's linear algebra at the timed shapes, then one timed pass."""
    import numpy as np
    import torch

    import nkdata
    from paper_2303_05420_gb300.api import nngp_block

    convs = (3, 3, 3)
    sup = nkdata.standardise(nkdata.images(100, 32, 3, nkdata.SEED_SUPPORT, blur=True))[0]
    tgt = nkdata.standardise(nkdata.images(2048, 32, 3, nkdata.SEED_TEST, blur=True))[0]
    ys = torch.tensor(nkdata.labels(100, 10), device=dev)
    yt = torch.tensor(nkdata.labels(2048, 10, seed=9), device=dev)
    Xt = torch.tensor(tgt.astype(np.float32), device=dev)
    h.autotune(convs, 2.0, 0.01, 32, 32, 3)

    def once(ns, nt):
        Xs = torch.tensor(sup[:ns].astype(np.float32), device=dev, requires_grad=True)
        s = torch.tensor(2.0, dtype=torch.float64, device=dev, requires_grad=True)
        b = torch.tensor(0.01, dtype=torch.float64, device=dev, requires_grad=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        Kss = nngp_block(Xs, Xs, s, b, convs, h, symmetric=True, prec="mixed", bprec="plain_fp32").double()
        Kts = nngp_block(Xt[:nt], Xs, s, b, convs, h, prec="mixed", bprec="plain_fp32").double()
        lam = 1e-6 * float(torch.trace(Kss.detach())) / ns
        A = torch.linalg.solve(Kss + lam * torch.eye(ns, dtype=torch.float64, device=dev), ys[:ns])
        L = 0.5 * ((Kts @ A - yt[:nt]) ** 2).mean()
        ev[1].record()
        L.backward()
        ev[2].record()
        torch.cuda.synchronize()
        return (float(L.detach()), float(s.grad), float(b.grad), ev[0].elapsed_time(ev[1]) / 1e3,
                ev[1].elapsed_time(ev[2]) / 1e3)

    once(4, 8)  # loads every kernel; untimed
    # the first torch.linalg.solve / matmul at a new shape loads its library
    # kernels (about 2 s on this machine), so the loss's linear algebra is run
    # once, untimed, at the timed shapes
    Ad = torch.linalg.solve(torch.eye(n_sup, dtype=torch.float64, device=dev), ys[:n_sup])
    _ = (0.5 * ((torch.zeros((n_tgt, n_sup), dtype=torch.float64, device=dev) @ Ad - yt[:n_tgt]) ** 2).mean())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, gs, gb, t_fwd, t_bwd = once(n_sup, n_tgt)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    entries = n_sup * (n_sup + 1) // 2 + n_tgt * n_sup
    return {"grad_workload": f"myrtle10_(3,3,3)_32x32_support{n_sup}_target{n_tgt}_krr_loss_fp32_adjoint",
            f"grad_myrtle10_{n_sup}x{n_tgt}_s": dt, "grad_entries_per_s": entries / dt,
            "grad_forward_s": t_fwd, "grad_backward_s": t_bwd,
            "grad_backward_entries_per_s": entries / t_bwd,
            # K_ss: both input gradients (one image set); K_ts: the support side only
            "grad_adjoint_hbm": adjoint_roofline(t_bwd, n_sup * (n_sup + 1) // 2, n_tgt * n_sup, load_peaks()),
            "grad_loss": L, "grad_dsw2": gs, "grad_dsb2": gb}


def queue_leg(h, dev):
    """The mixed-resolution workload at full size: 512 train + 128 test 64x64
    images (blur generator) and their 2x2-average 32x32 companions, Myrtle-5
    (2,1,0), sigma_w^2 = 2, sigma_b^2 = 0, 200 classes.  The four blocks
    (train upper triangle and test block at each resolution) run as ONE
    persistent launch of the tiled form, timed once directly (its first call
    also sizes the slot workspace) and once as a replay of a CUDA graph
    holding it; then the 200-right-hand-side MIXED PCG solve of the 64x64
    train block."""
    import numpy as np
    import torch

    import nkdata

    n_tr, n_te = 512, 128
    prob = nkdata.image_problem(n_tr, n_te, 64, n_classes=200, blur=True)
    x64 = np.concatenate([prob.x_train, prob.x_test]).astype(np.float32)
    x32 = nkdata.downsample2(np.concatenate([prob.x_train, prob.x_test])).astype(np.float32)
    X64 = torch.tensor(x64, device=dev)
    X32 = torch.tensor(x32, device=dev)
    q64 = h.self_diag(X64, CONVS, SW2, SB2)
    q32 = h.self_diag(X32, CONVS, SW2, SB2)
    tasks = []
    for X, q in ((X64, q64), (X32, q32)):
        tasks.append(dict(Xa=X, qa=q, Xb=X, qb=q, a_range=(0, n_tr), b_range=(0, n_tr), symmetric=True,
                          out=torch.empty((n_tr, n_tr), dtype=torch.float32, device=dev)))
        tasks.append(dict(Xa=X, qa=q, Xb=X, qb=q, a_range=(n_tr, n_tr + n_te), b_range=(0, n_tr),
                          out=torch.empty((n_te, n_tr), dtype=torch.float32, device=dev)))
    per_res = n_tr * (n_tr + 1) // 2 + n_te * n_tr
    entries = 2 * per_res
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    h.block_queue(tasks, CONVS, SW2, SB2)
    b.record(stream)
    torch.cuda.synchronize()
    h.sync_status()
    t_direct = a.elapsed_time(b) / 1e3
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        h.block_queue(tasks, CONVS, SW2, SB2)
    a, b = ev(), ev()
    a.record(stream)
    g.replay()
    b.record(stream)
    torch.cuda.synchronize()
    h.sync_status()
    t_graph = a.elapsed_time(b) / 1e3
    Y = torch.tensor(prob.y_train, device=dev)
    a, b = ev(), ev()
    a.record(stream)
    _, its, rel = h.pcg_solve(tasks[0]["out"], Y, -REL_LAMBDA, precond="jacobi", prec="mixed", tol=1e-6,
                              maxit=20000, allow_not_converged=True)
    b.record(stream)
    torch.cuda.synchronize()
    # equivalent 32x32 work: a 64x64 entry is 16 times a 32x32 entry
    return {"queue_workload": "myrtle5_(2,1,0)_64x64+32x32_train512_test128_200cls_one_launch_tiled",
            "queue_entries": entries, "queue_direct_ms": 1e3 * t_direct, "queue_graph_ms": 1e3 * t_graph,
            "queue_entries_per_s": entries / t_graph,
            "queue_32x32_equivalent_entries_per_s": 17 * per_res / t_graph,
            "queue_pcg200_iters": its, "queue_pcg200_ms": a.elapsed_time(b),
            "queue_pcg200_relres": max(rel)}


def config1_leg(h, dev):
    """The small FP64 configuration: Myrtle-5 (2,1,0), sigma_w^2 = 2,
    sigma_b^2 = 0, 128 train + 32 test 8x8x3 images (N(0,1), standardised per
    channel), 10 classes (one-hot minus 0.1): the full 128 x 128 and 32 x 128
    blocks in PLAIN_FP64 and the FP64 Jacobi PCG solve with lambda =
    1e-4 tr(K)/N.  One untimed warm-up, then one timed pass."""
    import numpy as np
    import torch

    import nkdata

    prob = nkdata.image_problem(128, 32, 8, n_classes=10, blur=False)
    X = torch.tensor(np.concatenate([prob.x_train, prob.x_test]).astype(np.float32), device=dev)
    Y = torch.tensor(prob.y_train, device=dev)
    stream = torch.cuda.current_stream()

    def once():
        q = h.self_diag(X, CONVS, SW2, SB2)
        Ktr = h.block(X, q, X, q, CONVS, SW2, SB2, prec="plain_fp64", a_range=(0, 128), b_range=(0, 128))
        Kte = h.block(X, q, X, q, CONVS, SW2, SB2, prec="plain_fp64", a_range=(128, 160), b_range=(0, 128))
        return Ktr, Kte

    Ktr, _ = once()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    Ktr, Kte = once()
    ev[1].record(stream)
    K32 = Ktr.float().contiguous()
    _, its, rel = h.pcg_solve(K32, Y, -REL_LAMBDA, precond="jacobi", prec="plain_fp64", tol=1e-6, maxit=20000,
                              allow_not_converged=True)
    ev[2].record(stream)
    torch.cuda.synchronize()
    t_blk = ev[0].elapsed_time(ev[1]) / 1e3
    t_pcg = ev[1].elapsed_time(ev[2]) / 1e3
    return {"config1_workload": "myrtle5_(2,1,0)_8x8_train128_test32_fp64_full_blocks_jacobi_pcg",
            "config1_entries_per_s": (128 * 128 + 32 * 128) / t_blk, "config1_blocks_ms": 1e3 * t_blk,
            "config1_pcg_iters": its, "config1_pcg_iters_per_s": its / t_pcg, "config1_pcg_relres": max(rel)}


def erf_leg(h, dev):
    """The Erf activation (the tuned-Myrtle options) on the headline workload:
    Myrtle-5 (2,1,0) with Erf, sigma_w^2 = 2, sigma_b^2 = 0, the 2048-image
    symmetric train block in the tiled fused form (MIXED)."""
    import numpy as np
    import torch

    import nkdata

    prob = nkdata.image_problem(2048, 512, 32, n_classes=10, blur=True)
    X = torch.tensor(prob.x_train.astype(np.float32), device=dev)
    q = h.self_diag(X, CONVS, SW2, SB2, act="erf")
    K = torch.empty((2048, 2048), dtype=torch.float32, device=dev)
    h.block(X, q, X, q, CONVS, SW2, SB2, prec="mixed", act="erf", symmetric=True, a_range=(0, 256),
            b_range=(0, 256), out=K[:256, :256])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    h.block(X, q, X, q, CONVS, SW2, SB2, prec="mixed", act="erf", symmetric=True, out=K)
    b.record()
    torch.cuda.synchronize()
    h.sync_status()
    t = a.elapsed_time(b) / 1e3
    return {"erf_workload": "myrtle5_(2,1,0)_erf_32x32_train2048_symmetric_mixed_tiled",
            "erf_entries_per_s": 2048 * 2049 / 2 / t, "erf_block_ms": 1e3 * t}


def cv8_leg(h, dev):
    """The CV8 listing (eight conv + ReLU layers, Flatten, Dense; sigma_w^2 = 2,
    sigma_b^2 = 0.01) on the headline images: the 2048 symmetric train block
    and the 512 x 2048 test block by the diagonal recursion (MIXED), and the
    layer-wise FP32 form on a 16 x 16 sample for comparison."""
    import numpy as np
    import torch

    import nkdata

    prob = nkdata.image_problem(2048, 512, 32, n_classes=10, blur=True)
    X = torch.tensor(np.concatenate([prob.x_train, prob.x_test]).astype(np.float32), device=dev)
    convs, sb2 = (8,), 0.01
    q = h.self_diag(X, convs, SW2, sb2)
    Ktr = torch.empty((2048, 2048), dtype=torch.float32, device=dev)
    Kte = torch.empty((512, 2048), dtype=torch.float32, device=dev)

    def blocks():
        h.block(X, q, X, q, convs, SW2, sb2, prec="mixed", readout="flatten", a_range=(0, 2048),
                b_range=(0, 2048), symmetric=True, out=Ktr)
        h.block(X, q, X, q, convs, SW2, sb2, prec="mixed", readout="flatten", a_range=(2048, 2560),
                b_range=(0, 2048), out=Kte)

    blocks()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    blocks()
    ev[1].record()
    ev[2].record()
    Kp = h.block(X, q, X, q, convs, SW2, sb2, prec="plain_fp32", readout="flatten", a_range=(0, 16),
                 b_range=(16, 32))
    ev[3].record()
    torch.cuda.synchronize()
    h.sync_status()
    t = ev[0].elapsed_time(ev[1]) / 1e3
    tp = ev[2].elapsed_time(ev[3]) / 1e3
    entries = 2048 * 2049 // 2 + 512 * 2048
    # FP32 operations of the diagonal recursion per entry: per pixel and layer
    # the vertical and horizontal 3-tap sums (4 adds), the scale and bias (1),
    # the factor products and the scaled map output (2 + 3) and the map
    # (J01: a degree-5 polynomial, a square root and the combine, about 10),
    # plus C = 3 contraction FMAs per pixel; the same count as DESIGN's
    # H W (8 + 9 + 12) per layer, rounded to 29 + 3 C / L
    ops = 32 * 32 * (8 * 29 + 3)
    props = torch.cuda.get_device_properties(dev)
    peak, src = fp32_peak(props.multi_processor_count, 2070.0)
    achieved = ops * entries / t / 1e12
    return {"cv8_workload": "cv8_relu_32x32_train2048_test512_flatten_mixed_diagonal",
            "cv8_entries_per_s": entries / t, "cv8_blocks_ms": 1e3 * t,
            "cv8_roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "ops_per_entry": ops, "peak_source": src},
            "cv8_plain_fp32_entries_per_s": 256 / tp,
            "cv8_maxrel_mixed_vs_plain_fp32": float(((Ktr[:16, 16:32] - Kp).abs() / Kp.abs()).max())}


def probe_peaks(path: str):
    """Measures the peak rates the roofline fractions divide by (nk_probe:
    FP32 and FP64 FMA issue, L2-resident and HBM reads) with the SM clocks
    sampled during the probes, and writes them per SM and cycle to `path`."""
    import torch

    from paper_2303_05420_gb300.api import probe

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    sm = props.multi_processor_count
    probe("fp32_fma", 1 << 10)  # context and module load
    sampler = ClockSampler(0)
    sampler.start()
    res = {}
    for name in ("fp32_fma", "fp64_fma", "l2_read", "hbm_read"):
        best = (0.0, 0.0)
        for _ in range(3):
            r, ms = probe(name)
            if r > best[0]:
                best = (r, ms)
        res[name] = best
    torch.cuda.synchronize()
    clocks = sampler.stop()
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    out = {"gpu": props.name, "sm_count": sm, "clocks": clocks,
           "fp32_fma_per_s": res["fp32_fma"][0], "fp64_fma_per_s": res["fp64_fma"][0],
           "l2_read_GBs": res["l2_read"][0] / 1e9, "hbm_read_GBs": res["hbm_read"][0] / 1e9,
           "fp32_fma_per_sm_per_cycle": res["fp32_fma"][0] / (sm * mhz * 1e6) if mhz else None,
           "fp64_fma_per_sm_per_cycle": res["fp64_fma"][0] / (sm * mhz * 1e6) if mhz else None,
           "how": "nk_probe (CUDA events, best of 3 after a warm-up): 8 independent FMA chains per thread at "
                  "2048 threads per SM; float4 reads bypassing L1 of a 32 MB (L2) and a 1 GB (HBM) buffer; "
                  "per-cycle rates divide by the median SM clock sampled during the probes"}
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out), flush=True)


FC_N_TRAIN, FC_N_TEST, FC_D, FC_DEPTH = 50000, 10000, 3072, 3
FC_SW2, FC_SB2 = 2.0, 0.01  # the FC3 listing's W_std = sqrt 2, b_std = 0.1


def fc_leg(h, dev, peaks, n=FC_N_TRAIN, m=FC_N_TEST):
    """Depth-3 fully-connected ReLU NNGP (sigma_w^2 = 2, sigma_b^2 = 0.01) on
    3072-dim N(0,1) rows scaled to norm sqrt(d): the 50000 x 50000 train Gram (upper triangle, mirrored)
    and the 10000 x 50000 test block by the split-BF16 tensor-core kernel
    with the fused arc-cosine recursion, then the PCG ridge solve of the
    10 GB train kernel (10 right-hand sides, lambda = 1e-4 tr(K)/N), mixed
    and plain FP64.  Inputs are resident in HBM; one untimed warm-up."""
    import numpy as np
    import torch

    import nkdata

    d = FC_D
    xtr = torch.tensor(nkdata.fc_rows(n, d, nkdata.SEED_TRAIN), dtype=torch.float32, device=dev)
    xte = torch.tensor(nkdata.fc_rows(m, d, nkdata.SEED_TEST), dtype=torch.float32, device=dev)
    Y = torch.tensor(nkdata.labels(n, 10), device=dev)
    Ktr = torch.empty((n, n), dtype=torch.float32, device=dev)
    Kte = torch.empty((m, n), dtype=torch.float32, device=dev)
    A = torch.empty((n, 10), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def grams():
        h.fc_block(xtr, xtr, FC_SW2, FC_SB2, FC_DEPTH, symmetric=True, out=Ktr)
        h.fc_block(xte, xtr, FC_SW2, FC_SB2, FC_DEPTH, out=Kte)

    grams()
    torch.cuda.synchronize()
    marks = [ev() for _ in range(3)]
    marks[0].record(stream)
    h.fc_block(xtr, xtr, FC_SW2, FC_SB2, FC_DEPTH, symmetric=True, out=Ktr)
    marks[1].record(stream)
    h.fc_block(xte, xtr, FC_SW2, FC_SB2, FC_DEPTH, out=Kte)
    marks[2].record(stream)
    torch.cuda.synchronize()
    t_sym = marks[0].elapsed_time(marks[1]) / 1e3
    t_te = marks[1].elapsed_time(marks[2]) / 1e3
    uniq = n * (n + 1) // 2 + m * n
    # algorithmic Gram flops: 2 d per unique entry; the split-BF16 form runs
    # three BF16 products per FP32 product on the tensor pipe
    alg = 2.0 * d * uniq
    t_gram = t_sym + t_te
    out = {"fc3_workload": f"fc3_relu_d{d}_train{n}_test{m}_pcg10rhs",
           "fc3_gram_ms": 1e3 * t_gram, "fc3_sym_ms": 1e3 * t_sym, "fc3_test_ms": 1e3 * t_te,
           "fc3_entries_per_s": uniq / t_gram,
           "fc3_roofline": {"bound": "tensor", "kernel": "k_fc_gram",
                            "achieved": alg / t_gram / 1e12, "unit": "TFLOP/s",
                            "tensor_pipe_tflops": 3 * alg / t_gram / 1e12,
                            "peak": peaks.get("bf16_tflops"),
                            "frac": (3 * alg / t_gram / 1e12) / peaks["bf16_tflops"]
                            if peaks.get("bf16_tflops") else None,
                            "frac_algorithmic": (alg / t_gram / 1e12) / peaks["bf16_tflops"]
                            if peaks.get("bf16_tflops") else None,
                            "note": "achieved = 2 d flops per unique entry (algorithmic); frac = "
                                    "tensor-pipe BF16 rate (3 products per split-BF16 entry) of measured "
                                    "burst bf16 peak; frac_algorithmic = achieved of the same peak"}}
    for prec in ["mixed", "plain_fp64"]:
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        _, its, rel = h.pcg_solve(Ktr, Y, -REL_LAMBDA, precond="jacobi", prec=prec, tol=1e-6,
                                  maxit=5000, A=A, allow_not_converged=True)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        out[f"fc3_pcg_{prec}_iters"] = its
        out[f"fc3_pcg_{prec}_ms"] = ms
        out[f"fc3_pcg_{prec}_iters_per_s"] = its / (ms / 1e3)
        out[f"fc3_pcg_{prec}_relres"] = max(rel)
    # the FP32 matvec streams K (n^2 x 4 bytes) once per iteration
    its = out["fc3_pcg_mixed_iters"]
    if its:
        gbs = its * n * n * 4 / (out["fc3_pcg_mixed_ms"] / 1e3) / 1e9
        out["fc3_pcg_mixed_hbm"] = {"achieved": gbs, "unit": "GB/s", "peak": peaks.get("hbm_gbs"),
                                    "frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                                    "note": "K bytes per CG iteration / whole-solve time (includes the "
                                            "FP64 true residuals of the refinement)"}
    # out of core: the same 10 GB kernel in pinned host memory, read by the
    # matvec over the chip-to-chip link
    del Kte
    Kh = torch.empty(Ktr.shape, dtype=torch.float32).pin_memory()
    Kh.copy_(Ktr)
    del Ktr
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    _, its, rel = h.pcg_solve(Kh, Y, -REL_LAMBDA, precond="jacobi", prec="mixed", tol=1e-6, maxit=5000, A=A,
                              allow_not_converged=True)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out["fc3_pcg_hostK_mixed_iters"] = its
    out["fc3_pcg_hostK_mixed_ms"] = ms
    out["fc3_pcg_hostK_mixed_relres"] = max(rel)
    out["fc3_pcg_hostK_GBs"] = its * n * n * 4 / (ms / 1e3) / 1e9
    del Kh
    return out


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = CONFIGS[args.config]
    cores = host_cores()
    per_step = []
    for k in range(args.warmup + args.steps):
        rate, pairs, tmax, wall = cpu_oracle_rate(cores, args.ref_pairs, cfg["hw"], seed0=1000 + 97 * k)
        if k >= args.warmup:
            per_step.append((rate, pairs, tmax))
    value = statistics.mean(r for r, _, _ in per_step)
    n_tr, n_te = cfg["n_train"], cfg["n_test"]
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "entries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(t for _, _, t in per_step),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"myrtle5_(2,1,0)_{cfg['hw']}x{cfg['hw']}_train{n_tr}_test{n_te}_pcg10rhs",
                   "parallelism": "cpu_processes"},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step {cores * args.ref_pairs} pixel-pair recursions of the "
                                   f"workload's 32x32 Myrtle-5 kernel, {cores} spawned processes x 1 thread"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nk", choices=["nk", "reference"])
    ap.add_argument("--config", default="headline", choices=sorted(CONFIGS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-pairs", type=int, default=20)
    ap.add_argument("--ref-pairs", type=int, default=4)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused-variant", type=int, default=None,
                    help="pin the fused kernel's launch variant instead of autotuning it")
    ap.add_argument("--skip-queue", action="store_true",
                    help="skip the mixed-resolution block-queue leg")
    ap.add_argument("--skip-fc", action="store_true",
                    help="skip the depth-3 FC NNGP leg (50000 x 50000 Gram and its PCG solve)")
    ap.add_argument("--fc-train", type=int, default=FC_N_TRAIN)
    ap.add_argument("--fc-test", type=int, default=FC_N_TEST)
    ap.add_argument("--fc-only", action="store_true",
                    help="run only the FC leg (prints its keys as one JSON line)")
    ap.add_argument("--grad-support", type=int, default=100, help="support images of the gradient leg")
    ap.add_argument("--grad-targets", type=int, default=2048, help="target images of the gradient leg")
    ap.add_argument("--skip-grad", action="store_true",
                    help="skip the Myrtle-10 kernel-ridge gradient leg (100 support x 2048 targets)")
    ap.add_argument("--probe-peaks", default=None, metavar="PATH",
                    help="measure the peak rates (nk_probe) and write them to PATH as JSON, then exit")
    args = ap.parse_args()
    if args.probe_peaks:
        probe_peaks(args.probe_peaks)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.fc_only:
        import torch

        from paper_2303_05420_gb300.api import Handle

        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(dev)
        h = Handle()
        out = fc_leg(h, dev, load_peaks(), args.fc_train, args.fc_test)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
