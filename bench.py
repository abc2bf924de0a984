#!/usr/bin/env python3
"""Benchmark of volumetric field synthesis (voxels/s).

Workload: the single-wavelength sample -- 64 x 64 x 32 voxels of 0.25 um with
1-8 seeded ellipsoids (seed = rank), lit by a focused Gaussian beam (NA 0.5),
solved on the GPU at 21x21 orders (M = 441) -- synthesised on a 256 x 256 x 256
grid (8 planes per layer). A step is one scw_synthesize: phases (a), mode
contraction (b), pruned inverse FFT (c). W (597 MB) and the output (403 MB) are
both larger than the 129 MB L2, so no flush is needed between steps.

The line carries the metric's two arms on the same inputs -- split-BF16 tensor
cores (the headline value) and the FP32 SIMT contraction -- and, from the
oracle leg on rank 0, every voxel of both compared with the FP64 oracle's
direct sum (per-component rel-L2 and max-abs).

Prints ONE JSON line on rank 0. With --impl reference the FP64 CPU oracle is
timed instead (bounded sample of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

U_ORD, F_XY = 21, 256
L_LAYERS, PLANES_PER_LAYER = 32, 8   # overridable with --layers / --planes-per-layer (profiling cases)
LAM, X_PERIOD, DZ = 1.0, 16.0, 0.25


def workload_name():
    fz = L_LAYERS * PLANES_PER_LAYER
    return f"single_wavelength_21x21_orders_{L_LAYERS}_layers_256x256x{fz}"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.json), or None
    when the kernel's source changed since the capture or the workload differs."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except Exception:
        return None
    if not sha.startswith(rec["source_sha256_prefix"]) or rec["workload"] != workload:
        return None
    return rec["traffic_bytes_per_launch"]


def bf16_sustained():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except Exception:
        return 1700.0


def geometry():
    zb = np.arange(L_LAYERS + 1) * DZ
    Fz = L_LAYERS * PLANES_PER_LAYER
    zp = zb[0] + (np.arange(Fz) + 0.5) * ((zb[-1] - zb[0]) / Fz)
    return zb, zp


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
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
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---- replicas: every rank synthesises its own volume; no data-path collective ----
def replica_seed(rank: int) -> int:
    """Seed of a rank's synthetic layer set (independent replicas)."""
    return rank


def reduce_over_ranks(x: float, op: str, device) -> float:
    """MAX or SUM of a host scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX if op == "max" else tdist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units_local: float, seconds_local: float, device):
    """Whole-job throughput of independent replicas: the units all ranks processed
    over the slowest rank's time. Returns (value, max_seconds)."""
    total = reduce_over_ranks(units_local, "sum", device)
    slowest = reduce_over_ranks(seconds_local, "max", device)
    return total / slowest, slowest


def oracle_sample_rate(W, g, a, zb, zp, seconds=12.0, max_planes=None):
    """Voxels/s of the FP64 oracle (spectrum + direct sum) on whole planes of
    the same workload, planes taken in order until ~`seconds` elapse or
    `max_planes` planes are done (cycling through the volume)."""
    from oracle import cw, synth
    ls = cw.LayerSet(lam=LAM, X=X_PERIOD, Y=X_PERIOD, U=U_ORD, V=U_ORD, z_bounds=zb, W=W, gamma=g, alpha=a,
                     p_inc=None, p_ref=None, p_trn=None)
    xs, ys = synth.pixel_coords(ls, F_XY, F_XY)
    t0 = time.perf_counter()
    n = 0
    while True:
        z = zp[n % len(zp)]
        S = synth.spectrum_at(ls, float(z))
        synth.field_direct(ls, S, xs, ys)
        n += 1
        if (max_planes is not None and n >= max_planes) or time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return n * F_XY * F_XY / dt, n, dt


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
            if os.environ.get(k, "").isdigit():
                return min(int(os.environ[k]), os.cpu_count() or 1)
        return os.cpu_count() or 1


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import workloads as wl
    zb, zp = geometry()
    W, g, a, *_ = wl.random_layer_set(0, U_ORD, U_ORD, L_LAYERS)
    W = W.astype(np.complex128)
    for _ in range(args.warmup):
        oracle_sample_rate(W, g, a, zb, zp, seconds=0.0, max_planes=1)
    rates, planes = [], 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r, n, _ = oracle_sample_rate(W, g, a, zb, zp, seconds=0.0, max_planes=2)
        rates.append(r)
        planes += n
    dt = time.perf_counter() - t0
    value = planes * F_XY * F_XY / dt
    cores = blas_threads()
    line = {"impl": "reference", "metric": "field voxels/s", "value": value, "unit": "voxels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(), "orders": "21x21", "layers": L_LAYERS,
                                            "grid": [F_XY, F_XY, L_LAYERS * PLANES_PER_LAYER],
                                            "inputs": "synthetic layer sets of the sample's shapes (the oracle's "
                                                      "own solve of the 32 layers takes minutes; the synthesis cost "
                                                      "does not depend on the values)",
                                            "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": "2 whole 256x256 planes per step (spectrum + direct sum), FP64 NumPy"},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, dev, world, peaks_hbm):
    """Batched spectroscopic sweep: n wavenumbers in [1000, 1800] cm^-1, orders
    9x9 -> 25x25, 16 layers of 1 um, 128 x 128 x 64 voxels each, one
    scw_synthesize_batched call (one CUDA graph) per sweep."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    n = args.sweep_items
    items = []
    for i in range(n):
        lam, U, X, zb, zp, Fx, Fy = wl.sweep_geometry(i, n)
        items.append(dict(U=U, V=U, L=16, lam=lam, X=X, Y=X, z_bounds=zb, Fx=Fx, Fy=Fy, z_planes=zp))
    t0 = time.perf_counter()
    bp = scw.BatchedPlan(items, precision=args.precision, autotune=True)
    plan_s = time.perf_counter() - t0
    w_bytes = 0
    for i, kw in enumerate(items):
        W, g, a, *_ = wl.random_layer_set_torch(10_000 + i, kw["U"], kw["V"], 16, device=dev)
        bp.set_layers(i, W, g, a)
        torch.cuda.synchronize(dev)  # conversion done: W itself is not kept
        w_bytes += W.numel() * 8
        del W
    outs = [torch.empty(sh, dtype=torch.complex64, device=dev) for sh in bp.shapes]
    out_bytes = sum(o.numel() * 8 for o in outs)
    voxels = sum(sh[1] * sh[2] * sh[3] for sh in bp.shapes)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        bp.synthesize(outs)
    bp.check()
    steps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        bp.synthesize(outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    bp.check()
    ms = e0.elapsed_time(e1) / steps
    bp.enable_timing(True)
    for _ in range(3):
        bp.synthesize(outs)
    kt = bp.timings()
    bp.enable_timing(False)
    info = bp.info()
    roof_ms = (w_bytes + out_bytes) / (peaks_hbm * 1e9) * 1e3
    res = {"workload": f"sweep_{n}_wavenumbers_orders_9_to_25_16_layers_128x128x64", "items": n,
           "voxels_per_sweep": voxels, "ms_per_sweep": ms, "value": replica_throughput(voxels, ms * 1e-3, dev)[0],
           "unit": "voxels/s", "steps": steps, "graph": True,
           "algorithmic_bytes": w_bytes + out_bytes, "hbm_roofline_ms": roof_ms, "roofline_frac": roof_ms / ms,
           "contract_gbs": w_bytes / (kt["contract_ms"] * 1e-3) / 1e9,
           "kernel_ms": {k: kt[k] for k in ("phases_ms", "contract_ms", "xpass_ms", "ypass_ms", "total_ms")},
           "schedule": {k: info[k] for k in ("contract_ctas", "contract_tasks", "schedule_max_load",
                                             "schedule_mean_load")},
           "plan_create_s": plan_s, "tune": bp.tune_report()}
    bp.close()
    del outs
    return res


def run_illumination(args, dev, world, Wd, gd, zb, zp, hbm, bf16_tf, fxy=None, precisions=("split_bf16", "fp16", "fp32")):
    """Many illuminations of one solved sample: the single-wavelength workload
    (21x21 orders, 32 layers, fxy x fxy x 256 voxels, fxy = 256 by default) lit by I
    incident fields that share W and gamma, each with its own alpha (random draws
    of a solved alpha's distribution). One plan contracts all I against a single
    read of W, so the contraction has 8 I columns per layer and turns tensor-bound;
    every precision is timed on the same inputs."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    I = args.illuminations
    M = U_ORD * U_ORD
    fxy = fxy or F_XY
    alpha = wl.random_illuminations(4242, I, U_ORD, U_ORD, L_LAYERS)[0]
    ad = torch.from_numpy(alpha).to(dev)
    Fz = len(zp)
    voxels = I * fxy * fxy * Fz
    out = torch.empty((I, 3, Fz, fxy, fxy), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flops = 8.0 * (3 * M) * (4 * M) * Fz * I       # complex multiply-adds of S = W (alpha o g), 8 flops each
    products = {"fp32": 1, "split_bf16": 3, "fp16": 2}
    res = {"workload": f"single_wavelength_{fxy}x{fxy}x{Fz}_{I}_illuminations", "illuminations": I,
           "voxels_per_step": voxels, "contract_flops": flops, "unit": "voxels/s"}
    for prec in precisions:
        plan = scw.Plan(U_ORD, U_ORD, L_LAYERS, LAM, X_PERIOD, X_PERIOD, zb, fxy, fxy, zp,
                        precision=prec, illuminations=I)
        plan.set_layers(Wd, gd, ad)
        for _ in range(max(3, args.warmup)):
            plan.synthesize(out)
        plan.check()
        steps = max(3, min(args.steps, 10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            plan.synthesize(out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        plan.enable_timing(True)
        for _ in range(3):
            plan.synthesize(out)
        kt = plan.timings()
        plan.enable_timing(False)
        plan.check()
        tf = flops / (kt["contract_ms"] * 1e-3) / 1e12
        r = {"value": replica_throughput(voxels, ms * 1e-3, dev)[0], "ms_per_step": ms,
             "kernel_ms": {k: kt[k] for k in ("phases_ms", "contract_ms", "xpass_ms", "ypass_ms", "total_ms")},
             "contract_tflops": tf, "k_split": plan.info()["k_split"]}
        if prec != "fp32":
            r["tensor_frac_issued"] = tf * products[prec] / bf16_tf  # MMA flops issued / measured bf16 peak
        res[prec] = r
        plan.close()
    res["contract_speedup_split_bf16_vs_fp32"] = res["fp32"]["kernel_ms"]["contract_ms"] / \
        res["split_bf16"]["kernel_ms"]["contract_ms"]
    res["step_speedup_split_bf16_vs_fp32"] = res["fp32"]["ms_per_step"] / res["split_bf16"]["ms_per_step"]
    # the steps share everything but the contraction: (phases, recompose) cost the same on both paths
    rest = res["split_bf16"]["ms_per_step"] - res["split_bf16"]["kernel_ms"]["contract_ms"]
    res["common_ms"] = rest
    res["step_speedup_bound"] = (res["fp32"]["kernel_ms"]["contract_ms"] + rest) / \
        (res["split_bf16"]["kernel_ms"]["contract_ms"] + rest)
    res["out_bytes"] = out.numel() * 8
    res["step_hbm_roofline_ms"] = (L_LAYERS * 3 * M * 4 * M * 8 + res["out_bytes"]) / (hbm * 1e9) * 1e3
    res["peaks"] = {"bf16_tflops": bf16_tf, "hbm_gbs": hbm, "source": "MEASURED_PEAKS.json (burst)"}
    del out, ad
    return res


def run_points(args, dev, world, Wd, gd, ad, zb, zp, hbm, bf16_tf):
    """Field off the FFT grid on the single-wavelength workload (21x21 orders, 32
    layers, 256 planes): a zoomed 256 x 256 window of 4 x 4 um (points between the
    grid's pixels) and one x-z plane of 256 points, on every plane. The point
    product is a dense GEMM over the 441 orders; each precision is timed on the
    same inputs."""
    import torch
    import paper_2404_07293_gb300 as scw
    M = U_ORD * U_ORD
    Fz = len(zp)
    n = 256
    g = (np.arange(n) + 0.5) * (4.0 / n) + 6.0
    gx, gy = np.meshgrid(g, g)
    cases = {"window_256x256_of_4um": np.column_stack([gx.ravel(), gy.ravel()]),
             "xz_plane_256": np.column_stack([np.arange(n) * X_PERIOD / n, np.full(n, 0.5 * X_PERIOD)])}
    stream = torch.cuda.current_stream(dev)
    res = {"planes": Fz, "unit": "voxels/s", "peaks": {"bf16_tflops": bf16_tf, "source": "MEASURED_PEAKS.json (burst)"}}
    products = {"fp32": 1, "split_bf16": 3}
    for name, xy in cases.items():
        P = len(xy)
        flops = 8.0 * M * 3 * Fz * P  # complex multiply-adds of the point product, 8 flops each
        r = {"points": P, "voxels_per_step": P * Fz, "product_flops": flops}
        out = torch.empty((3, Fz, P), dtype=torch.complex64, device=dev)
        for prec in ("split_bf16", "fp32"):
            plan = scw.Plan(U_ORD, U_ORD, L_LAYERS, LAM, X_PERIOD, X_PERIOD, zb, F_XY, F_XY, zp, precision=prec)
            plan.set_layers(Wd, gd, ad)
            plan.set_points(xy)
            for _ in range(max(3, args.warmup)):
                plan.synthesize_points(out)
            plan.check()
            steps = max(3, min(args.steps, 10))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                plan.synthesize_points(out)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            plan.enable_timing(True)
            for _ in range(3):
                plan.synthesize_points(out)
            kt = plan.timings()
            plan.enable_timing(False)
            plan.check()
            tf = flops / (kt["ypass_ms"] * 1e-3) / 1e12
            q = {"value": replica_throughput(P * Fz, ms * 1e-3, dev)[0], "ms_per_step": ms,
                 "kernel_ms": {"phases_ms": kt["phases_ms"], "contract_ms": kt["contract_ms"],
                               "spectrum_operand_ms": kt["xpass_ms"], "point_product_ms": kt["ypass_ms"],
                               "total_ms": kt["total_ms"]},
                 "point_product_tflops": tf}
            if prec != "fp32":
                q["tensor_frac_issued"] = tf * products[prec] / bf16_tf
            r[prec] = q
            plan.close()
        r["point_product_speedup_split_bf16_vs_fp32"] = r["fp32"]["kernel_ms"]["point_product_ms"] / \
            r["split_bf16"]["kernel_ms"]["point_product_ms"]
        res[name] = r
        del out
    return res


def run_tiling(args, dev, world, Wd, gd, ad, zb, zp, hbm):
    """Large lateral fields from the single-wavelength workload (21x21 orders,
    32 layers, 256 planes of 256 x 256 per period):
      - periodic tiling: one unit cell stored to 4 x 4 periods (1024 x 1024 x 256);
      - patch mosaic: 4 x 4 different samples (one batched plan, one graph), each
        written as a 256 x 256 patch of one 1024 x 1024 x 256 field (strided views).
    Both write 6.4 GB per step."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    Fz, n = len(zp), 4
    H = W = n * F_XY
    stream = torch.cuda.current_stream(dev)
    mosaic = torch.empty((3, Fz, H, W), dtype=torch.complex64, device=dev)
    out_bytes = mosaic.numel() * 8
    M = U_ORD * U_ORD
    w_bytes = L_LAYERS * 3 * M * 4 * M * 8

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    steps = max(3, min(args.steps, 10))
    res = {"unit": "voxels/s", "voxels_per_step": H * W * Fz, "out_bytes": out_bytes}
    plan = scw.Plan(U_ORD, U_ORD, L_LAYERS, LAM, X_PERIOD, X_PERIOD, zb, F_XY, F_XY, zp, precision=args.precision,
                    tiles=(n, n))
    plan.set_layers(Wd, gd, ad)
    ms = timed(lambda: plan.synthesize(mosaic), steps)
    plan.check()
    plan.enable_timing(True)
    for _ in range(3):
        plan.synthesize(mosaic)
    kt = plan.timings()
    plan.enable_timing(False)
    plan.close()
    roof = (w_bytes + out_bytes) / (hbm * 1e9) * 1e3
    res["periodic_4x4"] = {"value": replica_throughput(H * W * Fz, ms * 1e-3, dev)[0], "ms_per_step": ms,
                           "ypass_ms": kt["ypass_ms"], "ypass_write_gbs": out_bytes / (kt["ypass_ms"] * 1e-3) / 1e9,
                           "hbm_roofline_ms": roof, "roofline_frac": roof / ms}
    items = [dict(U=U_ORD, V=U_ORD, L=L_LAYERS, lam=LAM, X=X_PERIOD, Y=X_PERIOD, z_bounds=zb, Fx=F_XY, Fy=F_XY,
                  z_planes=zp, out_ld=W, out_plane_stride=H * W) for _ in range(n * n)]
    bp = scw.BatchedPlan(items, precision=args.precision)
    for i in range(n * n):
        Wi, gi, ai, *_ = wl.random_layer_set_torch(20_000 + i, U_ORD, U_ORD, L_LAYERS, device=dev)
        bp.set_layers(i, Wi, gi, ai)
        torch.cuda.synchronize(dev)
        del Wi
    views = [mosaic[:, :, (i // n) * F_XY:(i // n + 1) * F_XY, (i % n) * F_XY:(i % n + 1) * F_XY]
             for i in range(n * n)]
    ms = timed(lambda: bp.synthesize(views), steps)
    bp.check()
    bp.close()
    roof = (n * n * w_bytes + out_bytes) / (hbm * 1e9) * 1e3
    res["mosaic_4x4_patches"] = {"value": replica_throughput(H * W * Fz, ms * 1e-3, dev)[0], "ms_per_step": ms,
                                 "hbm_roofline_ms": roof, "roofline_frac": roof / ms}
    del mosaic
    return res


def solve_sample(dev, seed, L):
    """The single-wavelength sample (64 x 64 x L voxels of 0.25 um, seeded ellipsoids,
    focused Gaussian beam at NA 0.5) solved on the GPU at 21 x 21 orders. The first
    solve also creates the solver's library handles. Returns (problem, solver, n,
    p_inc, (W, gamma, alpha), seconds)."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    p = wl.config_single_wavelength(seed, U=U_ORD, L=L)
    n = torch.from_numpy(p.n_volume.astype(np.complex128)).to(dev)
    img = torch.from_numpy(p.incident_image.astype(np.complex128)).to(dev)
    t0 = time.perf_counter()
    s = scw.Solver(p.U, p.V, L, p.lam, p.X, p.Y, p.z_bounds, p.n_volume.shape[2], p.n_volume.shape[1])
    p_inc = s.incident(img)
    W, g, a, _, _ = s.solve(n, p_inc)
    torch.cuda.synchronize(dev)
    return p, s, n, p_inc, (W, g, a), time.perf_counter() - t0


def run_solve(args, dev, with_oracle, p, s, n, p_inc):
    """The solve stage on the GPU for the single-wavelength sample itself: 64 x 64 x 32
    voxels of 0.25 um with seeded ellipsoids, a focused Gaussian beam (NA 0.5), 21 x 21
    orders (4M = 1764 modes per layer). Times a second solve on the already warmed-up
    solver and reports, beside it, the FP64 oracle timed on one layer of the same
    sample (its eigendecomposition of D and its connection step), scaled to the layers."""
    import torch
    L = len(p.z_bounds) - 1
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    W, g, a, pr, pt = s.solve(n, p_inc)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    t = s.times()
    N4 = 4 * p.U * p.V
    # connection step per layer: LU of T (2/3 N^3), the solve with N right-hand sides (2 N^3) and the
    # product with B (N^3) complex multiply-adds, 8 real flops each
    conn_flops = L * (2.0 / 3.0 + 2.0 + 1.0) * N4 ** 3 * 8
    fp64_peak = 1.25  # TFLOP/s, the nominal FP64 rate of the part (no measured FP64 peak is recorded)
    res = {"workload": f"single_wavelength_sample_64x64x{L}_21x21_orders", "layers": L,
           "modes_per_layer": 4 * p.U * p.V,
           "gpu_s": wall, "gpu_step_ms": {k: t[k] for k in ("fourier_ms", "modes_ms", "connect_ms", "system_ms",
                                                             "alpha_ms", "erows_ms", "total_ms")},
           "eig_ms_per_layer_effective": t["modes_ms"] / L,
           "roofline": {"kernel": "connection step (getrf, getrs, zgemm)", "bound": "fp64",
                        "achieved": conn_flops / (t["connect_ms"] * 1e-3) / 1e12, "peak": fp64_peak,
                        "unit": "TFLOP/s", "frac": conn_flops / (t["connect_ms"] * 1e-3) / 1e12 / fp64_peak,
                        "traffic": None, "peak_source": "nominal FP64 rate"},
           "arith": "FP64 (complex128); eigendecompositions of the 2M x 2M reduced problem, 8 worker threads"}
    if with_oracle:
        from oracle import cw
        u, v = cw.orders(p.U, p.V)
        sx, sy = cw.directions(p.U, p.V, p.lam, p.X, p.Y)
        t0 = time.perf_counter()
        _, _, D = cw.layer_operators(p.n_volume[0], sx, sy, u, v)
        gam, Q = cw.layer_modes(D)
        t_eig = time.perf_counter() - t0
        t0 = time.perf_counter()
        T, B = cw.top_bottom(gam, Q, p.z_bounds[1] - p.z_bounds[0], 2 * np.pi / p.lam)
        K = B @ np.linalg.solve(T, np.eye(T.shape[0], dtype=np.complex128))
        t_conn = time.perf_counter() - t0
        del K
        res["cpu_baseline"] = {"value": L * (t_eig + t_conn), "unit": f"s ({L} layers, scaled from one)",
                               "cores": blas_threads(), "kind": "oracle",
                               "sample": f"layer 0: assembly + full 4M x 4M eig {t_eig:.2f} s, connection "
                                         f"step {t_conn:.2f} s; times {L} layers"}
        res["speedup_vs_oracle"] = res["cpu_baseline"]["value"] / wall
    del W, g, a, pr, pt
    return res


def timed_steps(fn, steps, warmup, stream, barrier):
    """ms per call of fn() over `steps` calls after `warmup` untimed ones (CUDA events on
    `stream`, barrier + synchronize on both sides)."""
    import torch
    for _ in range(warmup):
        fn()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1) / steps


def kernel_times(plan, fn, calls=3):
    """Per-kernel CUDA-event times of `calls` direct (non-graph) calls."""
    plan.enable_timing(True)
    for _ in range(calls):
        fn()
    kt = plan.timings()
    plan.enable_timing(False)
    return {k: kt[k] for k in ("phases_ms", "contract_ms", "xpass_ms", "ypass_ms", "recompose_ms", "total_ms")}


def step_timeline(plan, fn, reps=5):
    """Begin / end of each kernel of one graph-replayed step (us from the step's first kernel),
    from the plan's %globaltimer trace; the median over `reps` isolated steps."""
    plan.enable_trace(True)
    traces = []
    for _ in range(reps):
        fn()
        traces.append(plan.trace())
    plan.enable_trace(False)
    fn()  # recapture the untraced graph
    return {k: [statistics.median(t[k][0] for t in traces), statistics.median(t[k][1] for t in traces)]
            for k in traces[0]}


def oracle_volume(W, g, a, zb, zp, U=None, X=None, Fxy=None):
    """The FP64 oracle's field of every voxel (spectrum per plane, then the direct sum
    of Eq. 10) and the seconds it took on the host cores."""
    from oracle import cw, synth
    U = U or U_ORD
    X = X or X_PERIOD
    Fxy = Fxy or F_XY
    ls = cw.LayerSet(lam=LAM, X=X, Y=X, U=U, V=U, z_bounds=zb, W=W, gamma=g, alpha=a,
                     p_inc=None, p_ref=None, p_trn=None)
    t0 = time.perf_counter()
    E = synth.synthesize_direct(ls, Fxy, Fxy, zp)
    return E, time.perf_counter() - t0


def error_vs_oracle(E, ref):
    """Per-component rel-L2 and max-abs (absolute, and over the component's largest magnitude)."""
    out = {"rel_l2": [], "max_abs": [], "max_abs_over_max": []}
    for c in range(3):
        d = E[c].astype(np.complex128) - ref[c]
        out["rel_l2"].append(float(np.linalg.norm(d) / np.linalg.norm(ref[c])))
        m = float(np.abs(d).max())
        out["max_abs"].append(m)
        out["max_abs_over_max"].append(m / float(np.abs(ref[c]).max()))
    out["components"] = ["Ex", "Ey", "Ez"]
    return out


def run_config3(args, dev, world, barrier, with_oracle):
    """The precision form of the tiny sample and the compute-bound variant of the
    single-wavelength sample.
      tiny: 16x16x4 voxels, one sphere, 7x7 orders, 64x64x32 output, solved by the
            oracle; FP32, split-BF16 and FP16 fields against the oracle's direct sum
            (per-component rel-L2 and max-abs).
      layers_4_planes_64: the single-wavelength geometry with 4 layers of 0.25 um
            (64 x 64 x 4 voxels, solved on the GPU) and 64 planes per layer, 256^3
            output: the contraction has 64 columns per layer against each read of W.
            FP32 and split-BF16 timed on the same inputs (contraction and whole step)."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    stream = torch.cuda.current_stream(dev)
    res = {}
    if with_oracle:
        from oracle import cw, synth
        p = wl.config_tiny()
        sol = cw.solve_problem(p)
        ref = synth.synthesize_direct(sol, p.Fx, p.Fy, p.z_planes)
        Wt = torch.from_numpy(sol.W.astype(np.complex64)).to(dev)
        gt, at = torch.from_numpy(sol.gamma).to(dev), torch.from_numpy(sol.alpha).to(dev)
        tiny = {"workload": "tiny_16x16x4_sphere_7x7_orders_64x64x32"}
        for prec in ("fp32", "split_bf16", "fp16"):
            plan = scw.Plan(p.U, p.V, p.L, p.lam, p.X, p.Y, p.z_bounds, p.Fx, p.Fy, p.z_planes, precision=prec)
            plan.set_layers(Wt, gt, at)
            E = plan.synthesize().cpu().numpy()
            plan.check()
            plan.close()
            tiny[prec] = error_vs_oracle(E, ref)
        res["tiny"] = tiny
    # compute-bound variant: 4 solved layers, 64 planes each
    L4 = 4
    p4, s4, _, _, (W4, g4, a4), solve_s = solve_sample(dev, replica_seed(int(os.environ.get("RANK", "0"))), L4)
    s4.close()
    zb4 = p4.z_bounds
    zp4 = wl.cell_centred_planes(zb4[0], zb4[-1], 256)
    voxels = F_XY * F_XY * len(zp4)
    out = torch.empty((3, len(zp4), F_XY, F_XY), dtype=torch.complex64, device=dev)
    v = {"workload": "single_wavelength_4_layers_64_planes_per_layer_256x256x256", "solve_s": solve_s}
    steps = max(3, min(args.steps, 20))
    for prec in ("split_bf16", "fp32"):
        plan = scw.Plan(U_ORD, U_ORD, L4, LAM, X_PERIOD, X_PERIOD, zb4, F_XY, F_XY, zp4, precision=prec)
        plan.set_layers(W4, g4, a4)
        ms = timed_steps(lambda: plan.synthesize(out), steps, max(3, args.warmup), stream, barrier)
        kt = kernel_times(plan, lambda: plan.synthesize(out))
        plan.check()
        plan.close()
        v[prec] = {"value": replica_throughput(voxels, ms * 1e-3, dev)[0], "ms_per_step": ms, "kernel_ms": kt}
    v["contract_speedup_split_bf16_vs_fp32"] = v["fp32"]["kernel_ms"]["contract_ms"] / \
        v["split_bf16"]["kernel_ms"]["contract_ms"]
    v["step_speedup_split_bf16_vs_fp32"] = v["fp32"]["ms_per_step"] / v["split_bf16"]["ms_per_step"]
    rest = v["split_bf16"]["ms_per_step"] - v["split_bf16"]["kernel_ms"]["contract_ms"]
    v["common_ms"] = rest
    v["step_speedup_bound"] = (v["fp32"]["kernel_ms"]["contract_ms"] + rest) / \
        (v["split_bf16"]["kernel_ms"]["contract_ms"] + rest)
    res["layers_4_planes_64"] = v
    del out, W4, g4, a4
    return res


def run_surrogate(args, dev, bf16_peaks):
    """Learned surrogate at its full size: 4 Fourier layers of width 32, 16x16
    kept modes on a 64x64 grid, inputs 8 slices of 32x32 complex n (seeded
    ellipsoid phantoms), targets complex exit-plane fields [3][64][64] (random
    values of that shape: throughput does not depend on them). Times one Adam
    training step and one inference call per batch through the C ABI."""
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl
    B = args.fno_batch
    n = torch.from_numpy(wl.phantom_batch(77, B).astype(np.complex64)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    target = torch.randn((B, 3, 64, 64), dtype=torch.complex64, device=dev, generator=g)
    s = scw.Surrogate(grid=64, modes=16, layers=4, slices=8, in_grid=32, batch_max=B, precision="bf16", seed=1)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        s.train_step(n, target, lr=1e-4, read_loss=False)
    steps = max(3, min(args.steps, 20))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        s.train_step(n, target, lr=1e-4, read_loss=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    train_ms = e0.elapsed_time(e1) / steps
    loss = s.train_step(n, target, lr=1e-4)
    field = torch.empty((B, 3, 64, 64), dtype=torch.complex64, device=dev)
    for _ in range(3):
        s.infer(n, field=field)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        s.infer(n, field=field)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    infer_ms = e0.elapsed_time(e1) / steps
    launches = s.launches()
    # per-family breakdown of the training step (events between launches)
    s.enable_timing(True)
    for _ in range(3):
        s.train_step(n, target, lr=1e-4, read_loss=False)
    t = s.timings()
    s.enable_timing(False)
    calls = max(1, t["calls"])
    fam = {k: t[k + "_ms"] / calls for k in ("dft", "layer", "dw", "mix", "other")}
    tf = {k: (t[k + "_flops"] / calls) / (fam[k] * 1e-3) / 1e12 for k in ("dft", "layer", "dw") if fam[k] > 0}
    dom = max(("dft", "layer"), key=lambda k: fam[k])
    peak = bf16_peaks[1]
    # the layer products' DRAM bytes per training step: activation layouts of B C P BF16 values,
    # forward layers 0..L-2 read V_l and write V_{l+1} and GELU'(Z_l), the last writes V_L;
    # backward layers L-1..1 read dZ_l and GELU'(Z_{l-1}) and write dZ_{l-1}, layer 0 writes dV_0
    L_fno, C_fno, P_fno = 4, 32, 64 * 64
    layer_bytes = 2 * (3 * (L_fno - 1) + 2) * B * C_fno * P_fno * 2
    hbm = bf16_peaks[2]
    layer_gbs = layer_bytes / (fam["layer"] * 1e-3) / 1e9
    s.close()
    return {
        "workload": "fno_4_layers_width_32_modes_16x16_grid_64x64_from_8x32x32", "batch": B,
        "train_samples_per_s": B / (train_ms * 1e-3), "train_ms_per_step": train_ms,
        "infer_samples_per_s": B / (infer_ms * 1e-3), "infer_ms_per_batch": infer_ms,
        "loss_after": [float(x) for x in loss],
        "kernel_ms_per_train_step": fam, "tflops": tf,
        "roofline": {"kernel": {"dft": "gemm_layer_persistent<EPI_MODES> (truncated DFT)",
                                "layer": "gemm_layer_persistent (inverse DFT + 1x1 conv + GELU)"}[dom],
                     "bound": "tensor", "achieved": tf[dom], "peak": peak, "unit": "TFLOP/s",
                     "frac": tf[dom] / peak, "traffic": None,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured; fallback 1700 if absent)"},
        # the layer family against both ceilings: its activation traffic takes longer at the
        # measured HBM rate than its MMAs at the sustained tensor rate, so HBM is the binding one
        "layer_rooflines": {
            "hbm": {"bytes_per_step": layer_bytes, "achieved_gbs": layer_gbs, "peak_gbs": hbm,
                    "frac": layer_gbs / hbm, "floor_ms": layer_bytes / (hbm * 1e9) * 1e3},
            "tensor": {"achieved_tflops": tf["layer"], "peak_tflops": peak, "frac": tf["layer"] / peak,
                       "floor_ms": t["layer_flops"] / calls / (peak * 1e12) * 1e3},
            "binding": "hbm" if layer_bytes / (hbm * 1e9) > t["layer_flops"] / calls / (peak * 1e12) else "tensor"},
        "gpu_launches": {"train_step": launches["train_step"], "infer": launches["infer"]},
        "dtype": "bf16 activations and weights, fp32 accumulation and master weights",
    }


def _r(x, sig=4):
    """x with `sig` significant digits (floats in nested lists / dicts; other values as they are)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}")
    if isinstance(x, (list, tuple)):
        return [_r(v, sig) for v in x]
    if isinstance(x, dict):
        return {k: _r(v, sig) for k, v in x.items()}
    return x


def _get(d, *keys):
    """d[k0][k1]..., or None where a level is missing."""
    for k in keys:
        if not isinstance(d, dict):
            return None
        d = d.get(k)
    return d


def summary(line):
    """The line's key figures in a compact block: headline and its rooflines, the kernel timeline of
    one replayed step, the FP32 arm and the split/FP32 ratios with their bound, the error of every
    voxel against the FP64 oracle, the compute-bound variants and the other workloads' headlines."""
    out = {"ms_per_step": line["ms_per_step"], "voxels_per_s": line["value"],
           "step_roofline_frac": _get(line, "step_roofline", "frac"),
           "contraction": {"frac_of_hbm": _get(line, "roofline", "frac"), "gbs": _get(line, "roofline", "achieved"),
                           "traffic_over_algorithmic": (line["roofline"]["traffic"] / line["roofline"]["algorithmic_bytes"]
                                                        if line["roofline"].get("traffic") else None)},
           "timeline_us": line.get("timeline_us"),
           "fp32": {"ms_per_step": _get(line, "fp32", "ms_per_step"), "contract_ms": _get(line, "fp32", "kernel_ms", "contract_ms"),
                    "voxels_per_s": _get(line, "fp32", "value")},
           "split_bf16_vs_fp32": {k: v for k, v in (line.get("split_bf16_vs_fp32") or {}).items() if k != "note"}}
    err = line.get("error_vs_fp64")
    if err:
        out["error_vs_fp64"] = {"voxels": err.get("voxels"), "components": "Ex Ey Ez",
                                **{f"{p}_{m}": _get(err, p, m) for p in ("split_bf16", "fp32")
                                   for m in ("rel_l2", "max_abs_over_max")}}
    c3 = line.get("config3") or {}
    out["config3"] = {k: {m: v.get(m) for m in ("contract_speedup_split_bf16_vs_fp32", "step_speedup_split_bf16_vs_fp32",
                                                 "step_speedup_bound")}
                      for k, v in c3.items() if isinstance(v, dict) and "step_speedup_split_bf16_vs_fp32" in v}
    out["e2e_voxels_per_s"] = _get(line, "e2e", "value")
    out["cpu_baseline_voxels_per_s"] = _get(line, "cpu_baseline", "value")
    out["sweep"] = {"voxels_per_s": _get(line, "sweep", "value"), "roofline_frac": _get(line, "sweep", "roofline_frac")}
    out["illumination16"] = {"ms": _get(line, "illumination", "split_bf16", "ms_per_step"),
                             "contract_tflops": _get(line, "illumination", "split_bf16", "contract_tflops")}
    out["points_window"] = {"tflops": _get(line, "points", "window_256x256_of_4um", "split_bf16", "point_product_tflops"),
                            "vs_fp32": _get(line, "points", "window_256x256_of_4um", "point_product_speedup_split_bf16_vs_fp32")}
    out["tiling"] = {"periodic_frac": _get(line, "tiling", "periodic_4x4", "roofline_frac"),
                     "mosaic_frac": _get(line, "tiling", "mosaic_4x4_patches", "roofline_frac")}
    out["solve_s"] = {"gpu": _get(line, "solve", "gpu_s"), "oracle_scaled": _get(line, "solve", "cpu_baseline", "value")}
    sg = line.get("surrogate")
    if sg:
        out["surrogate"] = {"train_ms": sg.get("train_ms_per_step"), "infer_ms": sg.get("infer_ms_per_batch"),
                            "kernel_ms": sg.get("kernel_ms_per_train_step"),
                            "layer_hbm_frac": _get(sg, "layer_rooflines", "hbm", "frac"),
                            "layer_tensor_frac": _get(sg, "layer_rooflines", "tensor", "frac"),
                            "launches": sg.get("gpu_launches")}
    return _r(out)


def run_ours(args, world, rank, local):
    import torch
    import paper_2404_07293_gb300 as scw
    import workloads as wl

    dist = world > 1
    if dist:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    zb, zp = geometry()
    Fz = len(zp)
    voxels = F_XY * F_XY * Fz
    oracle_leg = rank == 0 and not args.no_cpu_baseline

    # inputs: the sample solved on the GPU (default), or synthetic layer sets of the same shapes
    solver = None
    if args.input == "solved":
        prob, solver, n_dev, pinc_dev, (Wd, gd, ad), first_solve_s = solve_sample(dev, replica_seed(rank), L_LAYERS)
        inputs = (f"single-wavelength sample seed {replica_seed(rank)} (64x64x{L_LAYERS} voxels of ellipsoids, "
                  "Gaussian beam NA 0.5) solved on the GPU by scw_solve")
    else:
        W, g, a, *_ = wl.random_layer_set(replica_seed(rank), U_ORD, U_ORD, L_LAYERS)
        Wd, gd, ad = (torch.from_numpy(x).to(dev) for x in (W, g, a))
        inputs = "synthetic layer sets (workloads.random_layer_set) of the same shapes"
        first_solve_s = None

    def make_plan(precision, host_io=False):
        return scw.Plan(U_ORD, U_ORD, L_LAYERS, LAM, X_PERIOD, X_PERIOD, zb, F_XY, F_XY, zp,
                        precision=precision, host_io=host_io, k_split=args.k_split)

    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    plan = make_plan(args.precision)
    if args.pipeline > 1:
        plan.set_pipeline(args.pipeline)
    plan.set_layers(Wd, gd, ad)
    torch.cuda.synchronize(dev)
    plan_ms = plan.info()["convert_ms"]
    out = torch.empty(plan.out_shape(), dtype=torch.complex64, device=dev)

    for _ in range(args.warmup):
        plan.synthesize(out)
    plan.check()
    barrier()
    # timed region: the library's default path (each scw_synthesize replays one captured CUDA graph)
    plan.synthesize(out)
    plan.synthesize(out)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            plan.synthesize(out)
        ev1.record(stream)
        barrier()
    plan.check()
    ms = ev0.elapsed_time(ev1)
    E_head = out.cpu().numpy() if oracle_leg else None
    # per-kernel breakdown: the same steps as direct launches with events between the kernels
    plan.enable_timing(True)
    barrier()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    for _ in range(args.steps):
        plan.synthesize(out)
    d1.record(stream)
    barrier()
    kt = plan.timings()
    plan.enable_timing(False)
    plan.check()
    direct_ms = d0.elapsed_time(d1) / args.steps
    timeline = step_timeline(plan, lambda: plan.synthesize(out))
    value, seconds = replica_throughput(voxels * args.steps, ms * 1e-3, dev)
    ms = seconds * 1e3
    info = plan.info()

    # roofline of the dominant kernel: algorithmic bytes per launch / live launch time
    hbm, bf16_tf, peak_kind = peaks()
    M = U_ORD * U_ORD
    w_bytes = L_LAYERS * 3 * M * 4 * M * 8            # W read once (8 B per complex in every mode but FP16)
    if args.precision == "fp16":
        w_bytes //= 2
    s_bytes = Fz * 3 * M * 8                           # spectrum, once
    t_bytes = Fz * 3 * U_ORD * F_XY * 8                # x-pass rows, once
    out_bytes = 3 * voxels * 8                         # field written once
    per_kernel = {
        "contract": (w_bytes + s_bytes, kt["contract_ms"],
                     "contract_tc_kernel" if args.precision != "fp32" else "contract_fp32_kernel"),
        "ypass": (t_bytes + out_bytes, kt["ypass_ms"], "ypass_kernel"),
        "xpass": (s_bytes + t_bytes, kt["xpass_ms"], "xpass_kernel"),
    }
    kernels = {k: {"kernel": name, "algorithmic_bytes": b, "launch_ms": t, "gbs": b / (t * 1e-3) / 1e9,
                   "frac": b / (t * 1e-3) / 1e9 / hbm} for k, (b, t, name) in per_kernel.items()}
    dominant = max(kernels, key=lambda k: kernels[k]["launch_ms"])
    d = kernels[dominant]
    roof = {"kernel": d["kernel"], "bound": "hbm", "achieved": d["gbs"], "peak": hbm, "unit": "GB/s",
            "frac": d["frac"], "traffic": recorded_traffic(d["kernel"], workload_name()),
            "algorithmic_bytes": d["algorithmic_bytes"],
            "launch_ms": d["launch_ms"], "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"}
    whole_bytes = w_bytes + out_bytes
    step_roofline_ms = whole_bytes / (hbm * 1e9) * 1e3

    # the metric's other arm: the FP32 SIMT contraction on the same inputs, same timing rules
    other = "fp32" if args.precision != "fp32" else "split_bf16"
    fp = make_plan(other)
    fp.set_layers(Wd, gd, ad)
    f_ms = timed_steps(lambda: fp.synthesize(out), args.steps, args.warmup, stream, barrier)
    fp.check()
    E_other = out.cpu().numpy() if oracle_leg else None
    f_kt = kernel_times(fp, lambda: fp.synthesize(out))
    fp.check()
    fp.close()
    arm = {"value": replica_throughput(voxels, f_ms * 1e-3, dev)[0], "ms_per_step": f_ms, "kernel_ms": f_kt,
           "precision": other, "dtype": {"fp32": "fp32", "split_bf16": "bf16x3->fp32"}[other]}
    head_c, other_c = kt["contract_ms"], f_kt["contract_ms"]
    if args.precision == "fp32":
        head_c, other_c = other_c, head_c
    ratio = {"step": (f_ms / (ms / args.steps)) if other == "fp32" else ((ms / args.steps) / f_ms),
             "contraction": other_c / head_c,
             "note": "FP32 time / split-BF16 time on the same inputs; the phases and the recompose are the same "
                     "kernels on both paths, so the step ratio is bounded by (C32 + R) / (Cs + R)"}

    # the other contraction precisions on the same inputs (same step, same timing rules)
    variants = {}
    if args.compare:
        for prec in ("fp16",):
            vp = make_plan(prec)
            vp.set_layers(Wd, gd, ad)
            vms = timed_steps(lambda: vp.synthesize(out), args.steps, args.warmup, stream, barrier)
            vk = kernel_times(vp, lambda: vp.synthesize(out))
            vp.check()
            variants[prec] = {"value": world * voxels / (vms * 1e-3), "ms_per_step": vms,
                              "contract_ms": vk["contract_ms"], "k_split": vp.info()["k_split"]}
            vp.close()

    # end to end through the C ABI with HOST buffers (H2D of W/gamma/alpha, D2H of the field)
    e2e = None
    out = None  # the device output is not needed any more; free it for the next measurements
    Wh = gh = ah = None
    if not args.no_e2e or oracle_leg:
        Wh = torch.empty(tuple(Wd.shape), dtype=torch.complex64).pin_memory()
        Wh.copy_(Wd)
        gh = gd.cpu().pin_memory()
        ah = ad.cpu().pin_memory()
        Wh, gh, ah = Wh.numpy(), gh.numpy(), ah.numpy()
    if not args.no_e2e:
        hplan = make_plan(args.precision, host_io=True)
        oh = torch.empty(hplan.out_shape(), dtype=torch.complex64).pin_memory().numpy()
        for _ in range(max(1, args.warmup // 2)):
            hplan.synthesize_host(Wh, gh, ah, out=oh)
        n_e2e = max(2, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            hplan.synthesize_host(Wh, gh, ah, out=oh)
        t_e2e = time.perf_counter() - t0
        e2e_value, t_e2e = replica_throughput(voxels * n_e2e, t_e2e, dev)
        hplan.check()
        e2e = {"value": e2e_value, "unit": "voxels/s",
               "h2d_bytes_per_step": Wh.nbytes + gh.nbytes + ah.nbytes, "d2h_bytes_per_step": oh.nbytes,
               "steps": n_e2e, "ms_per_step": 1e3 * t_e2e / n_e2e,
               "includes": "H2D of W, gamma, alpha; W conversion; synthesis; D2H of the field"}
        hplan.close()
        del oh

    illum = None
    if args.illuminations > 1:
        illum = run_illumination(args, dev, world, Wd, gd, zb, zp, hbm, bf16_tf)
        torch.cuda.empty_cache()

    config3 = None
    if not args.no_config3:
        config3 = run_config3(args, dev, world, barrier, oracle_leg)
        if illum is not None:
            config3["illuminations_16_256x256"] = {
                k: illum[k] for k in ("contract_speedup_split_bf16_vs_fp32", "step_speedup_split_bf16_vs_fp32",
                                      "common_ms", "step_speedup_bound")}
            small = run_illumination(args, dev, world, Wd, gd, zb, zp, hbm, bf16_tf, fxy=128,
                                     precisions=("split_bf16", "fp32"))
            config3["illuminations_16_128x128"] = {
                "workload": small["workload"],
                "fp32_ms_per_step": small["fp32"]["ms_per_step"],
                "split_bf16_ms_per_step": small["split_bf16"]["ms_per_step"],
                **{k: small[k] for k in ("contract_speedup_split_bf16_vs_fp32", "step_speedup_split_bf16_vs_fp32",
                                         "common_ms", "step_speedup_bound")}}
        torch.cuda.empty_cache()

    points = None
    if not args.no_points:
        points = run_points(args, dev, world, Wd, gd, ad, zb, zp, hbm, bf16_tf)
        torch.cuda.empty_cache()

    tiling = None
    if not args.no_tiling:
        tiling = run_tiling(args, dev, world, Wd, gd, ad, zb, zp, hbm)
        torch.cuda.empty_cache()

    plan.close()
    del Wd, gd, ad
    torch.cuda.empty_cache()

    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(args, dev, world, hbm)

    solve = None
    if solver is not None and not args.no_solve:
        torch.cuda.empty_cache()
        solve = run_solve(args, dev, oracle_leg, prob, solver, n_dev, pinc_dev)
        solve["first_call_s"] = first_solve_s
    if solver is not None:
        solver.close()

    surrogate = None
    if not args.no_surrogate:
        torch.cuda.empty_cache()
        surrogate = run_surrogate(args, dev, (bf16_tf, bf16_sustained(), peaks()[0]))

    # the oracle leg: the FP64 oracle synthesises every voxel of the same inputs on the host
    # cores (timed: cpu_baseline); both GPU arms are compared with it voxel by voxel
    cpu = None
    error = None
    if oracle_leg:
        ref, dt = oracle_volume(Wh.astype(np.complex128), gh, ah, zb, zp)
        cpu = {"value": voxels / dt, "unit": "voxels/s", "cores": blas_threads(), "kind": "oracle",
               "sample": f"the whole {F_XY}x{F_XY}x{Fz} volume of the timed inputs (FP64 spectrum per plane + "
                         f"direct sum of Eq. 10), {dt:.1f} s"}
        error = {args.precision: error_vs_oracle(E_head, ref), other: error_vs_oracle(E_other, ref),
                 "voxels": voxels, "oracle": "FP64 direct sum, every voxel"}
        del ref

    if rank == 0:
        line = {
            "metric": "field voxels/s", "value": value, "unit": "voxels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "fp32", "split_bf16": "bf16x3->fp32", "fp16": "fp16x2->fp32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": workload_name(), "orders": "21x21", "M": M, "layers": L_LAYERS,
                       "grid": [F_XY, F_XY, Fz], "precision": args.precision, "k_split": info["k_split"],
                       "inputs": inputs,
                       "l2": (f"inputs larger than L2 (W {L_LAYERS * 3 * M * 4 * M * 8 / 1e6:.0f} MB, field "
                              f"{3 * voxels * 8 / 1e6:.0f} MB)"),
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "step_roofline": {"bytes": whole_bytes, "ms": step_roofline_ms,
                              "frac": step_roofline_ms / (ms / args.steps)},
            other: arm,
            "split_bf16_vs_fp32": ratio,
            "error_vs_fp64": error,
            "kernel_ms": {k: kt[k] for k in ("phases_ms", "contract_ms", "xpass_ms", "ypass_ms", "recompose_ms",
                                             "total_ms")},
            "kernel_roofline": kernels,
            "schedule": {k: info[k] for k in ("contract_ctas", "contract_tasks", "schedule_max_load",
                                              "schedule_mean_load")},
            "timing": "CUDA-graph replay of scw_synthesize (the library's default path); kernel_ms from a "
                      "second pass of direct launches with events between kernels",
            "direct_launch": {"ms_per_step": direct_ms, "value": world * voxels / (direct_ms * 1e-3)},
            "timeline_us": timeline,
            "plan_convert_ms": plan_ms,
            "gpu_launches": info["kernels_per_synthesis"] * args.steps,
            "clocks": clocks.summary(),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "config3": config3,
            "variants": variants or None,
            "sweep": sweep,
            "illumination": illum,
            "points": points,
            "tiling": tiling,
            "solve": solve,
            "surrogate": surrogate,
        }
        line["summary"] = summary(line)  # last: the part of a long line that a tail of the output keeps
        print(json.dumps(line), flush=True)
    if dist:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["split_bf16", "fp32", "fp16"], default="split_bf16")
    ap.add_argument("--k-split", dest="k_split", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--compare", action="store_true", help="also time the other contraction precisions")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched spectroscopic sweep")
    ap.add_argument("--sweep-items", type=int, default=128)
    ap.add_argument("--no-surrogate", action="store_true", help="skip the learned-surrogate block")
    ap.add_argument("--fno-batch", type=int, default=256)
    ap.add_argument("--no-points", action="store_true", help="skip the off-grid point-set block")
    ap.add_argument("--no-tiling", action="store_true", help="skip the periodic-tiling / patch-mosaic block")
    ap.add_argument("--no-solve", action="store_true", help="skip the GPU solve-stage block")
    ap.add_argument("--no-config3", action="store_true", help="skip the precision / compute-bound block")
    ap.add_argument("--input", choices=["solved", "random"], default="solved",
                    help="headline inputs: the GPU-solved sample or synthetic layer sets of the same shapes")
    ap.add_argument("--illuminations", type=int, default=16,
                    help="incident fields of the multi-illumination block (1 skips it)")
    ap.add_argument("--only-surrogate", action="store_true",
                    help="run only the learned-surrogate block and print its JSON (a profiling aid, not the bench line)")
    ap.add_argument("--layers", type=int, default=32)
    ap.add_argument("--pipeline", type=int, default=1, help="layer groups overlapped in graph replay")
    ap.add_argument("--planes-per-layer", type=int, default=8)
    args = ap.parse_args()
    global L_LAYERS, PLANES_PER_LAYER
    L_LAYERS, PLANES_PER_LAYER = args.layers, args.planes_per_layer
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.only_surrogate:
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        print(json.dumps({"surrogate": run_surrogate(args, dev, (peaks()[1], bf16_sustained(), peaks()[0]))}), flush=True)
        return 0
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
