#!/usr/bin/env python
"""Benchmark of the GB300 path: exact H0 + top-dimension persistence pairs of a
512^3 float32 blurred-noise volume (white noise, Gaussian sigma = 3 voxels,
normalised to [0, 1]), one step = the whole hot path: lookup + pruning, sorts,
both union-finds, emission, then the total-persistence loss and its backward
scatter to the voxels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (one
volume per rank; a single volume's union-find is global and does not shard).
The volume (512 MiB) is larger than L2, so no L2 flush is done between steps.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

SIDE = 512
SIGMA = 3.0
METRIC = "Mvoxels/s for exact H0+top-dim diagrams (512^3 fp32), % HBM roofline; fwd+bwd batched vs plain"
WORKLOAD = "3D 512^3 float32 blurred noise (sigma 3 vox), H0 + H2 pairs, fwd + total-persistence loss bwd"
TAU = 0.05  # persistence threshold of the loss
COUNTERS_BYTES = 4056  # status/count block the forward call copies back (sizeof the library's counters)


def _volume(seed: int) -> np.ndarray:
    cache = f"/tmp/cp_bench_vol_{SIDE}_{SIGMA}_{seed}.npy"
    if os.path.exists(cache):
        try:
            return np.load(cache)
        except Exception:
            pass
    v = workloads.blurred((SIDE, SIDE, SIDE), SIGMA, seed)
    try:
        np.save(cache + ".tmp.npy", v)
        os.replace(cache + ".tmp.npy", cache)
    except OSError:
        pass
    return v


def job_time(local_s: float, world: int, device) -> float:
    """Wall time of the job: the maximum over ranks (the job ends with its slowest rank)."""
    if world <= 1:
        return local_s
    import torch

    t = torch.tensor([local_s], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step: float, world: int, steps: int, seconds: float) -> float:
    """Whole-job throughput in millions of units per second: every rank is a
    replica that processes its own units each step (weak scaling)."""
    return units_per_rank_step * world * steps / seconds / 1e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "50", "-i", str(self.idx)],
                stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL,
                text=True,
            )
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.p is not None:
            time.sleep(0.2)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """The oracle (plain single-threaded C) on bounded crops of the same workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    oracle.build()
    n_runs = args.steps + args.warmup
    # the oracle runs at ~0.3-0.5 Mvox/s; aim at ~2 minutes in total
    side = int(round((0.35e6 * 120.0 / max(1, n_runs)) ** (1.0 / 3.0)))
    side = max(24, min(192, side))
    vol = _volume(0)
    crop = np.ascontiguousarray(vol[:side, :side, :side])
    for _ in range(args.warmup):
        oracle.persistence(crop)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.persistence(crop)
    dt = time.perf_counter() - t0
    value = crop.size * args.steps / dt / 1e6
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "Mvoxels/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{side}^3 crop of the 512^3 volume per step", "parallelism": "replicas"},
        "cpu_baseline": {
            "value": value,
            "unit": "Mvoxels/s",
            "cores": 1,
            "host": _host(),
            "kind": "oracle",
            "sample": f"{side}^3 crop of the 512^3 blurred volume (same recipe), H0 + H2 pairs",
        },
        "e2e": {"value": value, "unit": "Mvoxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _host():
    """The host the CPU baseline ran on: logical CPUs and the CPU model (lscpu,
    else /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    k, _, v = line.partition(":")
                    if k.strip() in ("model name", "Model", "CPU part") and v.strip():
                        model = v.strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu": model or platform.machine(), "machine": platform.machine()}


def cpu_baseline(vol, budget_s=20.0):
    """The oracle as it stands, timed on this host (1 thread) on a crop of the volume."""
    import oracle

    oracle.build()
    side = 96
    crop = np.ascontiguousarray(vol[:side, :side, :side])
    t0 = time.perf_counter()
    oracle.persistence(crop)
    dt = time.perf_counter() - t0
    # grow the crop towards the time budget
    side2 = int(side * min(2.0, max(1.0, (budget_s / max(dt, 1e-3)) ** (1 / 3) * 0.8)))
    side2 = min(side2, 192)
    if side2 > side:
        crop = np.ascontiguousarray(vol[:side2, :side2, :side2])
        t0 = time.perf_counter()
        oracle.persistence(crop)
        dt = time.perf_counter() - t0
        side = side2
    return {
        "value": crop.size / dt / 1e6,
        "unit": "Mvoxels/s",
        "cores": 1,
        "host": _host(),
        "kind": "oracle",
        "sample": f"{side}^3 crop of the 512^3 volume, H0 + H2 pairs, single-threaded C oracle, {dt:.1f} s",
    }


def _oracle_item(a):
    import oracle

    oracle.persistence(a)
    return a.size


def batched_cpu_baseline(items, budget_s=10.0):
    """The oracle as it stands on the batched workload's items, spread over all
    host cores (a spawn pool): a bounded sample of the items (those up to 3 M
    voxels, in workload order, up to about budget_s seconds of wall time)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    cap = cores * budget_s * 0.3e6  # voxels the pool clears in the budget at ~0.3 Mvox/s per core
    sample, total = [], 0
    for a in items:
        if a.size <= 3_000_000 and total + a.size <= cap:
            sample.append(a)
            total += a.size
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_item, sample[:cores])  # warm the workers (import, load the library)
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_item, sample, chunksize=1))
        dt = time.perf_counter() - t0
    return {
        "value": done / dt / 1e6,
        "unit": "Mvoxels/s",
        "cores": cores,
        "host": _host(),
        "kind": "oracle",
        "sample": f"{len(sample)} of {len(items)} items ({done / 1e6:.1f} M voxels, items up to 3 M voxels), "
        f"one item per task in a pool of {cores} processes, {dt:.1f} s",
    }


def _batch_items():
    cache = "/tmp/cp_bench_batch_v1.npz"
    if os.path.exists(cache):
        try:
            z = np.load(cache)
            return [z[f"a{i}"] for i in range(len(z.files))]
        except Exception:
            pass
    items = workloads.batch(0)
    try:
        np.savez(cache + ".tmp.npz", **{f"a{i}": a for i, a in enumerate(items)})
        os.replace(cache + ".tmp.npz", cache)
    except OSError:
        pass
    return items


def batched_vs_plain(dev, steps: int, warmup: int):
    """Fwd + loss bwd of the batched workload: one CUDA-graph launch for the
    whole batch against one call per item (same kernels, no graph)."""
    import torch

    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    items = _batch_items()
    shapes = [a.shape for a in items]
    nvox = int(sum(a.size for a in items))
    from paper_2606_04801_gb300 import autotune

    tuned = autotune.autotune([torch.from_numpy(a).to(dev) for a in items])
    bp = cp.BatchedPersistence(shapes, tau=TAU, device=dev, graph=True)
    bp.load([torch.from_numpy(a) for a in items])
    for _ in range(warmup):
        bp.step()
    st = bp.status()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        bp.step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_batched = e0.elapsed_time(e1) / 1e3 / steps
    # plain: one forward and one loss backward per item, sequential on one stream
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    per = []
    for a in items:
        nd = a.ndim
        dims = (ctypes.c_int64 * nd)(*a.shape)
        wsb = lib.cubical_persistence_workspace_size(nd, dims, 0)
        cap = a.size // 2 + 65536 + 4096
        per.append((nd, dims, wsb, cap))
    ws = torch.empty(max(p[2] for p in per), dtype=torch.uint8, device=dev)
    outs = [torch.empty((p[3], 8), dtype=torch.int32, device=dev) for p in per]
    cnts = torch.zeros(len(items), dtype=torch.int64, device=dev)
    loss = torch.zeros(len(items), dtype=torch.float64, device=dev)
    grad = torch.empty(nvox, dtype=torch.float32, device=dev)
    bws = torch.empty(lib.cubical_persistence_loss_backward_workspace_size(max(a.size for a in items)),
                      dtype=torch.uint8, device=dev)
    offs = np.concatenate([[0], np.cumsum([a.size for a in items])[:-1]])

    def plain_step():
        for i, ((nd, dims, wsb, cap), a) in enumerate(zip(per, items)):
            fn = lib.cubical_persistence_2d if nd == 2 else lib.cubical_persistence_3d
            rc = fn(ctypes.c_void_p(bp.views[i].data_ptr()), dims, ctypes.c_void_p(outs[i].data_ptr()), cap, None,
                    ctypes.c_void_p(cnts[i:].data_ptr()), ctypes.c_void_p(ws.data_ptr()), wsb, 0, sp)
            if rc != 0:
                raise RuntimeError(f"plain forward {i}: {rc}")
            rc = lib.cubical_persistence_loss_backward(
                ctypes.c_void_p(outs[i].data_ptr()), cap, ctypes.c_void_p(cnts[i:].data_ptr()), ctypes.c_float(TAU),
                ctypes.c_void_p(loss[i:].data_ptr()), None, ctypes.c_void_p(grad[int(offs[i]):].data_ptr()), a.size,
                ctypes.c_void_p(bws.data_ptr()), bws.numel(), sp)
            if rc != 0:
                raise RuntimeError(f"plain backward {i}: {rc}")

    for _ in range(max(1, warmup)):
        plain_step()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        plain_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_plain = e0.elapsed_time(e1) / 1e3 / steps
    same = bool(abs(float(loss.sum().item()) - float(bp.loss.item())) <= 1e-9 * max(1.0, float(bp.loss.item())))
    return {
        "workload": "64 2D (sides 128-1024) + 8 3D (sides 64-192) blurred, rank-spaced; fwd + loss bwd",
        "voxels": nvox,
        "batched_graph_ms": t_batched * 1e3,
        "batched_mvox_per_s": nvox / t_batched / 1e6,
        "batched_items_per_s": len(items) / t_batched,
        "plain_ms": t_plain * 1e3,
        "plain_mvox_per_s": nvox / t_plain / 1e6,
        "speedup": t_plain / t_batched,
        "same_loss": same,
        "status": st["rc"],
        "tuning": {k: tuned[k] for k in ("zchunk3d", "ctas3d", "rows2d", "uf_variant")},
    }


def run_survivors():
    """Survivor fractions (H0 and top-dimension survivors of the pruning pass
    per vertex) and pair counts of every config, through the public API."""
    import torch

    import paper_2606_04801_gb300 as cp

    out = {}
    for name in ("2d_64_uniform", "2d_2048_grf", "3d_128", "3d_512_blurred", "batch"):
        arrs = workloads.config(name)
        if name == "batch":
            d = cp.persistence_batched([torch.from_numpy(a).cuda() for a in arrs], with_stats=True)
            n = sum(a.size for a in arrs)
            rows = [("all", n, d.stats, len(d))]
        else:
            rows = []
            for i, a in enumerate(arrs):
                d = cp.persistence(torch.from_numpy(a).cuda(), with_stats=True)
                rows.append((str(i), a.size, d.stats, len(d)))
        for tag, n, st, npairs in rows:
            out[f"{name}/{tag}"] = {"N": n, "h0_survivors_per_N": st["h0_survivors"] / n,
                                    "top_survivors_per_N": st["top_survivors"] / n,
                                    "h0_roots_per_N": st["h0_roots"] / n, "top_roots_per_N": st["top_roots"] / n,
                                    "pairs": npairs, "h0_rounds": st["h0_rounds"], "top_rounds": st["top_rounds"]}
    print(json.dumps({"metric": "survivor fractions S/N per config", "configs": out}), flush=True)


def run_batched(args):
    """The batched workload alone: fwd + loss bwd of 64 images and 8 volumes of
    uneven sizes, one CUDA-graph launch per step (or eager with --eager)."""
    import torch

    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import autotune

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    items = _batch_items()
    nvox = int(sum(a.size for a in items))
    autotune.autotune([torch.from_numpy(a).to(dev) for a in items])
    bp = cp.BatchedPersistence([a.shape for a in items], tau=TAU, device=dev, graph=not args.eager)
    bp.load([torch.from_numpy(a) for a in items])
    for _ in range(args.warmup):
        bp.step()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            bp.step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    t = job_time(e0.elapsed_time(e1) / 1e3 / args.steps, ws, dev)
    st = bp.status()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = batched_cpu_baseline(items)
    if rank == 0:
        print(json.dumps({
            "metric": "Mvoxels/s fwd+bwd, batched workload (64 images + 8 volumes, uneven sizes)",
            "value": job_value(nvox, ws, 1, t),
            "unit": "Mvoxels/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "64 2D (sides 128-1024) + 8 3D (sides 64-192) blurred, rank-spaced; fwd + loss bwd",
                       "voxels": nvox, "graph": not args.eager, "status": st["rc"],
                       "l2": "inputs (166 MiB) larger than L2; no flush", "parallelism": "replicas" if ws > 1 else "single",
                       "survivor_fraction": (st["h0_survivors"] + st["top_survivors"]) / nvox},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_2d(args):
    """2D configuration: the 2048x2048 Gaussian random field (sigma 8 px) and
    the same field at 256 levels (heavy ties), fwd + total-persistence loss
    bwd on each, device-resident input; the pruning pass's roofline (2D K1)
    and the oracle on one host core on a crop."""
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        torch.distributed.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib, autotune

    lib = _lib.load()
    imgs = workloads.config("2d_2048_grf")
    names = ["grf", "grf_256_levels"]
    H, W = imgs[0].shape
    N = H * W
    T = (H - 1) * (W - 1)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    dims = (ctypes.c_int64 * 2)(H, W)
    ws_bytes = lib.cubical_persistence_workspace_size(2, dims, 0)
    wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cap = N // 2 + 65536 + 4096
    out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
    grad = torch.empty(N, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    bws = lib.cubical_persistence_loss_backward_workspace_size(N)
    bwsp = torch.empty(bws, dtype=torch.uint8, device=dev)
    dcount = torch.zeros(1, dtype=torch.int64, device=dev)
    peak, peak_kind = _peaks()
    lines = {}
    for name, img in zip(names, imgs):
        x = torch.from_numpy(img).to(dev)
        autotune.autotune([x])

        def step():
            rc = lib.cubical_persistence_2d(
                ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
                ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(wsp.data_ptr()), ws_bytes, 0, sp,
            )
            if rc != 0:
                raise cp.CpError(rc, "2D forward")
            rc = lib.cubical_persistence_loss_backward(
                ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(dcount.data_ptr()), ctypes.c_float(TAU),
                ctypes.c_void_p(loss.data_ptr()), None, ctypes.c_void_p(grad.data_ptr()), N,
                ctypes.c_void_p(bwsp.data_ptr()), bws, sp,
            )
            if rc != 0:
                raise cp.CpError(rc, "loss backward")

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        lib.cp_profile(1)
        stage = (ctypes.c_float * 6)()
        k1 = []
        # the image (16 MiB) fits in L2: each timed step starts from a flushed L2
        # (a 256 MiB write between steps, outside the timed events)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            step()
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            total += ev0.elapsed_time(ev1) / 1e3
            if lib.cp_stage_times(stage, 6) == 6:
                k1.append(stage[0])
        lib.cp_profile(0)
        st = cp.api._stats(wsp)
        if st["rc"] != 0:
            raise cp.CpError(st["rc"], "2D timed steps")
        eager_elapsed = job_time(total, ws, dev)
        # the same step captured once into a CUDA graph (the library's batched
        # form with one item): a single image's step is a chain of ~40 short
        # launches, and the graph removes the gaps between them
        bp = cp.BatchedPersistence([img.shape], tau=TAU, device=dev, graph=True)
        bp.load([torch.from_numpy(img)])
        for _ in range(args.warmup):
            bp.step()
        torch.cuda.synchronize(dev)
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(stream)
            bp.step()
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            total += ev0.elapsed_time(ev1) / 1e3
        if bp.status()["rc"] != 0:
            raise cp.CpError(bp.status()["rc"], "2D graph steps")
        elapsed = job_time(total, ws, dev)
        k1s = statistics.mean(k1) / 1e3 if k1 else None
        alg = 4 * N + 4 * N + 4 * (T + 1) + 8 * (st["h0_survivors"] + st["top_survivors"]) + 16 * (st["h0_roots"] + st["top_roots"])
        lines[name] = {
            "value": job_value(N, ws, args.steps, elapsed), "ms_per_step": elapsed / args.steps * 1e3,
            "eager_ms_per_step": eager_elapsed / args.steps * 1e3,
            "k1_ms": k1s * 1e3 if k1s else None,
            "roofline": {"bound": "hbm", "achieved": alg / k1s / 1e9 if k1s else None, "peak": peak, "unit": "GB/s",
                         "frac": alg / k1s / 1e9 / peak if (k1s and peak) else None, "kernel": "k_prune2d",
                         "peak_source": peak_kind, "algorithmic_bytes": alg},
            "counts": {k: st[k] for k in ("pairs", "h0_survivors", "top_survivors", "h0_roots", "top_roots",
                                          "h0_rounds", "top_rounds")},
        }
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        for img in imgs:
            oracle.persistence(img)
        dt = time.perf_counter() - t0
        cpu = {"value": 2 * N / dt / 1e6, "unit": "Mpixels/s", "cores": 1, "host": _host(), "kind": "oracle",
               "sample": f"both 2048x2048 images whole, H0 + H1 pairs, single-threaded C oracle, {dt:.1f} s"}
    if rank == 0:
        main = lines["grf"]
        print(json.dumps({
            "metric": "Mpixels/s, H0 + H1 pairs (2048x2048 fp32 Gaussian random field, sigma 8), fwd + loss bwd",
            "value": main["value"], "unit": "Mpixels/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2D 2048x2048 float32 Gaussian random field (sigma 8 px, min-max normalised), "
                                   "and the same field at 256 levels; fwd + total-persistence loss bwd",
                       "graph": "the step as one CUDA graph (BatchedPersistence with one item); eager_ms_per_step "
                                "per image beside it",
                       "l2": "input (16 MiB) smaller than L2: L2 flushed (256 MiB write) before every timed step, "
                             "each step timed alone",
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": main["roofline"],
            "per_image": lines,
            "cpu_baseline": cpu,
        }), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_tfilt(args):
    """T-filtration workload: a 510^3 blurred volume (the padded dual image the
    V pipeline runs on is exactly 512^3), forward + total-persistence loss
    backward, device-resident input; the T oracle on a crop as the CPU line."""
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        torch.distributed.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    side = min(SIDE, 510)
    cache = f"/tmp/cp_bench_tvol_{side}_{SIGMA}_{rank}.npy"
    vol = np.load(cache) if os.path.exists(cache) else workloads.blurred((side,) * 3, SIGMA, rank)
    if not os.path.exists(cache):
        np.save(cache, vol)
    N = vol.size
    x = torch.from_numpy(vol).to(dev)
    from paper_2606_04801_gb300 import autotune

    autotune.autotune([x])  # the dual image falls in the same shape class
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    dims = (ctypes.c_int64 * 3)(side, side, side)
    ws_bytes = lib.cubical_persistence_t_workspace_size(3, dims, 0)
    wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cap = (side + 2) ** 3 // 2 + 65536 + 4096
    out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
    grad = torch.empty(N, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    bws = lib.cubical_persistence_loss_backward_workspace_size(N)
    bwsp = torch.empty(bws, dtype=torch.uint8, device=dev)
    dcount = torch.zeros(1, dtype=torch.int64, device=dev)

    def step():
        rc = lib.cubical_persistence_t_3d(
            ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
            ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(wsp.data_ptr()), ws_bytes, 0, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "T forward")
        rc = lib.cubical_persistence_loss_backward(
            ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(dcount.data_ptr()), ctypes.c_float(TAU),
            ctypes.c_void_p(loss.data_ptr()), None, ctypes.c_void_p(grad.data_ptr()), N, ctypes.c_void_p(bwsp.data_ptr()),
            bws, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "loss backward")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = cp.api._stats(wsp)
    if st["rc"] != 0:
        raise cp.CpError(st["rc"], "T warm-up")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    launches0 = lib.cp_launch_count()
    lib.cp_profile(1)
    stage = (ctypes.c_float * 6)()
    stage_sum = [0.0] * 6
    with Clocks(gpu_index) as clk:
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            if lib.cp_stage_times(stage, 6) == 6:
                for i in range(6):
                    stage_sum[i] += stage[i]
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
    launches = lib.cp_launch_count() - launches0
    st = cp.api._stats(wsp)
    if st["rc"] != 0:
        raise cp.CpError(st["rc"], "T timed steps")
    elapsed = job_time(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    value = job_value(N, ws, args.steps, elapsed)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        c = 64
        crop = np.ascontiguousarray(vol[:c, :c, :c])
        t0 = time.perf_counter()
        oracle.persistence_t(crop)
        dt = time.perf_counter() - t0
        c2 = min(160, int(c * max(1.0, (10.0 / max(dt, 1e-3)) ** (1 / 3) * 0.8)))
        if c2 > c:
            crop = np.ascontiguousarray(vol[:c2, :c2, :c2])
            t0 = time.perf_counter()
            oracle.persistence_t(crop)
            dt = time.perf_counter() - t0
            c = c2
        cpu = {"value": crop.size / dt / 1e6, "unit": "Mvoxels/s", "cores": 1, "host": _host(), "kind": "oracle",
               "sample": f"{c}^3 crop of the {side}^3 volume, T-filtration H0 + H2 pairs, single-threaded C oracle, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": f"Mvoxels/s, T-filtration H0 + H2 pairs ({side}^3 fp32), fwd + loss bwd",
            "value": value, "unit": "Mvoxels/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3D {side}^3 float32 blurred noise (sigma 3 vox), T-filtration (dual image {side + 2}^3), "
                                   "fwd + total-persistence loss bwd", "status": st["rc"], "pairs": st["pairs"],
                       "h0_survivors": st["h0_survivors"], "top_survivors": st["top_survivors"],
                       "h0_roots": st["h0_roots"], "top_roots": st["top_roots"],
                       "rounds": [st["h0_rounds"], st["top_rounds"]],
                       "l2": "input larger than L2; no flush", "parallelism": "replicas" if ws > 1 else "single"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "stages_ms": {k: v / args.steps for k, v in zip(["prune", "sort", "uf", "-", "-", "emit_and_map"], stage_sum)
                          if k != "-"},
            "cpu_baseline": cpu,
        }), flush=True)
    lib.cp_profile(0)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_full(args):
    """The whole diagram of a volume (128^3 blurred, sigma 2, unless --side is
    given): H0, H1 and H2 pairs, forward + total-persistence loss backward,
    device-resident input; the oracle's full diagram on a crop as the CPU
    line."""
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        torch.distributed.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    # 128^3 blurred (sigma 2) by default: the cross-star reduction of a smooth
    # field's long-lived loops runs thousands of rounds, seconds at 128^3
    side = SIDE if "--side" in sys.argv else 128
    sigma = 2.0 if side == 128 else SIGMA
    vol = workloads.blurred((side,) * 3, sigma, 1) if side == 128 else _volume(rank)
    N = vol.size
    x = torch.from_numpy(vol).to(dev)
    from paper_2606_04801_gb300 import autotune

    autotune.autotune([x])
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    dims = (ctypes.c_int64 * 3)(side, side, side)
    one = (ctypes.c_int32 * 1)(3)
    pool = 0
    ws_bytes = lib.cubical_persistence_full_workspace_size(3, dims, 0, pool)
    wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cap = side ** 3 + 65536
    out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
    grad = torch.empty(N, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    bws = lib.cubical_persistence_loss_backward_workspace_size(N)
    bwsp = torch.empty(bws, dtype=torch.uint8, device=dev)
    dcount = torch.zeros(1, dtype=torch.int64, device=dev)

    def step():
        rc = lib.cubical_persistence_full_3d(
            ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
            ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(wsp.data_ptr()), ws_bytes, 0, pool, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "full forward")
        rc = lib.cubical_persistence_loss_backward(
            ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(dcount.data_ptr()), ctypes.c_float(TAU),
            ctypes.c_void_p(loss.data_ptr()), None, ctypes.c_void_p(grad.data_ptr()), N, ctypes.c_void_p(bwsp.data_ptr()),
            bws, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "loss backward")

    def h1_info():
        info = (ctypes.c_int64 * 36)()
        rc = lib.cubical_persistence_full_info(ctypes.c_void_p(wsp.data_ptr()), 1, one, dims, 0, pool, info, 36, sp)
        if rc != 0:
            raise cp.CpError(rc, "full info")
        return [int(v) for v in info]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = cp.api._stats(wsp)
    if st["rc"] != 0:
        raise cp.CpError(st["rc"], f"full warm-up (H1 stage: {h1_info()[:4]})")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    launches0 = lib.cp_launch_count()
    with Clocks(gpu_index) as clk:
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
    launches = lib.cp_launch_count() - launches0
    st = cp.api._stats(wsp)
    if st["rc"] != 0:
        raise cp.CpError(st["rc"], "full timed steps")
    info = h1_info()
    elapsed = job_time(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    value = job_value(N, ws, args.steps, elapsed)
    # the plain H0 + H2 call on the same volume, for the H1 stage's share
    pws = lib.cubical_persistence_workspace_size(3, dims, 0)
    pwsp = torch.empty(pws, dtype=torch.uint8, device=dev)

    def plain():
        rc = lib.cubical_persistence_3d(ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
                                        ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(pwsp.data_ptr()), pws, 0, sp)
        if rc != 0:
            raise cp.CpError(rc, "plain forward")

    for _ in range(3):
        plain()
    ev0.record(stream)
    for _ in range(args.steps):
        plain()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = ev0.elapsed_time(ev1) / args.steps
    del pwsp
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        c = 32
        crop = np.ascontiguousarray(vol[:c, :c, :c])
        t0 = time.perf_counter()
        oracle.persistence_full(crop)
        dt = time.perf_counter() - t0
        c2 = min(64, int(c * max(1.0, (8.0 / max(dt, 1e-3)) ** (1 / 3) * 0.8)))
        if c2 > c:
            crop = np.ascontiguousarray(vol[:c2, :c2, :c2])
            t0 = time.perf_counter()
            oracle.persistence_full(crop)
            dt = time.perf_counter() - t0
            c = c2
        cpu = {"value": crop.size / dt / 1e6, "unit": "Mvoxels/s", "cores": 1, "host": _host(), "kind": "oracle",
               "sample": f"{c}^3 crop of the {side}^3 volume, H0 + H1 + H2 pairs (H1 by the textbook column "
                         f"reduction), single-threaded C oracle, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": f"Mvoxels/s, H0 + H1 + H2 pairs ({side}^3 fp32), fwd + loss bwd",
            "value": value, "unit": "Mvoxels/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3D {side}^3 float32 blurred noise (sigma {sigma:g} vox), whole diagram (H0, H1, H2), "
                                   "fwd + total-persistence loss bwd", "status": st["rc"], "pairs": st["pairs"],
                       "h1_columns": info[0], "h1_columns_leaving_their_star": info[9], "h1_rounds": info[1],
                       "h1_pool_entries_used": info[2], "h1_pool_entries": info[3],
                       "h1_solo_from_round": info[10], "h1_grid_rounds_ms": info[11] / 1e6,
                       "h1_solo_rounds_ms": info[12] / 1e6,
                       "h1_rounds_by_log2_additions": info[13:29],
                       "h1_round_phases_ms": {k: v / 1e6 for k, v in zip(("bids", "wait", "additions", "wait2"),
                                                                          info[29:33])},
                       "h1_additions": info[33], "h1_entries_merged": info[34], "h1_solo_entries": info[35],
                       "plain_h0_h2_forward_ms": plain_ms,
                       "l2": "input larger than L2; no flush", "parallelism": "replicas" if ws > 1 else "single"},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_slabs(args):
    """The slab split of the union-finds on the 512^3 volume (forward, H0 + H2
    pairs): per slab count, the time per call, the stage times and what stage
    1 hands to stage 2 (the records a multi-device run would exchange, 24
    bytes each); the unsplit forward timed the same way beside it."""
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        torch.distributed.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib, autotune

    lib = _lib.load()
    vol = _volume(rank)
    N = vol.size
    x = torch.from_numpy(vol).to(dev)
    autotune.autotune([x])
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    dims = (ctypes.c_int64 * 3)(SIDE, SIDE, SIDE)
    cap = N // 2 + 65536 + 4096
    out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
    dcount = torch.zeros(1, dtype=torch.int64, device=dev)
    slab_counts = [int(v) for v in args.slabs.split(",")]
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) if os.environ.get("CUDA_VISIBLE_DEVICES") else local

    def timed(call, wsp):
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize(dev)
        st = cp.api._stats(wsp)
        if st["rc"] != 0:
            raise cp.CpError(st["rc"], "slabs warm-up")
        stage = (ctypes.c_float * 6)()
        stage_sum = [0.0] * 6
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        lib.cp_profile(1)
        ev0.record(stream)
        for _ in range(args.steps):
            call()
            if lib.cp_stage_times(stage, 6) == 6:
                for i in range(6):
                    stage_sum[i] += stage[i]
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        lib.cp_profile(0)
        st = cp.api._stats(wsp)
        if st["rc"] != 0:
            raise cp.CpError(st["rc"], "slabs timed steps")
        return ev0.elapsed_time(ev1) / args.steps, [v / args.steps for v in stage_sum], st

    # the unsplit forward
    pws = lib.cubical_persistence_workspace_size(3, dims, 0)
    pwsp = torch.empty(pws, dtype=torch.uint8, device=dev)

    def plain():
        rc = lib.cubical_persistence_3d(ctypes.c_void_p(x.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
                                        ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(pwsp.data_ptr()), pws, 0, sp)
        if rc != 0:
            raise cp.CpError(rc, "forward")

    sweep = []
    with Clocks(gpu_index) as clk:
        plain_ms, plain_stages, pst = timed(plain, pwsp)
        ref = out[: int(dcount.item())].clone()
        del pwsp
        for S in slab_counts:
            wsb = lib.cubical_persistence_slabs_workspace_size(3, dims, S, 0)
            wsp = torch.empty(wsb, dtype=torch.uint8, device=dev)
            sst = _lib.CpSlabStats()

            def split(S=S, wsp=wsp, wsb=wsb):
                rc = lib.cubical_persistence_slabs(3, ctypes.c_void_p(x.data_ptr()), dims, S, ctypes.c_void_p(out.data_ptr()),
                                                   cap, None, ctypes.c_void_p(dcount.data_ptr()),
                                                   ctypes.c_void_p(wsp.data_ptr()), wsb, 0, sp, None)
                if rc != 0:
                    raise cp.CpError(rc, "slabs")

            ms, stages, st = timed(split, wsp)
            rc = lib.cubical_persistence_slabs(3, ctypes.c_void_p(x.data_ptr()), dims, S, ctypes.c_void_p(out.data_ptr()),
                                               cap, None, ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(wsp.data_ptr()),
                                               wsb, 0, sp, ctypes.byref(sst))
            if rc != 0:
                raise cp.CpError(rc, "slabs stats")
            same = bool(torch.equal(out[: int(dcount.item())], ref))
            sd = {k: [int(v) for v in getattr(sst, k)] for k, _ in _lib.CpSlabStats._fields_}
            sweep.append({"slabs": S, "ms": ms, "same_as_unsplit": same,
                          "stages_ms": {"prune": stages[0], "roots+sort": stages[1], "stage1": stages[2],
                                        "stage2": stages[4], "emit": stages[5]},
                          "exchange_bytes": 24 * (sd["merged"][0] + sd["merged"][1]), **sd})
            del wsp
    if rank == 0:
        first = sweep[0]
        print(json.dumps({
            "metric": f"Mvoxels/s, H0 + H2 pairs ({SIDE}^3 fp32), union-finds split into slabs, forward",
            "value": N / (first["ms"] / 1e3) / 1e6, "unit": "Mvoxels/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": first["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3D {SIDE}^3 float32 blurred noise (sigma 3 vox), slab split into {first['slabs']} "
                                   "slabs along z (first entry of the sweep)",
                       "l2": "input larger than L2; no flush", "parallelism": "single"},
            "unsplit": {"ms": plain_ms, "stages_ms": {"prune": plain_stages[0], "roots+sort": plain_stages[1],
                                                      "uf": plain_stages[2], "emit": plain_stages[5]},
                        "survivors": [pst["h0_survivors"], pst["top_survivors"]],
                        "rounds": [pst["h0_rounds"], pst["top_rounds"]]},
            "sweep": sweep,
            "clocks": clk.summary(),
        }), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--side", type=int, default=512, help="cube side (512 is the benchmark; smaller for profiling)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--workload", default="volume",
                    choices=["volume", "batched", "survivors", "tfilt", "2d", "full", "slabs"],
                    help="volume: the 512^3 plain path (the headline line); batched: the batched fwd + bwd workload "
                    "alone; survivors: survivor fractions S/N of every config; tfilt: the T-filtration on 510^3; "
                    "2d: the 2048x2048 random field and its 256-level form; full: the whole diagram (H0, H1, H2) "
                    "of the 512^3 volume; slabs: the slab split of the union-finds on the 512^3 volume")
    ap.add_argument("--slabs", default="2,4,8,16,64,152", help="slab counts of the slabs workload (comma-separated)")
    ap.add_argument("--uf-variant", default="auto", choices=["auto", "0", "1"],
                    help="union-find design of the volume workload: the autotuner's pick (auto), reservation rounds "
                    "(0) or Borůvka's forest first (1)")
    ap.add_argument("--eager", action="store_true", help="batched workload without the CUDA graph (per-kernel profiling)")
    args = ap.parse_args()
    global SIDE
    SIDE = args.side
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "survivors":
        run_survivors()
        return
    if args.workload == "tfilt":
        run_tfilt(args)
        return
    if args.workload == "2d":
        run_2d(args)
        return
    if args.workload == "full":
        run_full(args)
        return
    if args.workload == "slabs":
        run_slabs(args)
        return

    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2606_04801_gb300 as cp
    from paper_2606_04801_gb300 import _lib

    lib = _lib.load()
    vol = _volume(rank)
    N = vol.size
    from paper_2606_04801_gb300 import autotune

    tuned = autotune.autotune([torch.from_numpy(vol).to(dev)])
    if args.uf_variant != "auto":  # profiling one union-find design regardless of the tuner's pick
        lib.cp_set_tuning(7, int(args.uf_variant))
        tuned["uf_variant"] = int(args.uf_variant)
    T = (SIDE - 1) ** 3
    x = torch.from_numpy(vol).to(dev)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    dims = (ctypes.c_int64 * 3)(SIDE, SIDE, SIDE)
    ms = 0
    ws_bytes = lib.cubical_persistence_workspace_size(3, dims, ms)
    wsp = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    cap = N // 2 + 65536 + 4096
    out = torch.empty((cap, 8), dtype=torch.int32, device=dev)
    grad = torch.empty(N, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    bws = lib.cubical_persistence_loss_backward_workspace_size(N)
    bwsp = torch.empty(bws, dtype=torch.uint8, device=dev)
    dcount = torch.zeros(1, dtype=torch.int64, device=dev)

    def step(src):
        # forward and loss backward with the pair count kept on the device: no
        # host round trip inside the step (the device status is checked by
        # cubical_persistence_stats after the timed steps, and after every
        # end-to-end step)
        rc = lib.cubical_persistence_3d(
            ctypes.c_void_p(src.data_ptr()), dims, ctypes.c_void_p(out.data_ptr()), cap, None,
            ctypes.c_void_p(dcount.data_ptr()), ctypes.c_void_p(wsp.data_ptr()), ws_bytes, ms, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "forward")
        rc = lib.cubical_persistence_loss_backward(
            ctypes.c_void_p(out.data_ptr()), cap, ctypes.c_void_p(dcount.data_ptr()), ctypes.c_float(TAU),
            ctypes.c_void_p(loss.data_ptr()), None, ctypes.c_void_p(grad.data_ptr()), N, ctypes.c_void_p(bwsp.data_ptr()),
            bws, sp,
        )
        if rc != 0:
            raise cp.CpError(rc, "loss backward")

    def checked(what):
        st = cp.api._stats(wsp)  # reads the call's status/count block back
        if st["rc"] != 0:
            raise cp.CpError(st["rc"], what)
        return st

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---------------- device-resident timing
    lib.cp_profile(1)
    stage = (ctypes.c_float * 6)()
    for _ in range(args.warmup):
        step(x)
    barrier()
    st = checked("warm-up steps")
    k1_ms = []
    stage_sum = [0.0] * 6
    launches0 = lib.cp_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) if os.environ.get("CUDA_VISIBLE_DEVICES") else local
    with Clocks(gpu_index) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step(x)
            if lib.cp_stage_times(stage, 6) == 6:
                k1_ms.append(stage[0])
                for i in range(6):
                    stage_sum[i] += stage[i]
        ev1.record(stream)
        barrier()
    checked("timed steps")
    launches = lib.cp_launch_count() - launches0
    elapsed = job_time(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    value = job_value(N, ws, args.steps, elapsed)

    # ---------------- end to end: pinned host input -> device -> pairs + loss/grad -> loss on host
    # Every step copies its whole input from pinned host memory and reads its status word and
    # loss back.  The headline form is double-buffered the way a serving loop runs: step i+1's
    # host-to-device copy runs on a copy stream while step i computes (two device input buffers,
    # events between the streams), and step i's status and loss land in pinned host slots by
    # asynchronous copies that the host checks while step i+1 runs.  The serial form (copy,
    # compute, read back, one after the other) is reported beside.
    lib.cp_profile(0)
    e2e_steps = 0 if args.no_e2e else max(3, min(args.steps, 10))
    e2e_reps = 3  # each form timed three times, alternating; the median is reported
    e2e_dts, e2e_serial_dts = [], []
    if e2e_steps:
        host = torch.from_numpy(vol).pin_memory()
        xb = [torch.empty_like(x), torch.empty_like(x)]
        cs = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        consumed = [torch.cuda.Event(), torch.cuda.Event()]
        done = [torch.cuda.Event(), torch.cuda.Event()]
        hstat = torch.zeros(2, dtype=torch.int32).pin_memory()  # the status word of the workspace's counters
        hloss = torch.zeros(2, dtype=torch.float64).pin_memory()
        status_word = wsp[0:4].view(torch.int32)

        def read_back(b):
            done[b].synchronize()
            if int(hstat[b]) != 0:
                checked("end-to-end step")  # reads the whole status block and raises
            return float(hloss[b])

        def pipelined():
            barrier()
            t0 = time.perf_counter()
            with torch.cuda.stream(cs):
                xb[0].copy_(host, non_blocking=True)
                copied[0].record(cs)
            for i in range(e2e_steps):
                b = i % 2
                if i + 1 < e2e_steps:
                    nb = 1 - b
                    if i >= 1:
                        cs.wait_event(consumed[nb])  # step i-1 has finished reading that buffer
                    with torch.cuda.stream(cs):
                        xb[nb].copy_(host, non_blocking=True)
                        copied[nb].record(cs)
                stream.wait_event(copied[b])
                step(xb[b])
                consumed[b].record(stream)
                hstat[b:b + 1].copy_(status_word, non_blocking=True)
                hloss[b:b + 1].copy_(loss, non_blocking=True)
                done[b].record(stream)
                if i >= 1:
                    _ = read_back(1 - b)  # step i-1's result, while step i runs
            _ = read_back((e2e_steps - 1) % 2)
            barrier()
            return time.perf_counter() - t0

        def serial():
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                xb[0].copy_(host, non_blocking=True)
                step(xb[0])
                checked("end-to-end step")
                _ = float(loss.item())
            barrier()
            return time.perf_counter() - t0

        for _ in range(e2e_reps):
            e2e_dts.append(pipelined())
            e2e_serial_dts.append(serial())
    e2e_dt = job_time(statistics.median(e2e_dts) if e2e_dts else 1.0, ws, dev)
    e2e_serial_dt = job_time(statistics.median(e2e_serial_dts) if e2e_serial_dts else 1.0, ws, dev)
    e2e = None if not e2e_steps else {
        "value": job_value(N, ws, e2e_steps, e2e_dt),
        "unit": "Mvoxels/s",
        "h2d_bytes_per_step": int(N * 4),
        "d2h_bytes_per_step": 8 + 4,  # the loss and the call's status word
        "pipeline": "double-buffered: step i+1's H2D copy on a second stream overlaps step i; step i's "
                    "status word and loss copied to pinned host slots and checked while step i+1 runs",
        "serial_d2h_bytes_per_step": 8 + COUNTERS_BYTES,  # the loss, and the call's status/count block
        "serial_value": job_value(N, ws, e2e_steps, e2e_serial_dt),
        "repeats": f"median of {e2e_reps} runs of {e2e_steps} steps per form",
        "runs_ms_per_step": [round(1e3 * t / e2e_steps, 3) for t in e2e_dts],
    }
    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return

    # ---------------- roofline of the pruning kernel (K1)
    peak, peak_kind = _peaks()
    k1 = statistics.mean(k1_ms) / 1e3 if k1_ms else None
    s0, stp, r0, rt = st["h0_survivors"], st["top_survivors"], st["h0_roots"], st["top_roots"]
    alg = 4 * N + 4 * N + 4 * (T + 1) + 8 * (s0 + stp) + 16 * (r0 + rt)
    achieved = alg / k1 / 1e9 if k1 else None
    traffic = None
    limiter = None
    tpath = os.path.join(ROOT, "profiles", "k1_prune3d_traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as fh:
                tj = json.load(fh)
            if tj.get("source_hash") == _k1_hash():
                traffic = tj.get("bytes_per_launch_full")
                lm = tj.get("limiter_metrics") or {}
                if lm:
                    limiter = (f"issue/ALU (ncu, {tj['capture']['side']}^3 capture of this source: issue slots "
                               f"{lm['issue_slots_busy_pct']}% busy, ALU pipe {lm['alu_pipe_pct']}%, DRAM "
                               f"{lm['dram_throughput_pct']}%, {lm['warp_instructions'] / lm['vertices'] * 32:.0f} warp "
                               f"instructions per 32 vertices)")
        except Exception:
            traffic = limiter = None
    roofline = {
        "bound": "hbm",
        "achieved": achieved,
        "peak": peak,
        "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None,
        "traffic": traffic,
        "kernel": "k_prune3d",
        # what limits the kernel, from the ncu capture recorded with the traffic
        # (null once the kernel source differs from the captured one)
        "limiter": limiter,
        "peak_source": peak_kind,
        "algorithmic_bytes": alg,
        "read_lower_bound_bytes": 4 * N,  # the image read once, nothing written
        "k1_ms": k1 * 1e3 if k1 else None,
    }
    trace = {}
    for dual, name in ((0, "h0"), (1, "top")):
        act = (ctypes.c_uint32 * 48)()
        us = (ctypes.c_double * 48)()
        usa = (ctypes.c_double * 48)()
        hops = (ctypes.c_uint64 * 48)()
        k = lib.cubical_persistence_uf_trace2(ctypes.c_void_p(wsp.data_ptr()), dual, act, us, usa, hops, 48, sp)
        trace[name] = [[int(act[i]), round(us[i], 1), round(usa[i], 1), int(hops[i])] for i in range(max(0, k))]
    batched = None if args.no_batched else batched_vs_plain(dev, max(3, min(args.steps, 10)), args.warmup)
    cpu = None if args.no_cpu_baseline else cpu_baseline(vol)
    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Mvoxels/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "shape": [SIDE, SIDE, SIDE],
            "note": None if SIDE == 512 else "reduced size for profiling; not the benchmark workload",
            "sigma": SIGMA,
            "loss_min_persistence": TAU,
            "l2": "input (512 MiB) larger than L2; no flush",
            "parallelism": "replicas" if ws > 1 else "single",
            "tuning": {k: tuned[k] for k in ("zchunk3d", "ctas3d", "rows2d", "uf_variant")},
        },
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "stages_ms": {
            k: v / max(1, len(k1_ms))
            for k, v in zip(["prune", "sort_h0", "uf_h0", "sort_top", "uf_top", "emit"], stage_sum)
        },
        "batched": batched,
        "uf_trace": trace,
        "counts": {"pairs": st["pairs"], "h0_survivors": s0, "top_survivors": stp, "h0_roots": r0, "top_roots": rt,
                   "survivor_fraction": (s0 + stp) / N,
                   "h0_rounds": st["h0_rounds"], "top_rounds": st["top_rounds"],
                   "mst_rounds": st.get("mst_rounds", 0)},
    }
    print(json.dumps(line), flush=True)


def _k1_hash():
    import hashlib

    h = hashlib.sha256()
    for f in ("cp_prune.cu", "cp_common.cuh", "cp_mask3.cuh"):
        with open(os.path.join(ROOT, "paper_2606_04801_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
