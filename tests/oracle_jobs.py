"""Oracle runs on the full-size workloads, in background processes.

The oracle is single-threaded and needs minutes on the 512^3 volume, so the
full-size parity tests start it early (from ``conftest.py``, once the test
selection is known) in processes of the ``spawn`` start method, and the GPU
tests run meanwhile.  Each job regenerates its input from the seeded recipe
in ``workloads`` (nothing large crosses a process boundary) and writes the
oracle's pairs to ``<dir>/<job>.npy``; the test waits for the file.

Jobs:
  ``3d_512``    the 512^3 blurred volume (sigma 3, seed 0): the benchmark's
                workload;
  ``batch_<i>`` item i of the batched workload ``workloads.batch(0)`` (64
                images and 8 volumes, rank-spaced).

Test infrastructure only: nothing outside ``tests/`` imports this module.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile
import time

import numpy as np

_state = {"dir": None, "procs": [], "jobs": set()}


def _job_input(job: str):
    import workloads

    if job == "3d_512":
        return workloads.config("3d_512_blurred")[0]
    if job.startswith("batch_"):
        i = int(job.split("_")[1])
        s2, s3 = workloads.batch_shapes(0)
        shape = (s2 + s3)[i]
        sigma = 4.0 if len(shape) == 2 else 2.0
        return workloads.rank_spaced(workloads.blurred(shape, sigma, 1000 + i))
    raise KeyError(job)


def _worker(jobs, out_dir):
    import oracle

    for job in jobs:
        img = _job_input(job)
        p = oracle.persistence(img)
        tmp = os.path.join(out_dir, f".{job}.{os.getpid()}.npy")
        np.save(tmp, p)
        os.replace(tmp, os.path.join(out_dir, f"{job}.npy"))


def batch_jobs():
    import workloads

    s2, s3 = workloads.batch_shapes(0)
    return [f"batch_{i}" for i in range(len(s2) + len(s3))]


def job_size(job: str) -> int:
    import workloads

    if job == "3d_512":
        return 512 ** 3
    s2, s3 = workloads.batch_shapes(0)
    return int(np.prod((s2 + s3)[int(job.split("_")[1])]))


def start(jobs, workers: int | None = None) -> None:
    """Starts the jobs not yet started, spread over `workers` processes
    (largest first, each to the least loaded process)."""
    todo = [j for j in jobs if j not in _state["jobs"]]
    if not todo:
        return
    if _state["dir"] is None:
        _state["dir"] = tempfile.mkdtemp(prefix="cp_oracle_jobs_")
    if workers is None:
        workers = max(1, min(len(todo), (os.cpu_count() or 2) - 2, 12))
    todo.sort(key=job_size, reverse=True)
    bins = [[] for _ in range(workers)]
    load = [0] * workers
    for j in todo:
        k = int(np.argmin(load))
        bins[k].append(j)
        load[k] += job_size(j)
    ctx = mp.get_context("spawn")
    for b in bins:
        if not b:
            continue
        p = ctx.Process(target=_worker, args=(b, _state["dir"]), daemon=True)
        p.start()
        _state["procs"].append(p)
    _state["jobs"].update(todo)


def result(job: str, timeout_s: float = 3600.0) -> np.ndarray:
    """The oracle's pairs for a job (starting it if needed), waiting up to
    timeout_s; fails early if every worker has exited without writing it."""
    if job not in _state["jobs"]:
        start([job], workers=1)
    path = os.path.join(_state["dir"], f"{job}.npy")
    t0 = time.time()
    while not os.path.exists(path):
        if all(not p.is_alive() for p in _state["procs"]) and not os.path.exists(path):
            codes = [p.exitcode for p in _state["procs"]]
            raise RuntimeError(f"oracle job {job}: workers exited ({codes}) without a result")
        if time.time() - t0 > timeout_s:
            raise TimeoutError(f"oracle job {job} not done after {timeout_s:.0f} s")
        time.sleep(0.5)
    return np.load(path)


def stop() -> None:
    """Ends the workers this module started (by their own process objects)."""
    for p in _state["procs"]:
        if p.is_alive():
            p.terminate()
    for p in _state["procs"]:
        p.join(timeout=10)
    _state["procs"].clear()
    _state["jobs"].clear()
