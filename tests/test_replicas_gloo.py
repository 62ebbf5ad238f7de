"""The multi-GPU path is replicas (every rank its own volume, no data-path
collective): the host logic of the benchmark -- each rank's workload, the
max over ranks of the timed region, the whole-job throughput -- checked with
two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        assert (ws, r, local) == (world, rank, rank)
        bench.SIDE = 12
        vol = bench._volume(rank)  # each replica its own volume (seed = rank)
        digest = torch.tensor([float(vol.sum())], dtype=torch.float64)
        sums = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sums, digest)
        local_s = 1.0 + 0.25 * rank  # this rank's timed region
        t = bench.job_time(local_s, world, torch.device("cpu"))
        out.put((rank, t, bench.job_value(vol.size, world, 10, t), [float(x) for x in sums]))
    finally:
        dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    times = [r[1] for r in res]
    assert times == [1.25, 1.25]  # the job ends with its slowest rank
    n = 12 ** 3
    assert all(abs(r[2] - n * world * 10 / 1.25 / 1e6) < 1e-12 for r in res)
    sums = res[0][3]
    assert sums[0] != sums[1]  # replicas work on different volumes


def test_job_value_single_rank():
    import bench

    assert bench.job_time(2.5, 1, None) == 2.5
    assert bench.job_value(1e6, 1, 4, 2.0) == 2.0
