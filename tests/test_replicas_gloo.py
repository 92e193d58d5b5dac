"""Multi-GPU is replicas only (independent transforms, no data-path
collective): the benchmark's per-rank timing is combined as max over ranks and
whole-job throughput = all ranks' work / slowest rank's time.  Checked here
with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_seconds = [2.0, 3.0][rank]
    bench.barrier(dist)
    t = bench.reduce_max(per_rank_seconds, dist, "cpu")
    v = bench.job_value(1000.0, world, t)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_replicas_max_time_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in res:
        assert t == pytest.approx(3.0)          # the slowest rank sets the time
        assert v == pytest.approx(2000.0 / 3.0)  # both ranks' units / max time
