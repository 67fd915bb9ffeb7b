"""Replica bookkeeping of multi-GPU runs, on two gloo ranks on the CPU (the
kernels do not shard: each rank runs the whole workload; the job reports all
ranks' bytes over the slowest rank's time)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1205_1098_gb300 import replicas
    gbs, ms = replicas.job_rate(torch, dist, 1e9 * (rank + 1), 10.0 + rank)
    mx = replicas.max_over_ranks(torch, dist, 3.0 * rank)
    sm = replicas.sum_over_ranks(torch, dist, rank + 1)
    replicas.barrier(torch, dist)
    out.put((rank, gbs, ms, mx, sm))
    dist.destroy_process_group()


def test_job_rate_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=180)
    assert sorted(r[0] for r in res) == [0, 1]
    for _, gbs, ms, mx, sm in res:
        assert ms == 11.0          # the slowest rank's time
        assert mx == 3.0 and sm == 3.0
        assert abs(gbs - 3e9 / 11e-3 / 1e9) < 1e-9   # all ranks' bytes over that time
    assert all(p.exitcode == 0 for p in procs)


def test_single_process_needs_no_group():
    from paper_1205_1098_gb300 import replicas
    gbs, ms = replicas.job_rate(torch, None, 2e9, 4.0)
    assert ms == 4.0 and gbs == 500.0
    assert replicas.max_over_ranks(torch, None, 7.5) == 7.5
