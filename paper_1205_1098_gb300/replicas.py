"""Replica bookkeeping for runs on several GPUs of one node.

The fused kernels do not shard: on N GPUs every rank runs the whole workload
on its own data (independent replicas, no collective on the data path).  A
run therefore reports the bytes all replicas moved over the time of the
slowest replica.  The only collectives are these reductions of one scalar
and the barriers around the timed region.  They take a torch.distributed
module with an initialised process group (NCCL for GPU runs, gloo for the
CPU tests), or None for a single process.
"""


def _reduce(torch, dist, value, op, device):
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(torch, dist, value, device="cpu"):
    """Largest value over the ranks (the local value without a process group)."""
    return _reduce(torch, dist, value, dist.ReduceOp.MAX if dist is not None else None, device)


def sum_over_ranks(torch, dist, value, device="cpu"):
    """Sum of the value over the ranks (the local value without a process group)."""
    return _reduce(torch, dist, value, dist.ReduceOp.SUM if dist is not None else None, device)


def job_rate(torch, dist, local_bytes, local_ms, device="cpu"):
    """Whole-job throughput of independent replicas: (GB/s over all ranks'
    bytes and the slowest rank's time, that time in ms)."""
    ms = max_over_ranks(torch, dist, local_ms, device)
    total = sum_over_ranks(torch, dist, local_bytes, device)
    return total / (ms * 1e-3) / 1e9, ms


def barrier(torch, dist):
    """Barrier across the ranks and the local device (no-op for one CPU process)."""
    if dist is not None:
        dist.barrier()
    if torch.cuda.is_available() and torch.cuda.is_initialized():
        torch.cuda.synchronize()
