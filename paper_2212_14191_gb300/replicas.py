"""Host-side coordination of independent replicas, one process per GPU.

Every limb transform and every ciphertext pair of the batched path is independent (the
batch dimension of the (L, B, N) layout, Sec. IV-D), so ranks never exchange data on the
path. They only agree on the timed region (a barrier on both sides of it), derive disjoint
input seeds from their rank, and report the whole-job rate as the units all ranks
processed divided by the slowest rank's elapsed time.
"""
import os

import torch


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment; (1, 0, 0) without it."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init(ws, backend, device=None):
    """Join the process group when ws > 1 (nccl for GPU ranks, gloo for host-only ranks)."""
    if ws <= 1:
        return
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=device)
    else:
        dist.init_process_group(backend)


def finish(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def rank_seed(base, rank):
    """Seed of a rank's synthetic inputs: disjoint problems per rank."""
    return int(base) + 7919 * int(rank)


def barrier(ws, cuda=True):
    """All ranks reach this point, then the local device is drained."""
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def max_over_ranks(v, ws, device="cuda"):
    """The largest v over all ranks (the slowest rank's elapsed time)."""
    if ws <= 1:
        return float(v)
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, slowest_seconds):
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    if slowest_seconds <= 0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * ws / slowest_seconds
