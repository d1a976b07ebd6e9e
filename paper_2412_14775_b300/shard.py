"""Host-side sharding over GPUs: the path has no exchange step.

Every (stream, baseline, channel) row is flagged independently (each correlator
stream is mitigated separately), so N GPUs take disjoint sets of streams and never
communicate on the data path.  Only the timing is combined: the job's time is the
slowest rank's, and its throughput the total work over that time.
"""


def shard_streams(stream_rows, world_size, rank):
    """Indices of the streams owned by `rank`: longest-processing-time-first greedy
    assignment by row count, deterministic for every rank."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world size or rank")
    load = [0] * world_size
    owner = {}
    for i in sorted(range(len(stream_rows)), key=lambda i: (-stream_rows[i], i)):
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += stream_rows[i]
    return sorted(i for i, r in owner.items() if r == rank)


def aggregate(local_units, local_seconds, group=None):
    """(total units over ranks, max seconds over ranks, units / max seconds).

    Without an initialised process group this is the single-process value."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_units), float(local_seconds), local_units / local_seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(t.item()), float(u.item()) / float(t.item())
