"""Multi-process (gloo, world size 2) checks of the sharding and timing aggregate."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2412_14775_b300.shard import aggregate, shard_streams


def test_shard_streams_partitions_and_balances():
    rows = [300 * 16, 741 * 32, 1176 * 64, 1953 * 128, 2926 * 64, 300 * 32, 1176 * 16, 1953 * 64]
    for ws in (1, 2, 3, 4, 8):
        parts = [shard_streams(rows, ws, r) for r in range(ws)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(rows)))
        loads = [sum(rows[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(rows)
    with pytest.raises(ValueError):
        shard_streams(rows, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    units, secs = (1000 * (rank + 1), 0.5 + rank)
    q.put((rank, aggregate(units, secs), shard_streams([5, 9, 2, 7], ws, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for _, (u, t, v), _ in res:
        assert u == 3000.0 and t == 1.5 and abs(v - 2000.0) < 1e-9
    owned = sorted(i for _, _, s in res for i in s)
    assert owned == [0, 1, 2, 3]


def test_aggregate_single_process():
    assert aggregate(10, 2.0) == (10.0, 2.0, 5.0)
