"""The multi-GPU path on CPU: world_size-2 gloo process groups run the rank
logic the benchmark uses (instance sharding, barrier, max and sum over
ranks); no GPU and no data-path collective are involved."""
import os
import socket

import pytest

from paper_1010_3816_gb300.distributed import shard


def test_shard_covers_every_item_once_and_balances():
    costs = [5.0, 1.0, 3.0, 3.0, 8.0, 2.0, 2.0, 7.0, 1.0]
    for world in (1, 2, 3, 4):
        parts = [shard(costs, r, world) for r in range(world)]
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        shard(costs, 2, 2)


def test_shard_batched_workload():
    from inputs import batched_instances
    inst = batched_instances()
    costs = [w.points for w in inst]
    a, b = shard(costs, 0, 2), shard(costs, 1, 2)
    assert sorted(a + b) == list(range(24))
    la, lb = sum(costs[k] for k in a), sum(costs[k] for k in b)
    assert abs(la - lb) / (la + lb) < 0.05


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1010_3816_gb300 import distributed as D
    D.barrier()
    mx = D.reduce_max(10.0 + rank)
    sm = D.reduce_sum(1.5 * (rank + 1))
    mine = D.shard([3.0, 1.0, 2.0, 2.0], rank, world)
    D.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, sm, mine))


def test_two_rank_gloo_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [11.0, 11.0]
    assert [o[2] for o in out] == [4.5, 4.5]
    assert sorted(out[0][3] + out[1][3]) == [0, 1, 2, 3]
