"""Multi-rank host logic on CPU: world size 2 over gloo (127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2501_16909_b300 import replicas


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
    try:
        cells = [(v, r, l) for v in range(5) for r in range(3) for l in range(4)]
        mine = replicas.shard(cells, world, rank)
        rows = [{"cell": c, "rank": rank} for c in mine]
        allrows = replicas.gather_rows(rows)
        t = replicas.max_over_ranks([1.0 + rank, 10.0 - rank])
        replicas.barrier()
        q.put((rank, len(mine), [r["cell"] for r in allrows], t))
    finally:
        dist.destroy_process_group()


def test_shard_round_robin_partition():
    items = list(range(11))
    parts = [replicas.shard(items, 3, r) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert parts[0] == [0, 3, 6, 9] and parts[2] == [2, 5, 8]
    with pytest.raises(ValueError):
        replicas.shard(items, 2, 2)


def test_single_process_fallbacks():
    assert replicas.max_over_ranks([1, 2.5]) == [1.0, 2.5]
    assert replicas.gather_rows([1, 2]) == [1, 2]


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    cells = [(v, r, l) for v in range(5) for r in range(3) for l in range(4)]
    (r0, n0, all0, t0), (r1, n1, all1, t1) = out
    assert n0 + n1 == len(cells)
    assert sorted(all0) == sorted(cells) and all0 == all1  # every cell exactly once, same order on both ranks
    assert t0 == t1 == [2.0, 10.0]
