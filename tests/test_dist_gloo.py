"""The multi-rank host logic on CPU processes over gloo (world size 2): the
timing collectives, the per-rank seeds and the partition of units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

from paper_1604_04740_gb300 import dist as D  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    D.init("gloo")
    r, w, lr = D.world_info()
    D.barrier()
    mx = D.max_over_ranks(10.0 + r, "cpu")
    sm = D.sum_over_ranks(1.0 + r, "cpu")
    start, stop = D.shard(4097, w, r)
    q.put((r, w, lr, mx, sm, start, stop, D.rank_seed(0, r)))
    D.barrier()
    D.finish()


def test_two_ranks_over_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == 11.0 for x in res)            # max of 10 and 11 on every rank
    assert all(x[4] == 3.0 for x in res)             # 1 + 2
    spans = [(x[5], x[6]) for x in res]
    assert spans[0][0] == 0 and spans[0][1] == spans[1][0] and spans[1][1] == 4097
    assert res[0][7] == 0 and res[1][7] != 0         # rank 0 keeps the one-GPU workload


def test_shard_partitions_any_count():
    for n in (0, 1, 5, 64, 4097):
        for w in (1, 2, 3, 8):
            spans = [D.shard(n, w, r) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
