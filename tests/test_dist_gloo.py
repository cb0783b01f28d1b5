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


# ---- one stream per rank (the paper's distribution): exchange, check, recovery ----------

def _stream_worker(rank, world, store_port, q, dead, flip):
    """Rank m computes only its stream's circular convolution delta_m (here
    with the oracle; on GPUs with the library), the ranks exchange by
    position block, and each checks (or, after a failure, recovers) its block."""
    import datetime

    import numpy as np
    import torch.distributed as dist

    import oracle
    from paper_1604_04740_gb300 import inputs

    store = dist.TCPStore("127.0.0.1", store_port, world, False, timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=dist.PrefixStore("pg", store), rank=rank, world_size=world)
    groups = D.stream_groups(world)
    M, n, l = world, 1000, 16
    c = inputs.streams(5 + world, (1, M, n))
    g = inputs.operator_int8(5 + world, (1, n))
    eps_m = oracle.entangle(c, l)[:, rank:rank + 1]                 # this rank's stream only
    delta_m = oracle.cconv(eps_m, g)[0, 0]
    if flip is not None and flip[0] == rank:
        delta_m[flip[1]] ^= np.int64(1 << flip[2])
    if rank == dead:
        q.put((rank, "failed"))                                      # fail-stop: never posts, never exchanges
        return
    lost = D.heartbeat(store, 0, rank, world, timeout_s=3.0)
    d = lost[0] if lost else None
    block, start, stop = D.exchange_streams(torch.from_numpy(delta_m), rank, world, d, groups)
    blk = block.numpy()[None]
    direct = oracle.cconv_direct(c, g)[0][:, start:stop]
    if d is None:
        dh, fl = oracle.extract(blk, l, 0)
        flagged = [start + int(i) for i in np.nonzero(fl[0])[0]]
    else:
        dh, flagged = oracle.recover(blk, l, d), []
    q.put((rank, lost, start, stop, bool((dh[0] == direct).all()) if not flagged else flagged))
    dist.barrier(group=groups[d] if d is not None else None)
    dist.destroy_process_group()


def _run_streams(world, dead=None, flip=None):
    import datetime

    import torch.distributed as dist
    port = _free_port()
    store = dist.TCPStore("127.0.0.1", port, world + 1, True, timeout=datetime.timedelta(seconds=60),
                          wait_for_workers=False)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_stream_worker, args=(r, world, port, q, dead, flip)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    del store
    return res


@pytest.mark.parametrize("world", [3, 4])
def test_streams_exchange_and_check_by_position_block(world):
    res = _run_streams(world)
    assert [r[0] for r in res] == list(range(world))
    assert res[0][2] == 0 and res[-1][3] == 1000
    assert all(res[i][3] == res[i + 1][2] for i in range(world - 1))
    assert all(r[1] == [] and r[4] is True for r in res)


def test_a_flipped_bit_is_flagged_by_the_rank_owning_its_block():
    res = _run_streams(3, flip=(1, 777, 41))
    owner = [r for r in res if r[2] <= 777 < r[3]]
    assert len(owner) == 1 and owner[0][4] == [777]
    assert all(r[4] is True for r in res if r is not owner[0])


@pytest.mark.parametrize("world,dead", [(3, 1), (4, 0), (4, 3)])
def test_survivors_rebuild_every_output_without_the_failed_rank(world, dead):
    res = _run_streams(world, dead=dead)
    live = [r for r in res if r[1] != "failed"]
    assert len(live) == world - 1 and res[dead][1] == "failed"
    assert all(r[1] == [dead] and r[4] is True for r in live)
    spans = sorted((r[2], r[3]) for r in live)
    assert spans[0][0] == 0 and spans[-1][1] == 1000
    assert all(spans[i][1] == spans[i + 1][0] for i in range(len(spans) - 1))
