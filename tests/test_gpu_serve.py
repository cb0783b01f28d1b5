"""GPU tests of the continuous-batching serving loop: every request's result
is bit-identical alone and in the overlapping mix (tolerance: zero) and
equals the oracle's direct result, lost-stream requests are recovered,
admission respects the HBM budget, and the plain comparison path computes the
plain operation."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    from paper_1604_04740_gb300 import serve as S
    return B, ne, S


def _direct(ne, srv, rq):
    s = rq.spec
    c = srv.c_host[rq.c_pool:rq.c_pool + s.M * s.positions_in].numpy()
    op = srv.op_host[rq.op_pool:rq.op_pool + s.op_bytes].numpy()
    if s.kind == ne.NE_JOB_GEMM:
        d = oracle.gemm_direct(c.reshape(s.M, s.rows, s.k), op.reshape(s.k, s.cols))
    else:
        d = oracle.cconv_direct(c.reshape(1, s.M, s.N), op.reshape(1, s.N))
    return d.reshape(-1)


@pytest.mark.parametrize("rate,lanes,max_batch,budget,work", [(20000.0, 3, 8, 96 << 20, None),
                                                              (50000.0, 4, 6, 48 << 20, None),
                                                              (2000.0, 2, 64, 512 << 20, None),
                                                              (50000.0, 4, 64, 512 << 20, 3e7)])
def test_mix_equals_alone_and_oracle(mods, rate, lanes, max_batch, budget, work):
    B, ne, S = mods
    specs = B.mixed_jobs(21, 40, mnk=(16, 192), conv=(64, 4096), recover_frac=0.15)
    assert any(s.fuse == ne.NE_FUSE_RECOVER for s in specs)
    srv = S.Server(budget_bytes=budget, lanes=lanes, max_batch=max_batch, keep_outputs=True, host_pool_elems=1 << 22,
                   max_batch_work=work)
    reqs = srv.run(specs, S.poisson_arrivals(3, len(specs), rate), seed=5)
    assert all(rq.done >= rq.arrival for rq in reqs)
    assert srv.pool.used == 0 and srv.flagged == 0
    alone = S.Server(budget_bytes=budget, lanes=1, keep_outputs=True, host_pool_elems=1 << 22)
    for rq in reqs:
        alone.outputs.clear()
        alone.run([rq.spec], np.zeros(1), offsets=[(rq.c_pool, rq.op_pool)])
        assert (alone.outputs[0] == srv.outputs[rq.idx]).all(), f"request {rq.idx}: alone differs from the mix"
        assert (srv.outputs[rq.idx] == _direct(ne, srv, rq)).all(), f"request {rq.idx} ({rq.spec})"


def test_transform_path_in_the_mix_equals_the_tensor_path_alone(mods):
    # convolutions of N >= 1024 run as exact transforms in the mix; alone they run on tensor tiles
    B, ne, S = mods
    specs = B.mixed_jobs(23, 40, mnk=(16, 192), conv=(64, 4096), recover_frac=0.15)
    specs += S.plain_copy(B.mixed_jobs(24, 6, mnk=(16, 64), conv=(1024, 4096)))
    srv = S.Server(budget_bytes=256 << 20, lanes=3, max_batch=8, keep_outputs=True, host_pool_elems=1 << 22,
                   cfg=B.default_config(ntt_min_n=1024))
    reqs = srv.run(specs, S.poisson_arrivals(4, len(specs), 20000.0), seed=6)
    assert srv.pool.used == 0 and srv.flagged == 0
    alone = S.Server(budget_bytes=256 << 20, lanes=1, keep_outputs=True, host_pool_elems=1 << 22)
    for rq in reqs:
        alone.outputs.clear()
        alone.run([rq.spec], np.zeros(1), offsets=[(rq.c_pool, rq.op_pool)])
        assert (alone.outputs[0] == srv.outputs[rq.idx]).all(), f"request {rq.idx}: transform mix differs"
        assert (srv.outputs[rq.idx] == _direct(ne, srv, rq)).all(), f"request {rq.idx} ({rq.spec})"


def test_plain_path_computes_the_plain_operation(mods):
    B, ne, S = mods
    specs = S.plain_copy(B.mixed_jobs(22, 16, mnk=(16, 192), conv=(64, 4096)))
    srv = S.Server(budget_bytes=128 << 20, lanes=2, keep_outputs=True, host_pool_elems=1 << 22)
    reqs = srv.run(specs, S.poisson_arrivals(5, len(specs), 10000.0), seed=7)
    for rq in reqs:
        assert (srv.outputs[rq.idx] == _direct(ne, srv, rq)).all()


def test_pool_allocator_coalesces(mods):
    B, ne, S = mods
    p = S.Pool(1 << 20, "cuda")
    a = p.alloc(1000)
    b = p.alloc(5000)
    c = p.alloc(300)
    assert a and b and c
    p.release(*b)
    p.release(*a)
    p.release(*c)
    assert p.used == 0 and p.free == [(0, p.size)]
    assert p.alloc(p.size + 1) is None


@pytest.mark.parametrize("count", [1, 7, 300])
def test_copy_regions_gathers_every_byte(mods, count):
    # regions of odd sizes at odd offsets (and empty ones), one copy per
    # region; bytes outside the regions stay untouched
    _, ne, _ = mods
    rng = np.random.default_rng(count)
    src = torch.from_numpy(rng.integers(0, 256, 1 << 20, dtype=np.uint8)).pin_memory()
    nbytes = rng.integers(0, 3000, count).astype(np.int64)
    nbytes[::5] = 0
    src_off = rng.integers(0, src.numel() - 3000, count).astype(np.int64)
    dst_off = np.concatenate([[3], 3 + np.cumsum(nbytes + rng.integers(0, 40, count))[:-1]]).astype(np.int64)
    size = int(dst_off[-1] + nbytes[-1] + 64)
    dst = torch.full((size,), 7, dtype=torch.uint8, device="cuda")
    ne.ne_copy_regions_h2d(dst, src, dst_off, src_off, nbytes)
    got = dst.cpu().numpy()
    want = np.full(size, 7, np.uint8)
    s = src.numpy()
    for d, o, b in zip(dst_off, src_off, nbytes):
        want[d:d + b] = s[o:o + b]
    assert (got == want).all()
