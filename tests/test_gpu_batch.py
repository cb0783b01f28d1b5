"""GPU tests of the ragged batch runner (persistent launches over mixed
product/convolution jobs, long convolutions on transforms): parity with the
oracle, detection of exactly the injected faults (sparse and dense),
batch-versus-alone equality, every tuner configuration, CUDA-graph replay,
and fused recovery of lost streams."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    return B, ne


def small_specs(B, ne):
    G, C, R = ne.NE_JOB_GEMM, ne.NE_JOB_CCONV, ne.NE_FUSE_RECOVER
    specs = [
        B.JobSpec(G, 3, rows=40, cols=72, k=48), B.JobSpec(G, 4, rows=16, cols=64, k=256),
        B.JobSpec(G, 5, rows=100, cols=136, k=32), B.JobSpec(C, 3, N=64), B.JobSpec(C, 4, N=1088),
        B.JobSpec(C, 5, N=256), B.JobSpec(C, 3, N=2048), B.JobSpec(G, 3, rows=33, cols=8, k=16, fuse=R, r=1),
        B.JobSpec(C, 4, N=512, fuse=R, r=3), B.JobSpec(G, 4, rows=1, cols=16, k=16),
    ]
    return specs + B.mixed_jobs(7, 14, mnk=(16, 160), conv=(64, 2048))


def job_l(spec, ne):
    K = spec.k if spec.kind == ne.NE_JOB_GEMM else spec.N
    return oracle.choose_l(spec.M, 64, K * 128 * 128, oracle.POLICY_BYTE)[0]


def oracle_job(b, j, ne, faults=True):
    """(d_hat, flags) the oracle gives for job j of batch b, with b's faults."""
    s = b.specs[j]
    c, op = b.job_inputs(j)
    l = job_l(s, ne)
    if s.kind == ne.NE_JOB_GEMM:
        eps = oracle.entangle(c.reshape(s.M, -1), l).reshape(s.M, s.rows, s.k)
        delta = np.stack([oracle.gemm(eps[m], op) for m in range(s.M)]).reshape(s.M, -1)
    else:
        delta = oracle.cconv(oracle.entangle(c, l), op).reshape(s.M, -1)
    if faults and b.faults is not None:
        sel = b.faults["job"] == j
        for p, m, bit in zip(b.faults["pos"][sel], b.faults["stream"][sel], b.faults["bit"][sel]):
            delta[m, p] ^= np.int64(np.uint64(1 << int(bit)).view(np.int64))
    if s.fuse == ne.NE_FUSE_RECOVER:
        return oracle.recover(delta, l, s.r), None
    dh, fl = oracle.extract(delta, l, s.r)
    return dh, fl


def test_device_generator_matches_host_generator(mods):
    dev = inputs.int8_uniform_device(3, inputs.TAG_C, 100003, 12345, "cuda").cpu().numpy()
    assert (dev == inputs.int8_uniform(3, inputs.TAG_C, (100003,), start=12345)).all()


def test_batch_matches_oracle_and_flags_exactly_the_faults(mods):
    B, ne = mods
    b = B.Batch(small_specs(B, ne), seed=4, fault_rate=2e-3)
    b.plan(B.default_config())
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    total = 0
    for j, s in enumerate(b.specs):
        dh, fl = oracle_job(b, j, ne)
        got = b.job_output(j).cpu().numpy().reshape(s.M, -1)
        assert (got == dh).all(), f"job {j} ({s})"
        if fl is not None:
            gf = unpack_flags(b.job_flags(j).cpu().numpy(), 1, s.positions_out)[0]
            assert (gf == fl).all(), f"job {j} flags"
            assert (gf == B.expected_flags(b, j)).all(), f"job {j}: flags are not exactly the injected faults"
            total += int(fl.sum())
    assert b.faults is not None and int(b.nflag.item()) == total == len(b.faults["pos"])


def test_dense_faults_take_the_band_scan_and_match_the_oracle(mods):
    # a flip in 3 % of the output words: product tiles hold more faults than
    # their shared-memory list (64), so positions scan the tile's row band
    B, ne = mods
    G, C = ne.NE_JOB_GEMM, ne.NE_JOB_CCONV
    specs = [B.JobSpec(G, 5, rows=64, cols=128, k=64), B.JobSpec(G, 3, rows=33, cols=200, k=48),
             B.JobSpec(G, 4, rows=20, cols=64, k=32), B.JobSpec(C, 4, N=1024), B.JobSpec(C, 3, N=5120)]
    b = B.Batch(specs, seed=12, fault_rate=0.03)
    b.plan(B.default_config(ntt_min_n=4096))
    assert b.info.ntransform == 1
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    tile0 = b.faults["pos"][(b.faults["job"] == 0) & (b.faults["pos"] < 16 * 128)]
    assert (tile0 % 128 < 64).sum() > 64          # the first tile of job 0 overflows the list
    total = 0
    for j, s in enumerate(b.specs):
        dh, fl = oracle_job(b, j, ne)
        got = b.job_output(j).cpu().numpy().reshape(s.M, -1)
        assert (got == dh).all(), f"job {j} ({s})"
        gf = unpack_flags(b.job_flags(j).cpu().numpy(), 1, s.positions_out)[0]
        assert (gf == fl).all() and (gf == B.expected_flags(b, j)).all(), f"job {j} flags"
        total += int(fl.sum())
    assert int(b.nflag.item()) == total == len(b.faults["pos"])


def test_transform_path_matches_oracle_tensor_path_and_graph(mods):
    # convolutions of N >= 512 leave the tensor tiles for the exact transforms
    B, ne = mods
    specs = small_specs(B, ne) + [B.JobSpec(ne.NE_JOB_CCONV, 3, N=4160), B.JobSpec(ne.NE_JOB_CCONV, 5, N=8192),
                                  B.JobSpec(ne.NE_JOB_CCONV, 4, N=2112, fuse=ne.NE_FUSE_RECOVER, r=0)]
    b = B.Batch(specs, seed=10, fault_rate=2e-3)
    b.plan(B.default_config(ntt_min_n=512))
    assert b.info.ntransform >= 5
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    total = 0
    for j, s in enumerate(b.specs):
        dh, fl = oracle_job(b, j, ne)
        got = b.job_output(j).cpu().numpy().reshape(s.M, -1)
        assert (got == dh).all(), f"job {j} ({s})"
        if fl is not None:
            gf = unpack_flags(b.job_flags(j).cpu().numpy(), 1, s.positions_out)[0]
            assert (gf == fl).all() and (gf == B.expected_flags(b, j)).all(), f"job {j} flags"
            total += int(fl.sum())
    assert int(b.nflag.item()) == total == len(b.faults["pos"])
    out_t, fl_t = b.out.clone(), b.flags.clone()
    # the tensor tiles give the same bits
    b.plan(B.default_config(ntt_min_n=0))
    b.run()
    torch.cuda.synchronize()
    assert torch.equal(b.out, out_t) and torch.equal(b.flags, fl_t)
    # and so does a graph replay of the transform plan
    b.plan(B.default_config(ntt_min_n=512))
    b.capture()
    b.out.fill_(0)
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.out, out_t) and torch.equal(b.flags, fl_t)


def test_batch_equals_each_job_alone_and_direct_results(mods):
    B, ne = mods
    b = B.Batch(small_specs(B, ne), seed=5)
    b.plan(B.default_config())
    b.run()
    torch.cuda.synchronize()
    for j, s in enumerate(b.specs):
        c, op = b.job_inputs(j)
        got = b.job_output(j).cpu().numpy()
        direct = oracle.gemm_direct(c, op) if s.kind == ne.NE_JOB_GEMM else oracle.cconv_direct(c, op)
        assert (got == direct.reshape(got.shape)).all(), f"job {j}"
        # the same job through the stand-alone entry points
        l = job_l(s, ne)
        p = ne.params(s.M, l)
        dg = ne.ne_plan_digits(l, -128, 127)
        cd, od = torch.from_numpy(c).cuda(), torch.from_numpy(op).cuda()
        if s.kind == ne.NE_JOB_GEMM:
            pl = ne.ne_entangle_digits(p, dg, cd.reshape(s.M, -1)).reshape(s.M, dg.S, s.rows, s.k)
            alone = ne.ne_gemm_digits(p, dg, pl, od, fuse=s.fuse, r=s.r)
        else:
            pl = ne.ne_entangle_digits(p, dg, cd)
            alone = ne.ne_cconv_digits(p, dg, pl, od, fuse=s.fuse, r=s.r)
        assert (alone.cpu().numpy().reshape(got.shape) == got).all(), f"job {j}: batch differs from alone"


def test_every_tuner_configuration_gives_the_same_bits(mods):
    B, ne = mods
    from paper_1604_04740_gb300 import autotune
    b = B.Batch(small_specs(B, ne), seed=6, fault_rate=1e-3)
    ref = None
    for cfg in autotune.candidates():
        try:
            b.plan(cfg)
        except ne.NEError:
            continue
        b.run()
        torch.cuda.synchronize()
        snap = (b.out.clone(), b.flags.clone(), int(b.nflag.item()))
        if cfg.l_policy == ne.NE_L_BYTE:
            if ref is None:
                ref = snap
            assert torch.equal(snap[0], ref[0]) and torch.equal(snap[1], ref[1]) and snap[2] == ref[2]
        else:
            # another l changes the words, not the extracted outputs or the detected set
            assert torch.equal(snap[1], ref[1]) and snap[2] == ref[2]


def test_graph_replay_is_identical_and_refreshes_inputs(mods):
    B, ne = mods
    b = B.Batch(small_specs(B, ne), seed=8, fault_rate=1e-3)
    b.plan(B.default_config())
    b.run()
    torch.cuda.synchronize()
    out0, fl0 = b.out.clone(), b.flags.clone()
    b.out.fill_(0)
    b.capture()
    b.out.fill_(0)
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.out, out0) and torch.equal(b.flags, fl0)
    # new inputs in the same arenas: the replay computes the new batch
    b.c.neg_().clamp_(-128, 127)
    b.replay()
    torch.cuda.synchronize()
    for j in (0, 4):
        s = b.specs[j]
        c, op = b.job_inputs(j)
        direct = oracle.gemm_direct(c, op) if s.kind == ne.NE_JOB_GEMM else oracle.cconv_direct(c, op)
        pos_ok = B.expected_flags(b, j) == 0
        got = b.job_output(j).cpu().numpy().reshape(s.M, -1)
        assert (got[:, pos_ok] == direct.reshape(s.M, -1)[:, pos_ok]).all()


def test_out_of_range_inputs_are_reported(mods):
    B, ne = mods
    b = B.Batch(small_specs(B, ne)[:4], seed=9)
    b.plan(B.default_config())
    b.c[b.jobs[1].c_off + 5] = 300
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == ne.NE_ERANGE


def test_plan_rejects_bad_jobs(mods):
    B, ne = mods
    for bad in (B.JobSpec(ne.NE_JOB_GEMM, 3, rows=0, cols=12, k=16), B.JobSpec(ne.NE_JOB_GEMM, 3, rows=8, cols=16, k=131057),
                B.JobSpec(ne.NE_JOB_CCONV, 3, N=1), B.JobSpec(ne.NE_JOB_CCONV, 3, N=65537),
                B.JobSpec(ne.NE_JOB_CCONV, 6, N=64)):
        b = B.Batch([bad], generate=False)
        with pytest.raises(ne.NEError):
            b.plan(B.default_config())


def test_ragged_sizes_run_as_drawn(mods):
    """Products with k not a multiple of 16 and cols of any size (rows padded
    to 16 in the digit planes) and convolutions whose N is not a multiple of
    64 (on the exact transforms), against the oracle under faults."""
    B, ne = mods
    G, C, R = ne.NE_JOB_GEMM, ne.NE_JOB_CCONV, ne.NE_FUSE_RECOVER
    specs = [B.JobSpec(G, 3, rows=17, cols=13, k=37), B.JobSpec(G, 4, rows=40, cols=70, k=100),
             B.JobSpec(G, 5, rows=1, cols=1, k=1), B.JobSpec(G, 3, rows=33, cols=5, k=250, fuse=R, r=2),
             B.JobSpec(G, 4, rows=64, cols=64, k=48), B.JobSpec(C, 3, N=100), B.JobSpec(C, 4, N=1000),
             B.JobSpec(C, 5, N=3, fuse=R, r=1), B.JobSpec(C, 3, N=4099), B.JobSpec(C, 3, N=256)]
    specs += B.mixed_jobs(31, 24, mnk=(8, 300), conv=(2, 3000), recover_frac=0.2)
    assert any(s.kind == G and s.k % 16 for s in specs) and any(s.kind == C and s.N % 64 for s in specs)
    b = B.Batch(specs, seed=12, fault_rate=3e-3)
    b.plan(B.default_config())
    b.run()
    torch.cuda.synchronize()
    assert int(b.status.item()) == 0
    for j, s in enumerate(b.specs):
        dh, fl = oracle_job(b, j, ne)
        got = b.job_output(j).cpu().numpy().reshape(s.M, -1)
        assert (got == dh).all(), f"job {j} ({s})"
        if fl is not None:
            assert (unpack_flags(b.job_flags(j).cpu().numpy(), 1, s.positions_out)[0] == fl).all(), f"job {j}"


def test_staged_plan_uploads_the_same_tables(mods):
    B, ne = mods
    b = B.Batch(small_specs(B, ne) + [B.JobSpec(ne.NE_JOB_CCONV, 3, N=4160)], seed=10, fault_rate=1e-3)
    cfg = B.default_config(ntt_min_n=4096)
    b.plan(cfg)
    b.run()
    torch.cuda.synchronize()
    out0, fl0, nf0 = b.out.clone(), b.flags.clone(), int(b.nflag.item())
    info = ne.ne_batch_plan(b.jobs, cfg)
    on_transforms = sum(1 for s in b.specs if s.kind == ne.NE_JOB_CCONV and (s.N % 64 or s.N >= 4096))
    assert info.table_bytes > 0 and info.ntransform == on_transforms >= 2
    with pytest.raises(ne.NEError):
        ne.ne_batch_plan(b.jobs, cfg, b.ws_view, staging=torch.empty(info.table_bytes - 1, dtype=torch.uint8).pin_memory())
    with pytest.raises(ValueError):
        ne.ne_batch_plan(b.jobs, cfg, b.ws_view, staging=torch.empty(info.table_bytes, dtype=torch.uint8))
    # stale tables in the workspace and garbage in the staging buffer change nothing
    b.ws_view.fill_(0xA5)
    staging = torch.full((info.table_bytes + 64,), 0x5A, dtype=torch.uint8).pin_memory()
    b.info = ne.ne_batch_plan(b.jobs, cfg, b.ws_view, staging=staging)
    b.out.fill_(0)
    b.run()
    torch.cuda.synchronize()
    assert torch.equal(b.out, out0) and torch.equal(b.flags, fl0) and int(b.nflag.item()) == nf0
