"""The batch entry point for callers that cannot allocate device memory.

Some callers cannot give the library a workspace: they run inside another
framework's memory pool or under a fixed device-memory budget, or in a loop
where a cudaMalloc (which synchronises the device) is not acceptable.
ne_batch_run_static serves them from a static scratch array that the library
owns.  This test calls it through the C ABI and checks that its outputs,
check bitmaps and flag counts are bit-identical to those of the workspace
entry point (ne_batch_plan + ne_batch_run) for batches run one after the
other (each call reuses the array the previous one left behind) -- tensor
tiles only, then long convolutions on the exact transforms (whose job table
and scratch then sit in the array too) with jobs that lost a stream and are
recovered in the epilogue -- and that a batch too large for the array is
refused.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_both(B, ne, specs, seed, cfg=None):
    b = B.Batch(specs, seed=seed, fault_rate=2e-3)
    cfg = cfg or B.default_config()
    b.plan(cfg)
    b.run()
    torch.cuda.synchronize()
    ref = (b.out.clone(), b.flags.clone(), int(b.nflag.item()))
    out = torch.full_like(b.out, -1)
    flags = torch.full_like(b.flags, -1)
    nflag = torch.full_like(b.nflag, -1)
    status = torch.zeros(1, dtype=torch.int32, device=b.out.device)
    ne.ne_batch_run_static(b.jobs, cfg, b.c, b.ops, out, flags, nflag, *b.fault_dev, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(out, ref[0]), "outputs differ from the workspace entry point"
    assert torch.equal(flags, ref[1]), "check bitmaps differ from the workspace entry point"
    assert int(nflag.item()) == ref[2] and ref[2] > 0


def test_static_scratch_batch_matches_workspace_batch_on_two_calls():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    _run_both(B, ne, B.mixed_jobs(11, 12, mnk=(16, 128), conv=(64, 1024)), seed=1)
    _run_both(B, ne, B.mixed_jobs(12, 10, mnk=(16, 160), conv=(64, 2048)), seed=2)


def test_static_scratch_holds_transform_jobs_and_recovery():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    cfg = B.default_config(ntt_min_n=1024)
    specs = B.mixed_jobs(13, 16, mnk=(16, 128), conv=(1024, 6000), recover_frac=0.3)
    assert any(s.fuse == ne.NE_FUSE_RECOVER for s in specs)
    _run_both(B, ne, specs, seed=3, cfg=cfg)
    _run_both(B, ne, B.mixed_jobs(14, 12, mnk=(16, 96), conv=(2048, 9000), recover_frac=0.3), seed=4, cfg=cfg)


def test_static_scratch_refuses_a_batch_larger_than_the_array():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    big = [B.JobSpec(ne.NE_JOB_GEMM, 4, rows=2048, cols=64, k=4096)]   # 64 MiB of digit planes
    b = B.Batch(big, generate=False)
    with pytest.raises(ne.NEError) as e:
        ne.ne_batch_run_static(b.jobs, B.default_config(), b.c, b.ops, b.out, b.flags, b.nflag)
    assert e.value.status == ne.NE_ENOMEM
