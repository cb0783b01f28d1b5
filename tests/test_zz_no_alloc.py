"""The batch entry point for callers that cannot allocate device memory.

Some callers cannot give the library a workspace: they run inside another
framework's memory pool or under a fixed device-memory budget, or in a loop
where a cudaMalloc (which synchronises the device) is not acceptable.
ne_batch_run_static serves them from a static scratch array that the library
owns.  This test calls it through the C ABI and checks that its outputs,
check bitmaps and flag counts are bit-identical to those of the workspace
entry point (ne_batch_plan + ne_batch_run) for two different batches run one
after the other (the second call reuses the array the first one left
behind), and that a batch too large for the array is refused.
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run_both(B, ne, specs, seed):
    b = B.Batch(specs, seed=seed, fault_rate=2e-3)
    cfg = B.default_config()
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


def test_static_scratch_refuses_a_batch_larger_than_the_array():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    big = [B.JobSpec(ne.NE_JOB_GEMM, 4, rows=2048, cols=64, k=4096)]   # 64 MiB of digit planes
    b = B.Batch(big, generate=False)
    with pytest.raises(ne.NEError) as e:
        ne.ne_batch_run_static(b.jobs, B.default_config(), b.c, b.ops, b.out, b.flags, b.nflag)
    assert e.value.status == ne.NE_ENOMEM
