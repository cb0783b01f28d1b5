"""Host-side logic of the serving loop (no GPU): the per-request work
estimate that bounds a micro-batch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_work_estimate_follows_the_operation_counts():
    from paper_1604_04740_gb300 import batch as B
    from paper_1604_04740_gb300 import ne
    from paper_1604_04740_gb300 import serve as S
    G, C = ne.NE_JOB_GEMM, ne.NE_JOB_CCONV
    specs = [B.JobSpec(G, 3, rows=40, cols=72, k=48), B.JobSpec(C, 4, N=1024), B.JobSpec(C, 5, N=8192),
             B.JobSpec(C, 3, N=2048, plain=1)]
    T = S._Table(specs, [0] * 4, [0] * 4, ntt_min_n=4096)
    w = np.diff(T.cum_work)
    assert w[0] == 2 * 3 * 2 * 40 * 72 * 48                  # two digit planes per entangled stream
    assert w[1] == 2 * 4 * 2 * 1024 * 1024                   # convolution on tensor tiles
    assert w[2] == 280 * (2 * 5 + 1) * 8192 * 13             # on the transform path (N >= ntt_min_n)
    assert w[3] == 2 * 3 * 1 * 2048 * 2048                   # the plain form: one digit plane
    T0 = S._Table(specs, [0] * 4, [0] * 4, ntt_min_n=0)      # no transform path: all on tiles
    assert np.diff(T0.cum_work)[2] == 2 * 5 * 2 * 8192 * 8192
