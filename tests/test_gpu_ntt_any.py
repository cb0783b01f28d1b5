"""GPU parity of the general-length transform convolution (two primes, Chinese
remainder reconstruction, any N up to 65536) against the CPU oracle,
bit-exact: full outputs where the oracle finishes in seconds, sampled
outputs (computed one by one by the oracle) at the longest lengths, every
epilogue, the plain operation, and the range checks."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"


@pytest.fixture(scope="module")
def ne():
    from paper_1604_04740_gb300 import ne as _ne
    return _ne


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.cpu().numpy()


# powers of two (cyclic transforms) and other lengths (linear, folded), with
# and without passes outside shared memory (transform lengths above 2^14)
@pytest.mark.parametrize("M,N,B", [(3, 2, 3), (3, 3, 2), (4, 64, 5), (3, 100, 4), (5, 1000, 2), (3, 1024, 3),
                                   (4, 4096, 2), (3, 5000, 2), (3, 8192, 1), (4, 9000, 1),
                                   (8, 3000, 2), (6, 20000, 1)])
def test_ntt_any_matches_oracle(ne, M, N, B):
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    c = inputs.streams(300 + N, (B, M, N))
    c[0, 0, 0] = -128
    c[-1, -1, -1] = 127
    g = inputs.operator_int8(300 + N, (B, N))
    cd, gd = dev(c), dev(g)
    direct = oracle.cconv_direct(c, g)
    delta = oracle.cconv(oracle.entangle(c, l), g)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = host(ne.ne_cconv_ntt_any(p, cd, gd, fuse=ne.NE_FUSE_NONE, status=status))
    assert (got == delta).all() and int(status.item()) == 0
    for r in sorted({0, M - 1}):
        flags = torch.full((ne.flag_words(B, N),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.full((1,), 4, dtype=torch.int64, device=DEV)
        got = host(ne.ne_cconv_ntt_any(p, cd, gd, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, r))
        assert (got == direct).all()
        assert not unpack_flags(host(flags), B, N).any() and int(nflag.item()) == 0
        got = host(ne.ne_cconv_ntt_any(p, cd, gd, fuse=ne.NE_FUSE_RECOVER, r=r))
        assert (got == direct).all()
    got = host(ne.ne_cconv_ntt_any(p, cd, gd, fuse=ne.NE_FUSE_NONE, plain=True))
    assert (got == direct).all()


@pytest.mark.parametrize("N", [16384, 16385, 40000, 65536])
def test_ntt_any_longest_lengths_on_sampled_outputs(ne, N):
    # transform lengths 2^14 (all in shared memory) to 2^17 (three passes over
    # the workspace); the oracle computes 64 sampled outputs one by one
    B, M = 1, 3
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    c = inputs.streams(400 + N, (B, M, N))
    g = inputs.operator_int8(400 + N, (B, N))
    cd, gd = dev(c), dev(g)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    got = host(ne.ne_cconv_ntt_any(p, cd, gd, None, None, nflag, ne.NE_FUSE_EXTRACT_CHECK, 1))
    assert int(nflag.item()) == 0
    rng = np.random.default_rng(N)
    sig = rng.integers(0, M, 64)
    pos = np.concatenate([[0, N - 1], rng.integers(0, N, 62)])
    want = oracle.cconv_at(c.astype(np.int64), g, sig, pos)
    assert (got.reshape(M, N)[sig, pos] == want).all()
    # the entangled words, sampled the same way, and a second path for every output
    delta = host(ne.ne_cconv_ntt_any(p, cd, gd, fuse=ne.NE_FUSE_NONE))
    eps = oracle.entangle(c, l)
    assert (delta.reshape(M, N)[sig, pos] == oracle.cconv_at(eps, g, sig, pos)).all()
    plain = host(ne.ne_cconv_ntt_any(p, cd, gd, fuse=ne.NE_FUSE_NONE, plain=True))
    assert (plain == got).all()
    if N % 64 == 0:
        dg = ne.ne_plan_digits(l, -128, 127)
        tensor = host(ne.ne_cconv_entangled(p, dg, cd, gd, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=1))
        assert (tensor == got).all()


def test_ntt_any_flags_injected_faults_and_reports_ranges(ne):
    B, M, N, l = 6, 3, 3000, 16
    p = ne.params(M, l)
    c = inputs.streams(500, (B, M, N))
    g = inputs.operator_int8(500, (B, N))
    delta = ne.ne_cconv_ntt_any(p, dev(c), dev(g), fuse=ne.NE_FUSE_NONE)
    rng = np.random.default_rng(501)
    cnt = 40
    flat = rng.choice(B * N, cnt, replace=False)
    grp, pos = flat // N, flat % N
    lists = [dev(v.astype(np.int64)) for v in (grp, pos, rng.integers(0, M, cnt), rng.integers(0, 64, cnt))]
    ne.ne_inject(delta, M, *lists)
    flags = torch.zeros(ne.flag_words(B, N), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    ne.ne_extract(p, delta, None, 0, flags, nflag)
    want = np.zeros((B, N), np.uint8)
    want[grp, pos] = 1
    assert (unpack_flags(host(flags), B, N) == want).all() and int(nflag.item()) == cnt
    # an input outside the declared range is reported on the device
    c2 = c.copy()
    c2[2, 1, 17] = 1000
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_cconv_ntt_any(p, dev(c2), dev(g), fuse=ne.NE_FUSE_NONE, status=status)
    assert int(status.item()) == ne.NE_ERANGE
    # a range whose outputs could leave the two-prime range is refused on the host
    with pytest.raises(ne.NEError):
        ne.ne_cconv_ntt_any(ne.params(3, 20), dev(c), dev(g), cmin=-(2 ** 20), cmax=2 ** 20)
