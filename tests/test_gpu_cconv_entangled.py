"""GPU parity of the fused tensor-path convolution (raw streams in: Eq. 16 and
the digit split done while the tiles load) against the CPU oracle, bit-exact:
every tile shape (hybrid 16-block groups, single-chunk and multi-chunk
windows), every epilogue, the plain operation, the input-range status, and
equality with the two-launch path."""
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


@pytest.mark.parametrize("M,N,B", [(3, 1024, 9), (4, 1024, 5), (3, 64, 4), (3, 576, 3), (4, 2048, 2),
                                   (5, 1216, 2), (3, 4096, 1)])
def test_fused_cconv_matches_oracle(ne, M, N, B):
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(200 + M, (B, M, N))
    c[0, 0, :2] = -128
    c[-1, -1, -2:] = 127
    g = inputs.operator_int8(200 + N, (B, N))
    cd, gd = dev(c), dev(g)
    direct = oracle.cconv_direct(c, g)
    delta = oracle.cconv(oracle.entangle(c, l), g)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = host(ne.ne_cconv_entangled(p, dg, cd, gd, fuse=ne.NE_FUSE_NONE, status=status))
    assert (got == delta).all() and int(status.item()) == 0
    for r in sorted({0, M - 1}):
        flags = torch.full((ne.flag_words(B, N),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.full((1,), 3, dtype=torch.int64, device=DEV)
        got = host(ne.ne_cconv_entangled(p, dg, cd, gd, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, r))
        assert (got == direct).all()
        assert not unpack_flags(host(flags), B, N).any() and int(nflag.item()) == 0
        got = host(ne.ne_cconv_entangled(p, dg, cd, gd, fuse=ne.NE_FUSE_RECOVER, r=r))
        assert (got == direct).all()
    # the plain operation on the raw streams
    got = host(ne.ne_cconv_entangled(p, ne.raw_digits(), cd, gd, fuse=ne.NE_FUSE_NONE, plain=True))
    assert (got == direct).all()


def test_fused_equals_two_launch_path_and_reports_range(ne):
    B, M, N, l = 64, 3, 1024, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = dev(inputs.streams(210, (B, M, N)))
    g = dev(inputs.operator_int8(210, (B, N)))
    a = ne.ne_cconv_entangled(p, dg, c, g, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=2)
    b = ne.ne_cconv_digits(p, dg, ne.ne_entangle_digits(p, dg, c), g, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=2)
    assert torch.equal(a, b)
    c[5, 1, 100] = 200
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_cconv_entangled(p, dg, c, g, fuse=ne.NE_FUSE_NONE, status=status)
    assert int(status.item()) == ne.NE_ERANGE


def test_fused_rejects_a_digit_set_that_is_not_a_plan(ne):
    p = ne.params(3, 16)
    c = torch.zeros((1, 3, 1024), dtype=torch.int32, device=DEV)
    g = torch.zeros((1, 1024), dtype=torch.int8, device=DEV)
    with pytest.raises(ne.NEError):
        ne.ne_cconv_entangled(p, ne.digits((0, 16)), c, g)
