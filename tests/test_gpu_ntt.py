"""GPU parity of the number-theoretic-transform convolution (raw streams in,
extracted outputs out, one launch) against the CPU oracle, bit-exact, through
the C ABI: the entangled words, the fused extract/check, the fused recovery,
the plain operation, the check on injected faults and the digit-plan range
status."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"
N = 1024


@pytest.fixture(scope="module")
def ne():
    from paper_1604_04740_gb300 import ne as _ne
    return _ne


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("M,policy", [(3, oracle.POLICY_BYTE), (3, oracle.POLICY_SMALLEST), (4, oracle.POLICY_BYTE),
                                      (5, oracle.POLICY_SMALLEST), (6, oracle.POLICY_SMALLEST)])
@pytest.mark.parametrize("B", [1, 5, 700])   # 700 > resident CTAs: the persistent loop
def test_ntt_cconv_matches_oracle(ne, M, policy, B):
    l = oracle.choose_l(M, 64, N * 2 ** 14, policy)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    if M * dg.S > 15:
        pytest.skip("more digit planes than the kernel's 15 warps")
    c = inputs.streams(60 + M, (B, M, N))
    c[0, 0, :3] = -128           # the extremes of the range
    c[-1, -1, -3:] = 127
    g = inputs.operator_int8(60 + M, (B, N))
    g[0, :2] = -128
    cd, gd = dev(c), dev(g)
    direct = oracle.cconv_direct(c, g)
    delta = oracle.cconv(oracle.entangle(c, l), g)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = host(ne.ne_cconv_ntt(p, dg, cd, gd, fuse=ne.NE_FUSE_NONE, status=status))
    assert (got == delta).all() and int(status.item()) == 0
    for r in sorted({0, M - 1}):
        flags = torch.full((ne.flag_words(B, N),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.full((1,), 5, dtype=torch.int64, device=DEV)
        got = host(ne.ne_cconv_ntt(p, dg, cd, gd, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, r))
        assert (got == direct).all()
        assert not unpack_flags(host(flags), B, N).any() and int(nflag.item()) == 0
        got = host(ne.ne_cconv_ntt(p, dg, cd, gd, fuse=ne.NE_FUSE_RECOVER, r=r))
        assert (got == direct).all()


def test_ntt_plain_operation_and_overflow_free_extremes(ne):
    B, M = 3, 3
    p = ne.params(M, 16)
    c = np.full((B, M, N), -128, np.int32)
    g = np.full((B, N), -128, np.int8)
    c[1] = inputs.streams(70, (M, N))
    want = oracle.cconv_direct(c, g)
    got = host(ne.ne_cconv_ntt(p, ne.digits((0,)), dev(c), dev(g),
                               fuse=ne.NE_FUSE_NONE, plain=True))
    assert (got == want).all()
    # every output at the bound N * 2^14 for the all -128 groups
    assert (got[0] == N * 2 ** 14).all()


def test_ntt_flags_exactly_the_injected_faults(ne):
    B, M, l = 64, 3, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(80, (B, M, N))
    g = inputs.operator_int8(80, (B, N))
    delta = ne.ne_cconv_ntt(p, dg, dev(c), dev(g), fuse=ne.NE_FUSE_NONE)
    rng = np.random.default_rng(81)
    cnt = 200
    flat = rng.choice(B * N, cnt, replace=False)
    grp, pos = flat // N, flat % N
    strm = rng.integers(0, M, cnt)
    bit = rng.integers(0, 64, cnt)
    ne.ne_inject(delta, M, dev(grp.astype(np.int64)), dev(pos.astype(np.int64)), dev(strm.astype(np.int64)),
                 dev(bit.astype(np.int64)))
    flags = torch.zeros(ne.flag_words(B, N), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    ne.ne_extract(p, delta, None, 0, flags, nflag)
    want = np.zeros((B, N), np.uint8)
    want[grp, pos] = 1
    assert (unpack_flags(host(flags), B, N) == want).all() and int(nflag.item()) == cnt


def test_ntt_word_outside_the_digit_plan_sets_erange(ne):
    B, M, l = 2, 3, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(90, (B, M, N))
    c[1, 2, 77] = 300            # outside [-128, 127]: its words need a digit the plan lacks
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_cconv_ntt(p, dg, dev(c), dev(inputs.operator_int8(90, (B, N))), fuse=ne.NE_FUSE_NONE, status=status)
    assert int(status.item()) == ne.NE_ERANGE


def test_ntt_matches_the_tensor_path(ne):
    B, M, l = 40, 4, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = dev(inputs.streams(95, (B, M, N)))
    g = dev(inputs.operator_int8(95, (B, N)))
    a = ne.ne_cconv_ntt(p, dg, c, g, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=1)
    b = ne.ne_cconv_digits(p, dg, ne.ne_entangle_digits(p, dg, c), g, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=1)
    assert torch.equal(a, b)
