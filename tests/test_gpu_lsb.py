"""GPU parity of the remaining LSB operators of Eq. 2 (element-wise +, -, x,
outer and inner products, permutation, circular cross-correlation) against
the CPU oracle, bit-exact, through the C ABI: the operator alone, with the
fused extract/check (clean and with a corrupted stream) and with the fused
recovery of a lost stream."""
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


def bound(op, n):
    return {"add": 255, "sub": 255, "mul": 2 ** 14, "outer": 2 ** 14, "inner": n * 2 ** 14,
            "permute": 128}[op]


def operand(op, B, n, k, seed, shared=False):
    rng = np.random.default_rng(seed)
    if op == "permute":
        return rng.permutation(n)
    rows = 1 if shared else B
    width = k if op == "outer" else n
    g = rng.integers(-128, 128, (rows, width), dtype=np.int64)
    g[g == 0] = 1          # a corrupted input word must change the result it meets
    return g


def run_gpu(ne, op, p, eps, g, fuse, r, flags=None, nflag=None):
    e = dev(eps)
    if op in ("add", "sub", "mul"):
        code = {"add": ne.NE_OP_ADD, "sub": ne.NE_OP_SUB, "mul": ne.NE_OP_MUL}[op]
        gd = dev(g)
        if op in ("add", "sub"):
            gd = ne.ne_entangle_kernel_self(p.l, gd)
        return ne.ne_elementwise(p, code, e, gd.reshape(-1) if g.shape[0] == 1 else gd, None, flags, nflag, fuse, r)
    if op == "outer":
        return ne.ne_outer(p, e, dev(g).reshape(-1) if g.shape[0] == 1 else dev(g), None, flags, nflag, fuse, r)
    if op == "inner":
        return ne.ne_inner(p, e, dev(g).reshape(-1) if g.shape[0] == 1 else dev(g), None, flags, nflag, fuse, r)
    return ne.ne_permute(p, e, dev(g.astype(np.int32)), None, flags, nflag, fuse, r)


def oracle_delta(op, eps, g, l):
    B = eps.shape[0]
    gg = g
    if op in ("add", "sub", "mul", "outer", "inner"):
        gg = np.ascontiguousarray(np.broadcast_to(g, (B, g.shape[1])))
    if op in ("add", "sub"):
        gg = oracle.entangle_kernel_self(gg, l)
    return oracle.lsb_apply(op, eps, gg)


OPS = ("add", "sub", "mul", "outer", "inner", "permute")


@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("M", [3, 4, 5, 6])
@pytest.mark.parametrize("n,shared", [(1000, False), (999, False), (64, True)])
@pytest.mark.parametrize("lchoice", ["smallest", "16"])
def test_lsb_operator_matches_oracle(ne, op, M, n, shared, lchoice):
    # l = 16 (valid for M <= 4) takes the kernels compiled for that l
    B, k = 3, (10 if n % 2 == 0 else 7)
    if lchoice == "16" and (M - 1) * 16 >= 64:
        pytest.skip("l = 16 needs (M - 1) l < 64")
    l = oracle.choose_l(M, 64, bound(op, n), oracle.POLICY_SMALLEST)[0] if lchoice == "smallest" else 16
    p = ne.params(M, l)
    c = inputs.streams(5 + M, (B, M, n))
    g = operand(op, B, n, k, 11 * M + n, shared)
    eps = oracle.entangle(c, l)
    direct = oracle.lsb_direct(op, c, np.broadcast_to(g, (B, g.shape[1])) if g.ndim == 2 else g)
    delta = oracle_delta(op, eps, g, l)
    P = delta.reshape(B, M, -1).shape[-1]
    # the operator alone: the entangled words
    got = host(run_gpu(ne, op, p, eps, g, ne.NE_FUSE_NONE, 0))
    assert (got == delta).all()
    for r in (0, M - 1):
        # fused extract/check on clean data
        flags = torch.full((ne.flag_words(B, P),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.full((1,), 7, dtype=torch.int64, device=DEV)
        got = host(run_gpu(ne, op, p, eps, g, ne.NE_FUSE_EXTRACT_CHECK, r, flags, nflag))
        assert (got == direct).all()
        assert not unpack_flags(host(flags), B, P).any() and int(nflag.item()) == 0
        # one corrupted word of stream (r + 1) mod M: flags and outputs as the oracle's
        bad = eps.copy()
        bad[1, (r + 1) % M, n // 3] ^= np.int64(1) << np.int64(20 + r)
        want_d, want_f = oracle.extract(oracle_delta(op, bad, g, l).reshape(B, M, -1), l, r)
        got = host(run_gpu(ne, op, p, bad, g, ne.NE_FUSE_EXTRACT_CHECK, r, flags, nflag))
        gf = unpack_flags(host(flags), B, P)
        assert (got.reshape(B, M, -1) == want_d).all()
        assert (gf == want_f).all() and gf.any() and int(nflag.item()) == int(want_f.sum())
        # fused recovery: stream r holds garbage and is never read
        lost = eps.copy()
        lost[:, r, :] = np.int64(0x5A5A5A5A5A5A5A5A)
        got = host(run_gpu(ne, op, p, lost, g, ne.NE_FUSE_RECOVER, r))
        assert (got == direct).all()


@pytest.mark.parametrize("B,n", [(2, 50000), (1, 4097), (64, 300), (3, 1)])
def test_inner_split_and_single_block_paths(ne, B, n):
    M = 3
    l = oracle.choose_l(M, 64, n * 2 ** 14, oracle.POLICY_SMALLEST)[0]
    p = ne.params(M, l)
    c = inputs.streams(21, (B, M, n))
    g = operand("inner", B, n, 0, 22)
    eps = oracle.entangle(c, l)
    direct = oracle.inner(c.astype(np.int64), g)
    assert (host(ne.ne_inner(p, dev(eps), dev(g), fuse=ne.NE_FUSE_NONE)) == oracle.inner(eps, g)).all()
    flags = torch.zeros(ne.flag_words(B, 1), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    assert (host(ne.ne_inner(p, dev(eps), dev(g), None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 2)) == direct).all()
    assert int(nflag.item()) == 0
    bad = eps.copy()
    bad[B - 1, 0, n - 1] += 1
    got = host(ne.ne_inner(p, dev(bad), dev(g), None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 2))
    want_d, want_f = oracle.extract(oracle.inner(bad, g)[:, :, None], l, 2)
    assert (got == want_d[..., 0]).all()
    assert (unpack_flags(host(flags), B, 1) == want_f).all() and int(nflag.item()) == int(want_f.sum())
    lost = eps.copy()
    lost[:, 1] = 12345
    assert (host(ne.ne_inner(p, dev(lost), dev(g), fuse=ne.NE_FUSE_RECOVER, r=1)) == direct).all()


def test_entangled_pipeline_on_the_gpu_end_to_end(ne):
    # GPU entangle -> element-wise x on the GPU -> fused extract; and the + form
    # with the self-entangled kernel produced on the GPU
    B, M, n = 4, 3, 4096
    l = 16
    p = ne.params(M, l)
    c = inputs.streams(31, (B, M, n))
    g = operand("mul", B, n, 0, 32)
    eps = ne.ne_entangle(p, dev(c))
    got = host(ne.ne_elementwise(p, ne.NE_OP_MUL, eps, dev(g), fuse=ne.NE_FUSE_EXTRACT_CHECK, r=1))
    assert (got == c.astype(np.int64) * g[:, None, :]).all()
    ge = ne.ne_entangle_kernel_self(l, dev(g))
    assert (host(ge) == oracle.entangle_kernel_self(g, l)).all()
    got = host(ne.ne_elementwise(p, ne.NE_OP_ADD, eps, ge, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=0))
    assert (got == c.astype(np.int64) + g[:, None, :]).all()


def test_permute_index_outside_range_is_reported_not_followed(ne):
    B, M, n = 2, 3, 64
    p = ne.params(M, 16)
    eps = oracle.entangle(inputs.streams(41, (B, M, n)), 16)
    perm = np.arange(n, dtype=np.int32)[::-1].copy()
    perm[5] = n + 1000
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = host(ne.ne_permute(p, dev(eps), dev(perm), fuse=ne.NE_FUSE_NONE, status=status))
    assert int(status.item()) == ne.NE_EINVAL
    ok = np.arange(n) != 5
    assert (out[..., ok] == eps[..., perm[ok]]).all()
    assert (out[..., 5] == eps[..., 0]).all()


@pytest.mark.parametrize("M,N", [(3, 1024), (4, 256), (3, 192)])
def test_cross_correlation_through_the_reversed_operand(ne, M, N):
    B = 5
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    c = inputs.streams(51, (B, M, N))
    g = inputs.operator_int8(51, (B, N))
    direct = oracle.cxcorr(c.astype(np.int64), g)
    grev = ne.ne_reverse_operand(dev(g))
    assert (host(grev) == g[:, (-np.arange(N)) % N]).all()
    # int8 tensor path with the fused extract/check
    dg = ne.ne_plan_digits(l, -128, 127)
    planes = ne.ne_entangle_digits(p, dg, dev(c))
    flags = torch.zeros(ne.flag_words(B, N), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    got = host(ne.ne_cconv_digits(p, dg, planes, grev, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 0))
    assert (got == direct).all() and int(nflag.item()) == 0
    # int64 CUDA-core form on the entangled words, then extract
    eps = ne.ne_entangle(p, dev(c))
    delta = ne.ne_cconv(p, eps, grev, fuse=ne.NE_FUSE_NONE)
    assert (host(delta) == oracle.cxcorr(oracle.entangle(c, l), g)).all()
    assert (host(ne.ne_extract(p, delta, r=2)) == direct).all()
