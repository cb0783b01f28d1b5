"""GPU parity of the int8 tensor-path operations (digit planes on mma.sync)
against the CPU oracle, bit-exact, through the C ABI: the product and the
circular convolution of entangled streams, with and without the fused
extraction/check, and the fused fail-stop recovery."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ne():
    from paper_1604_04740_gb300 import ne as _ne
    return _ne


DEV = "cuda"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    return t.cpu().numpy()


def zeros(n, dtype=torch.int64):
    return torch.zeros(n, dtype=dtype, device=DEV)


# ---- circular convolution -------------------------------------------------------------

CCONV_CASES = [
    # batch, M, N, l, value range
    (4, 3, 1024, 16, (-128, 127)),      # two digits (byte-aligned l)
    (3, 3, 1024, 13, (-128, 127)),      # three digits (smallest l)
    (2, 4, 512, 16, (-128, 127)),
    (2, 5, 256, 8, (-128, 127)),
    (2, 3, 64, 16, (-128, 127)),        # one Toeplitz block
    (1, 3, 2048, 16, (-128, 127)),      # two CTAs, two u-chunks
    (1, 3, 1088, 16, (-128, 127)),      # 17 blocks: ragged last CTA and u-chunk
    (1, 4, 4096, 16, (-128, 127)),
    (2, 6, 256, 8, (-128, 127)),        # generic M
    (2, 3, 320, 14, (-1000, 1000)),     # wider inputs (|d| <= 320 * 1000 * 128 needs l = 14)
    # 9..16 blocks with M*S in {6, 8}: the hybrid tile (tensor pipe + dp4a pipe)
    (3, 3, 576, 16, (-128, 127)),       # one block on the tensor pipe, eight on dp4a
    (2, 3, 960, 16, (-128, 127)),
    (2, 4, 1024, 16, (-128, 127)),
    (1, 4, 704, 16, (-128, 127)),
]


@pytest.mark.parametrize("B,M,N,l,rng_", CCONV_CASES)
def test_cconv_digits_all_modes(ne, B, M, N, l, rng_):
    lo, hi = rng_
    c = inputs.int32_uniform(N + M, inputs.TAG_C, (B, M, N), lo, hi)
    g = inputs.operator_int8(N + M, (B, N))
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, lo, hi)
    status = zeros(1, torch.int32)
    planes = ne.ne_entangle_digits(p, dg, dev(c), status=status)
    assert int(status.item()) == 0
    gd = dev(g)
    direct = oracle.cconv_direct(c, g)
    eps = oracle.entangle(c, l)
    delta = oracle.cconv(eps, g)
    # NONE: the entangled outputs delta
    got = host(ne.ne_cconv_digits(p, dg, planes, gd, fuse=ne.NE_FUSE_NONE))
    assert (got == delta).all()
    # EXTRACT_CHECK for several r
    for r in sorted({0, 1, M - 1}):
        flags = zeros(B * (N // 32), torch.int32)
        nf = zeros(1)
        dh = host(ne.ne_cconv_digits(p, dg, planes, gd, flags=flags, nflag=nf, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=r))
        want_d, want_f = oracle.extract(delta, l, r)
        assert (dh == want_d).all() and (dh == direct).all()
        assert (unpack_flags(host(flags), B, N) == want_f).all() and int(nf.item()) == 0
    # RECOVER: the lost stream's digit planes are poisoned and must not matter
    for r_lost in sorted({0, M - 1}):
        pois = planes.clone()
        pois[:, r_lost] = 0x55
        dh = host(ne.ne_cconv_digits(p, dg, pois, gd, fuse=ne.NE_FUSE_RECOVER, r=r_lost))
        assert (dh == direct).all()


def test_cconv_digits_extreme_values(ne):
    # every input and kernel value at -128: the largest outputs (N 2^14)
    B, M, N, l = 1, 3, 1024, 16
    c = np.full((B, M, N), -128, np.int32)
    g = np.full((B, N), -128, np.int8)
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l)
    planes = ne.ne_entangle_digits(p, dg, dev(c))
    dh = host(ne.ne_cconv_digits(p, dg, planes, dev(g)))
    assert (dh == oracle.cconv_direct(c, g)).all() and dh.max() == N * 2 ** 14


def test_cconv_digits_rejects_bad_sizes(ne):
    p = ne.params(3, 16)
    dg = ne.ne_plan_digits(16)
    N = 65537                                   # beyond the int32 accumulation bound of the tiles
    planes = torch.zeros((1, 3, dg.S, N), dtype=torch.int8, device=DEV)
    g = torch.zeros((1, N), dtype=torch.int8, device=DEV)
    with pytest.raises(ne.NEError):
        ne.ne_cconv_digits(p, dg, planes, g)
    dg6 = ne.digits((0, 8, 16, 24, 32, 40))      # 3 x 6 = 18 digit planes, above the 16 a tile holds
    planes = torch.zeros((1, 3, 6, 128), dtype=torch.int8, device=DEV)
    with pytest.raises(ne.NEError):
        ne.ne_cconv_digits(p, dg6, planes, torch.zeros((1, 128), dtype=torch.int8, device=DEV))


# ---- matrix product ---------------------------------------------------------------------

GEMM_CASES = [
    # M, rows, cols, k, l, value range
    (4, 128, 128, 128, 16, (-128, 127)),
    (3, 64, 64, 64, 11, (-128, 127)),       # three digits, l from the K = 64 bound
    (3, 100, 72, 48, 16, (-128, 127)),      # ragged rows, cols not a multiple of 32
    (5, 64, 64, 256, 8, (-128, 127)),
    (4, 96, 96, 1024, 10, (-128, 127)),     # smallest l for K = 1024: three digits
    (3, 33, 40, 16, 16, (-128, 127)),
    (6, 32, 64, 64, 8, (-128, 127)),        # generic M
]


@pytest.mark.parametrize("M,rows,cols,k,l,rng_", GEMM_CASES)
def test_gemm_digits_all_modes(ne, M, rows, cols, k, l, rng_):
    lo, hi = rng_
    c = inputs.int32_uniform(rows + k, inputs.TAG_C, (M, rows, k), lo, hi)
    G = inputs.operator_int8(rows + k, (k, cols))
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, lo, hi)
    planes = ne.ne_entangle_digits(p, dg, dev(c.reshape(M, rows * k))).reshape(M, dg.S, rows, k)
    Gd = dev(G)
    direct = oracle.gemm_direct(c, G)
    eps = oracle.entangle(c.reshape(M, -1), l).reshape(M, rows, k)
    delta = np.stack([oracle.gemm(eps[m], G) for m in range(M)])
    got = host(ne.ne_gemm_digits(p, dg, planes, Gd, fuse=ne.NE_FUSE_NONE))
    assert (got == delta).all()
    nw = (rows * cols + 31) // 32
    for r in sorted({0, M - 1}):
        flags = torch.full((nw,), -1, dtype=torch.int32, device=DEV)
        nf = zeros(1)
        dh = host(ne.ne_gemm_digits(p, dg, planes, Gd, flags=flags, nflag=nf, r=r))
        assert (dh == direct).all()
        assert not host(flags).any() and int(nf.item()) == 0
    pois = planes.clone()
    pois[1] = -7
    dh = host(ne.ne_gemm_digits(p, dg, pois, Gd, fuse=ne.NE_FUSE_RECOVER, r=1))
    assert (dh == direct).all()


def test_gemm_digits_extreme_values(ne):
    M, n, k, l = 4, 64, 4096, 10
    c = np.full((M, n, k), -128, np.int32)
    G = np.full((k, n), -128, np.int8)
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l)
    planes = ne.ne_entangle_digits(p, dg, dev(c.reshape(M, -1))).reshape(M, dg.S, n, k)
    dh = host(ne.ne_gemm_digits(p, dg, planes, dev(G)))
    assert (dh == k * 2 ** 14).all()
