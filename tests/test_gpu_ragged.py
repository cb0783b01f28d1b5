"""GPU parity of the stand-alone tensor-path operations at ragged sizes
against the CPU oracle, bit-exact, under seeded faults: circular convolutions
whose N is not a multiple of 64 (the block-Toeplitz tile over signed block
offsets, from raw streams, digit planes or entangled words, and groups that do
not start 16-byte aligned) and products whose k is not a multiple of 16 or
whose cols are not a multiple of 4 (element-wise loads), every epilogue."""
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


def inject(delta, flat, strm, bit, skip=None):
    d = np.array(delta, dtype=np.int64, copy=True).view(np.uint64)
    n = d.shape[-1]
    keep = np.ones(len(flat), bool) if skip is None else strm != skip
    np.bitwise_xor.at(d, (flat[keep] // n, strm[keep], flat[keep] % n), np.uint64(1) << bit[keep].astype(np.uint64))
    return d.view(np.int64)


def all_modes(ne, run, M, l, delta, direct, B, n, seed):
    grp, pos, strm, bit = inputs.fault_list(seed, B, n, M, max(2, B * n // 30))
    flat = grp * n + pos
    fl = (dev(flat.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))
    bad = inject(delta, flat, strm, bit)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert (run(ne.NE_FUSE_NONE, 0, None, None, fl, status) == bad).all()
    for r in sorted({0, M - 1}):
        flags = torch.full((B * ((n + 31) // 32),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
        got = run(ne.NE_FUSE_EXTRACT_CHECK, r, flags, nflag, fl, status)
        want, wflags = oracle.extract(bad, l, r)
        assert (got == want).all(), r
        gflags = unpack_flags(host(flags), B, n)
        assert (gflags == wflags).all() and int(nflag.item()) == len(flat)
        ok = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
        assert (got[ok] == direct[ok]).all()
        got = run(ne.NE_FUSE_RECOVER, r, None, None, fl, status)
        assert (got == oracle.recover(inject(delta, flat, strm, bit, skip=r), l, r)).all(), r
    assert int(status.item()) == 0


@pytest.mark.parametrize("form", ["entangled", "digits", "words"])
@pytest.mark.parametrize("B,M,N", [(3, 3, 100), (2, 4, 1000), (2, 3, 1095), (1, 5, 4095), (4, 3, 5), (2, 3, 1),
                                   (2, 4, 70)])
def test_ragged_circular_convolution(ne, form, B, M, N):
    l = oracle.choose_l(M, 64, max(N, 2) * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    seed = 2000 + 7 * N + M
    c = inputs.streams(seed, (B, M, N))
    g = inputs.operator_int8(seed, (B, N))
    direct = oracle.cconv_direct(c, g)
    eps = oracle.entangle(c, l)
    delta = oracle.cconv(eps, g)
    cd, gd, ed = dev(c), dev(g), dev(eps)
    planes = ne.ne_entangle_digits(p, dg, cd)

    def run(fuse, r, flags, nflag, fl, status):
        if form == "entangled":
            out = ne.ne_cconv_entangled(p, dg, cd, gd, None, flags, nflag, fuse, r, status=status, faults=fl)
        elif form == "digits":
            out = ne.ne_cconv_digits(p, dg, planes, gd, None, flags, nflag, fuse, r, faults=fl)
        else:
            out = ne.ne_cconv(p, ed, gd, None, flags, nflag, ne.NE_MODE_S8SLICE, dg, fuse, r, 0, fl, status)
        return host(out)

    all_modes(ne, run, M, l, delta, direct, B, N, seed)
    if form == "entangled":
        got = host(ne.ne_cconv_entangled(p, ne.raw_digits(), cd, gd, fuse=ne.NE_FUSE_NONE, plain=True))
        assert (got == direct).all()


@pytest.mark.parametrize("form", ["digits", "words"])
@pytest.mark.parametrize("M,rows,cols,k", [(3, 17, 13, 37), (4, 40, 70, 100), (5, 1, 1, 1), (3, 33, 5, 250),
                                           (4, 65, 66, 16), (3, 20, 100, 3)])
def test_ragged_product(ne, form, M, rows, cols, k):
    l = oracle.choose_l(M, 64, k * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    seed = 3000 + rows + cols + k
    c = inputs.streams(seed, (M, rows, k))
    G = inputs.operator_int8(seed, (k, cols))
    direct = oracle.gemm_direct(c, G).reshape(1, M, -1)
    eps = oracle.entangle(c.reshape(M, -1), l).reshape(M, rows, k)
    delta = np.stack([oracle.gemm(eps[m], G) for m in range(M)]).reshape(1, M, -1)
    planes = ne.ne_entangle_digits(p, dg, dev(c).reshape(M, rows * k)).reshape(M, dg.S, rows, k)
    ed, Gd = dev(eps), dev(G)

    def run(fuse, r, flags, nflag, fl, status):
        if form == "digits":
            out = ne.ne_gemm_digits(p, dg, planes, Gd, None, flags, nflag, fuse, r, faults=fl)
        else:
            out = ne.ne_gemm(p, ed, Gd, None, flags, nflag, ne.NE_MODE_S8SLICE, dg, fuse, r, 0, fl, status)
        return host(out).reshape(1, M, -1)

    all_modes(ne, run, M, l, delta, direct, 1, rows * cols, seed)


def test_misaligned_groups_take_the_element_path(ne):
    # streams whose groups start at odd int32 offsets (a view into a larger buffer)
    B, M, N, l = 3, 3, 1024, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(77, (B, M, N))
    g = inputs.operator_int8(77, (B, N))
    buf = torch.zeros(B * M * N + 1, dtype=torch.int32, device=DEV)
    buf[1:] = dev(c).reshape(-1)
    cv = buf[1:].view(B, M, N)
    got = host(ne.ne_cconv_entangled(p, dg, cv, dev(g)))
    assert (got == oracle.cconv_direct(c, g)).all()
