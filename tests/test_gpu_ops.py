"""GPU parity of the operation in the form of the problem statement (ne_gemm,
ne_cconv: entangled int64 words in, Eq. 10 with the shared operator, the
extraction/check or recovery behind it) against the CPU oracle, bit-exact,
in both modes -- int64 multiply-adds on the CUDA cores, and int8 digit slices
split from the words inside the tensor kernels' loaders -- with every fuse
mode, several r, dropped planes, and seeded transient faults."""
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


def inject(delta, flat, strm, bit, skip=()):
    d = np.array(delta, dtype=np.int64, copy=True).view(np.uint64)
    n = d.shape[-1]
    keep = ~np.isin(strm, list(skip))
    np.bitwise_xor.at(d, (flat[keep] // n, strm[keep], flat[keep] % n), np.uint64(1) << bit[keep].astype(np.uint64))
    return d.view(np.int64)


def check_all_modes(ne, run, p, dg, delta, direct, nb, npos, seed):
    """run(mode, fuse, r, flags, nflag, faults, drop, status) -> out [nb, M, npos]."""
    M, l = p.M, p.l
    grp, pos, strm, bit = inputs.fault_list(seed, nb, npos, M, max(4, nb * npos // 25))
    flat = grp * npos + pos
    fl = (dev(flat.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))
    bad = inject(delta, flat, strm, bit)
    for mode in (ne.NE_MODE_I64, ne.NE_MODE_S8SLICE):
        status = torch.zeros(1, dtype=torch.int32, device=DEV)
        got = run(mode, ne.NE_FUSE_NONE, 0, None, None, fl, 0, status)
        assert (got == bad).all(), mode
        for r in sorted({0, M - 1}):
            flags = torch.full((nb * ((npos + 31) // 32),), -1, dtype=torch.int32, device=DEV)
            nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
            got = run(mode, ne.NE_FUSE_EXTRACT_CHECK, r, flags, nflag, fl, 0, status)
            want, wflags = oracle.extract(bad, l, r)
            assert (got == want).all(), (mode, r)
            gflags = unpack_flags(host(flags), nb, npos)
            assert (gflags == wflags).all() and int(nflag.item()) == len(flat)
            assert (gflags[grp, pos] == 1).all()
            ok = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
            assert (got[ok] == direct[ok]).all()
            # recovery: stream r dropped (its faults cannot land), with or without the mask
            for drop in (0, 1 << r):
                got = run(mode, ne.NE_FUSE_RECOVER, r, None, None, fl, drop, status)
                assert (got == oracle.recover(inject(delta, flat, strm, bit, skip=(r,)), l, r)).all(), (mode, r)
        assert int(status.item()) == 0


@pytest.mark.parametrize("M,rows,cols,k", [(3, 64, 64, 64), (4, 96, 128, 512), (3, 40, 72, 48), (5, 33, 40, 256)])
def test_gemm_forms_match_oracle(ne, M, rows, cols, k):
    l = oracle.choose_l(M, 64, k * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(600 + rows, (M, rows, k))
    G = inputs.operator_int8(600 + cols, (k, cols))
    eps = oracle.entangle(c.reshape(M, -1), l).reshape(M, rows, k)
    delta = np.stack([oracle.gemm(eps[m], G) for m in range(M)]).reshape(1, M, -1)
    direct = oracle.gemm_direct(c, G).reshape(1, M, -1)
    ed, Gd = dev(eps), dev(G)

    def run(mode, fuse, r, flags, nflag, fl, drop, status):
        out = ne.ne_gemm(p, ed, Gd, None, flags, nflag, mode, dg, fuse, r, drop, fl, status)
        return host(out).reshape(1, M, -1)

    check_all_modes(ne, run, p, dg, delta, direct, 1, rows * cols, 610 + k)


@pytest.mark.parametrize("B,M,N", [(5, 3, 1024), (3, 4, 1024), (2, 3, 2048), (3, 5, 256), (2, 3, 640)])
def test_cconv_forms_match_oracle(ne, B, M, N):
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(700 + N, (B, M, N))
    g = inputs.operator_int8(700 + N, (B, N))
    eps = oracle.entangle(c, l)
    delta = oracle.cconv(eps, g)
    direct = oracle.cconv_direct(c, g)
    ed, gd = dev(eps), dev(g)

    def run(mode, fuse, r, flags, nflag, fl, drop, status):
        return host(ne.ne_cconv(p, ed, gd, None, flags, nflag, mode, dg, fuse, r, drop, fl, status))

    check_all_modes(ne, run, p, dg, delta, direct, B, N, 710 + N)


def test_drop_mask_leaves_planes_unwritten_and_slices_report_words_outside_the_plan(ne):
    M, N, l = 3, 1024, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(720, (2, M, N))
    g = dev(inputs.operator_int8(720, (2, N)))
    eps = oracle.entangle(c, l)
    out = torch.full((2, M, N), 5, dtype=torch.int64, device=DEV)
    ne.ne_cconv(ne.planes_of(M), dev(eps), g, out, fuse=ne.NE_FUSE_NONE, drop_mask=0b101)
    o = host(out)
    assert (o[:, 0] == 5).all() and (o[:, 2] == 5).all()
    assert (o[:, 1] == oracle.cconv(eps, host(g))[:, 1]).all()
    # a word with a digit the plan lacks (byte 1 non-zero) is reported
    bad = eps.copy()
    bad[1, 2, 17] += 1 << 9
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_cconv(p, dev(bad), g, mode=ne.NE_MODE_S8SLICE, dg=dg, status=status)
    assert int(status.item()) == ne.NE_ERANGE
    # invalid combinations are refused before any launch
    for kw in ({"fuse": ne.NE_FUSE_EXTRACT_CHECK, "drop_mask": 1}, {"fuse": ne.NE_FUSE_RECOVER, "r": 0, "drop_mask": 2},
               {"mode": 7}, {"mode": ne.NE_MODE_S8SLICE, "dg": dg, "fuse": ne.NE_FUSE_NONE, "drop_mask": 1}):
        with pytest.raises(ne.NEError):
            ne.ne_cconv(p, dev(eps), g, **kw)
