"""GPU parity of the long-stream linear convolution (ne_lconv: the full linear
convolution of every entangled stream with a short kernel, fused from the raw
streams to the extracted outputs) against the CPU oracle, bit-exact: ragged
lengths, kernels shorter and longer than a tile, K = 1, M up to 8, every
epilogue, seeded transient faults, the plain operation, and at the size of
the paper's second experiment (10^6 samples, kernels of 100 and 4500 taps)
on every fault plus a sample of the other outputs."""
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


def plan(ne, M, K):
    l = oracle.choose_l(M, 64, K * 2 ** 14, oracle.POLICY_BYTE)[0]
    return l, ne.params(M, l), ne.ne_plan_digits(l, -128, 127)


CASES = [
    # B, M, n, K
    (2, 3, 1000, 100),
    (1, 3, 3000, 4500),     # kernel longer than the stream, five chunks of shifts
    (3, 4, 777, 129),
    (1, 8, 2000, 64),       # eight streams, l = 8: 16 digit planes (the generic-M tile)
    (2, 5, 333, 1),         # K = 1: a scaled copy
    (1, 3, 5, 70),          # a stream shorter than one block
    (2, 3, 1024, 64),       # block-aligned lengths
    (1, 4, 2049, 1500),
]


@pytest.mark.parametrize("B,M,n,K", CASES)
def test_lconv_matches_oracle(ne, B, M, n, K):
    l, p, dg = plan(ne, M, K)
    seed = 1000 + n + K
    c = inputs.streams(seed, (B, M, n))
    c[0, 0, :2] = -128
    c[-1, -1, -2:] = 127
    g = inputs.operator_int8(seed, (B, K))
    g[0, 0] = -128
    no = n + K - 1
    direct = oracle.lconv_direct(c, g)
    delta = oracle.lconv(oracle.entangle(c, l), g)
    grp, pos, strm, bit = inputs.fault_list(seed, B, no, M, max(3, B * no // 40))
    flat = grp * no + pos
    fl = (dev(flat.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))
    bad = inject(delta, flat, strm, bit)
    cd, gd = dev(c), dev(g)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = host(ne.ne_lconv(p, dg, cd, gd, fuse=ne.NE_FUSE_NONE, status=status, faults=fl))
    assert (got == bad).all()
    for r in sorted({0, M - 1}):
        flags = torch.full((B * ((no + 31) // 32),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
        got = host(ne.ne_lconv(p, dg, cd, gd, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, r, status=status,
                               faults=fl))
        want, wflags = oracle.extract(bad, l, r)
        assert (got == want).all(), r
        gflags = unpack_flags(host(flags), B, no)
        assert (gflags == wflags).all() and int(nflag.item()) == len(flat)
        assert (gflags[grp, pos] == 1).all()
        ok = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
        assert (got[ok] == direct[ok]).all()
        got = host(ne.ne_lconv(p, dg, cd, gd, fuse=ne.NE_FUSE_RECOVER, r=r, status=status, faults=fl))
        assert (got == oracle.recover(inject(delta, flat, strm, bit, skip=r), l, r)).all()
    assert int(status.item()) == 0
    # the plain operation: one digit, and the entangled digit set
    assert (host(ne.ne_lconv(p, ne.raw_digits(), cd, gd, fuse=ne.NE_FUSE_NONE, plain=True)) == direct).all()
    assert (host(ne.ne_lconv(p, dg, cd, gd, fuse=ne.NE_FUSE_NONE, plain=True)) == direct).all()


@pytest.mark.parametrize("M,K", [(3, 4500), (8, 100)])
def test_lconv_at_the_second_experiments_size(ne, M, K):
    """10^6 samples per stream, one bit flip per 10^4 output words."""
    n = 10 ** 6
    l, p, dg = plan(ne, M, K)
    c = inputs.streams(0, (1, M, n))
    g = inputs.operator_int8(0, (1, K))
    no = n + K - 1
    grp, pos, strm, bit = inputs.fault_list(1, 1, no, M, M * no // 10 ** 4)
    fl = (dev(pos.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))
    flags = torch.zeros((no + 31) // 32, dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = ne.ne_lconv(p, dg, dev(c), dev(g), None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 0, status=status,
                      faults=fl)
    assert int(status.item()) == 0 and int(nflag.item()) == len(pos)
    want = np.zeros(no, np.uint8)
    want[pos] = 1
    assert (unpack_flags(host(flags), 1, no)[0] == want).all()
    # every 5th fault in full: the oracle's entangled words there, the flip, Eq. 17-20
    take = np.arange(0, len(pos), 5)
    eps = oracle.entangle(c, l)
    sig = np.repeat(np.arange(M)[None, :], len(take), 0).reshape(-1)
    col = oracle.lconv_at(eps, g, sig, np.repeat(pos[take], M)).reshape(len(take), M, 1)
    col = inject(col, np.arange(len(take)), strm[take], bit[take])
    wd, wf = oracle.extract(col, l, 0)
    assert wf.all()
    gt = host(got[0][:, torch.from_numpy(pos[take]).to(DEV)])
    assert (gt.T == wd[:, :, 0]).all()
    # a sample of the other outputs (the ends included) against the direct convolution
    rng = np.random.default_rng(4)
    sp = np.concatenate([rng.integers(0, no, 400), [0, 1, K - 1, n - 1, no - 2, no - 1]])
    sp = sp[~np.isin(sp, pos)]
    sig = np.repeat(np.arange(M)[None, :], len(sp), 0).reshape(-1)
    wd = oracle.lconv_at(c.astype(np.int64), g, sig, np.repeat(sp, M)).reshape(len(sp), M)
    gt = host(got[0][:, torch.from_numpy(sp).to(DEV)])
    assert (gt.T == wd).all()


def test_lconv_checks_inputs_and_arguments(ne):
    M, n, K = 3, 1000, 200
    l, p, dg = plan(ne, M, K)
    g = dev(inputs.operator_int8(7, (1, K)))
    for r in range(M):
        c = inputs.streams(7, (1, M, n))
        c[0, r, 999] = 128                       # one past the range, on the lost stream
        status = torch.zeros(1, dtype=torch.int32, device=DEV)
        ne.ne_lconv(p, dg, dev(c), g, fuse=ne.NE_FUSE_RECOVER, r=r, status=status)
        assert int(status.item()) == ne.NE_ERANGE
    c = dev(inputs.streams(7, (1, M, n)))
    with pytest.raises(ne.NEError):
        ne.ne_lconv(p, dg, c, torch.zeros((1, 131072), dtype=torch.int8, device=DEV))   # K too long
    with pytest.raises(ne.NEError):
        ne.ne_lconv(p, dg, c, g, plain=True)                                          # plain has no extraction
