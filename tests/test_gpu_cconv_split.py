"""GPU parity of every tensor / dp4a split of the convolution tile
(ne_set_cconv_split) against the CPU oracle, bit-exact, under seeded faults:
each split from raw streams, digit planes and entangled words, at 16-block
groups and at shorter groups (where a split that leaves no block for the
tensor pipe falls back to it), with the extraction and check of Eq. 17-20 /
Eq. 24 and with recovery.  The dp4a threads own outputs 4 apart and slide one
filter word per 4 inputs along them, so a wrong index shows up here as a
wrong output block."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs
from tests.helpers import unpack_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"

SPLITS = [0, 23, 24, 34, 42, 43, 44, 443, 444]


@pytest.fixture(scope="module")
def ne():
    from paper_1604_04740_gb300 import ne as _ne
    yield _ne
    _ne.ne_set_cconv_split(-1)


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


@pytest.mark.parametrize("M,N,B", [(3, 1024, 5), (4, 1024, 3), (3, 640, 3), (4, 832, 2)])
def test_every_split_matches_oracle_under_faults(ne, M, N, B):
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    seed = 4000 + 10 * M + N
    c = inputs.streams(seed, (B, M, N))
    c[0, 0, :3] = -128
    c[-1, -1, -3:] = 127
    g = inputs.operator_int8(seed, (B, N))
    g[0, :5] = -128
    direct = oracle.cconv_direct(c, g)
    eps = oracle.entangle(c, l)
    delta = oracle.cconv(eps, g)
    grp, pos, strm, bit = inputs.fault_list(seed, B, N, M, B * N // 40)
    flat = grp * N + pos
    fl = (dev(flat.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))
    bad = inject(delta, flat, strm, bit)
    r = M - 1
    want, wflags = oracle.extract(bad, l, r)
    want_rec = oracle.recover(inject(delta, flat, strm, bit, skip=r), l, r)
    cd, gd, ed = dev(c), dev(g), dev(eps)
    planes = ne.ne_entangle_digits(p, dg, cd)
    forms = {
        "raw": lambda **kw: ne.ne_cconv_entangled(p, dg, cd, gd, **kw),
        "planes": lambda **kw: ne.ne_cconv_digits(p, dg, planes, gd, **kw),
        "words": lambda **kw: ne.ne_cconv(p, ed, gd, mode=ne.NE_MODE_S8SLICE, dg=dg, **kw),
    }
    for split in SPLITS:
        ne.ne_set_cconv_split(split)
        for name, run in forms.items():
            assert (host(run(fuse=ne.NE_FUSE_NONE, faults=fl)) == bad).all(), (split, name)
            flags = torch.full((ne.flag_words(B, N),), -1, dtype=torch.int32, device=DEV)
            nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
            got = host(run(flags=flags, nflag=nflag, fuse=ne.NE_FUSE_EXTRACT_CHECK, r=r, faults=fl))
            assert (got == want).all(), (split, name)
            gflags = unpack_flags(host(flags), B, N)
            assert (gflags == wflags).all() and int(nflag.item()) == len(flat), (split, name)
            ok = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
            assert (got[ok] == direct[ok]).all()
            got = host(run(fuse=ne.NE_FUSE_RECOVER, r=r, faults=fl))
            assert (got == want_rec).all(), (split, name)
        # the plain operation through the same tile
        got = host(ne.ne_cconv_entangled(p, ne.raw_digits(), cd, gd, fuse=ne.NE_FUSE_NONE, plain=True))
        assert (got == direct).all(), split
    ne.ne_set_cconv_split(-1)


def test_unknown_splits_are_refused(ne):
    for v in (1, 22, 25, 33, 45, 52, 62, 99, -2):
        with pytest.raises(ne.NEError):
            ne.ne_set_cconv_split(v)
    ne.ne_set_cconv_split(-1)
