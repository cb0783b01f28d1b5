"""GPU parity of the fused operations under seeded transient faults (the fault
model of Sec. I: one stream's result of the operation corrupted), through the
C ABI's fault hook, against the CPU oracle, bit-exact: the entangled words
with the faults XORed in (NE_FUSE_NONE), the extracted outputs and the Eq. 24
flags (NE_FUSE_EXTRACT_CHECK, several r), and recovery with the lost stream's
faults never seen (NE_FUSE_RECOVER).  Every form of the convolution (tensor
tiles from digit planes, the fused tile from raw streams -- its dp4a blocks
included -- and both exact transforms) and the product are covered, at small
sizes in full and at the full workload sizes on every fault plus a sample of
the other outputs.  Also: the lost stream's inputs are range-checked under
fused recovery."""
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


def fault_set(seed, groups, positions, M, count):
    """Flat positions (group * positions + i), streams and bits, sorted, at most
    one fault per co-located group (inputs.fault_list)."""
    grp, pos, strm, bit = inputs.fault_list(seed, groups, positions, M, count)
    return grp * positions + pos, strm, bit


def dev_faults(flat, strm, bit):
    return (dev(flat.astype(np.int64)), dev(strm.astype(np.int32)), dev(bit.astype(np.int32)))


def inject(delta, flat, strm, bit, skip_stream=None):
    """delta [B, M, n] with bit b of delta[g, m, i] flipped for every fault
    (those on skip_stream left out)."""
    d = np.array(delta, dtype=np.int64, copy=True).view(np.uint64)
    n = d.shape[-1]
    keep = np.ones(len(flat), bool) if skip_stream is None else (strm != skip_stream)
    g, i = flat[keep] // n, flat[keep] % n
    np.bitwise_xor.at(d, (g, strm[keep], i), np.uint64(1) << bit[keep].astype(np.uint64))
    return d.view(np.int64)


def flags_of(flat, B, n):
    want = np.zeros((B, n), np.uint8)
    want[flat // n, flat % n] = 1
    return want


# ---- the convolution forms in full -----------------------------------------------------

def run_cconv(ne, form, p, dg, c, g, fuse, r, fl, flags=None, nflag=None, status=None):
    cd, gd = dev(c), dev(g)
    if form == "entangled":
        return ne.ne_cconv_entangled(p, dg, cd, gd, None, flags, nflag, fuse, r, status=status, faults=fl)
    if form == "digits":
        planes = ne.ne_entangle_digits(p, dg, cd)
        return ne.ne_cconv_digits(p, dg, planes, gd, None, flags, nflag, fuse, r, faults=fl)
    if form == "ntt":
        return ne.ne_cconv_ntt(p, dg, cd, gd, None, flags, nflag, fuse, r, status=status, faults=fl)
    if form == "ntt_any":
        return ne.ne_cconv_ntt_any(p, cd, gd, None, flags, nflag, fuse, r, status=status, faults=fl)
    raise ValueError(form)


CCONV_CASES = [
    # form, B, M, N
    ("entangled", 9, 3, 1024),      # hybrid tile: 10 blocks on the tensor pipe, 6 on dp4a
    ("entangled", 5, 4, 1024),      # hybrid tile of 8 planes
    ("entangled", 3, 3, 2048),      # two chunks of shifts, two tiles per group
    ("entangled", 4, 5, 576),       # generic tile, ragged chunk
    ("entangled", 2, 8, 1024),      # eight streams (l = 8, 16 digit planes)
    ("digits", 2, 6, 512),          # a stream count without its own instantiation
    ("digits", 9, 3, 1024),
    ("digits", 3, 4, 1088),
    ("ntt", 7, 3, 1024),
    ("ntt", 3, 4, 1024),
    ("ntt_any", 4, 3, 1000),        # not a power of two: linear convolution folded
    ("ntt_any", 2, 4, 4096),
]


@pytest.mark.parametrize("form,B,M,N", CCONV_CASES)
def test_cconv_under_faults_matches_oracle(ne, form, B, M, N):
    l = oracle.choose_l(M, 64, N * 2 ** 14, oracle.POLICY_BYTE)[0]
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    seed = 300 + 7 * M + N
    c = inputs.streams(seed, (B, M, N))
    c[0, 0, :3] = -128
    c[-1, -1, -3:] = 127
    g = inputs.operator_int8(seed, (B, N))
    direct = oracle.cconv_direct(c, g)
    delta = oracle.cconv(oracle.entangle(c, l), g)
    flat, strm, bit = fault_set(seed, B, N, M, max(8, B * N // 40))
    fl = dev_faults(flat, strm, bit)
    bad = inject(delta, flat, strm, bit)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    # NE_FUSE_NONE: the words with the faults in them
    got = host(run_cconv(ne, form, p, dg, c, g, ne.NE_FUSE_NONE, 0, fl, status=status))
    assert (got == bad).all()
    for r in sorted({0, 1, M - 1}):
        flags = torch.full((ne.flag_words(B, N),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
        got = host(run_cconv(ne, form, p, dg, c, g, ne.NE_FUSE_EXTRACT_CHECK, r, fl, flags, nflag, status))
        want, wflags = oracle.extract(bad, l, r)
        assert (got == want).all(), (form, r)                        # flagged positions included
        gflags = unpack_flags(host(flags), B, N)
        assert (gflags == wflags).all()
        assert (gflags == flags_of(flat, B, N)).all()                # every single-stream fault flagged
        assert int(nflag.item()) == len(flat)
        unflagged = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
        assert (got[unflagged] == direct[unflagged]).all()
        # fused recovery: stream r is never computed, so its faults cannot land
        got = host(run_cconv(ne, form, p, dg, c, g, ne.NE_FUSE_RECOVER, r, fl, status=status))
        want = oracle.recover(inject(delta, flat, strm, bit, skip_stream=r), l, r)
        assert (got == want).all(), (form, r)
    assert int(status.item()) == 0


# ---- the product in full ---------------------------------------------------------------

GEMM_CASES = [
    # M, rows, cols, k, l
    (4, 96, 128, 1024, 16),     # the large product's plan (two digits, 8 planes); whole flag words
    (3, 70, 40, 256, 16),       # ragged row tile, flags by atomics
    (5, 33, 64, 512, 8),
]


@pytest.mark.parametrize("M,rows,cols,k,l", GEMM_CASES)
def test_gemm_under_faults_matches_oracle(ne, M, rows, cols, k, l):
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    seed = 400 + rows + cols
    c = inputs.streams(seed, (M, rows, k))
    G = inputs.operator_int8(seed, (k, cols))
    planes = ne.ne_entangle_digits(p, dg, dev(c).reshape(M, rows * k)).reshape(M, dg.S, rows, k)
    Gd = dev(G)
    direct = oracle.gemm_direct(c, G).reshape(1, M, rows * cols)
    eps = oracle.entangle(c.reshape(M, rows * k), l).reshape(M, rows, k)
    delta = np.stack([oracle.gemm(eps[m], G) for m in range(M)]).reshape(1, M, rows * cols)
    flat, strm, bit = fault_set(seed, 1, rows * cols, M, rows * cols // 30)
    fl = dev_faults(flat, strm, bit)
    bad = inject(delta, flat, strm, bit)
    got = host(ne.ne_gemm_digits(p, dg, planes, Gd, fuse=ne.NE_FUSE_NONE, faults=fl)).reshape(1, M, -1)
    assert (got == bad).all()
    for r in sorted({0, M - 1}):
        flags = torch.full((ne.flag_words(1, rows * cols),), -1, dtype=torch.int32, device=DEV)
        nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
        got = host(ne.ne_gemm_digits(p, dg, planes, Gd, None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, r,
                                     faults=fl)).reshape(1, M, -1)
        want, wflags = oracle.extract(bad, l, r)
        assert (got == want).all()
        gflags = unpack_flags(host(flags), 1, rows * cols)
        assert (gflags == wflags).all() and (gflags == flags_of(flat, 1, rows * cols)).all()
        assert int(nflag.item()) == len(flat)
        unflagged = np.broadcast_to((gflags == 0)[:, None, :], got.shape)
        assert (got[unflagged] == direct[unflagged]).all()
        got = host(ne.ne_gemm_digits(p, dg, planes, Gd, fuse=ne.NE_FUSE_RECOVER, r=r, faults=fl)).reshape(1, M, -1)
        assert (got == oracle.recover(inject(delta, flat, strm, bit, skip_stream=r), l, r)).all()


# ---- the full workload sizes: every fault plus a sample of the other outputs -------------

def test_config2_size_cconv_flags_exactly_the_injected_faults(ne):
    """4096 groups x M = 3 x N = 1024, l = 16, the one-launch fused step
    (hybrid tile, its dp4a blocks included), one flip per 10^4 output words."""
    B, M, N, l = 4096, 3, 1024, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(0, (B, M, N))
    g = inputs.operator_int8(0, (B, N))
    flat, strm, bit = fault_set(1, B, N, M, B * M * N // 10 ** 4)
    fl = dev_faults(flat, strm, bit)
    flags = torch.zeros(ne.flag_words(B, N), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = host(ne.ne_cconv_entangled(p, dg, dev(c), dev(g), None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 0,
                                     status=status, faults=fl))
    assert int(status.item()) == 0
    assert int(nflag.item()) == len(flat)
    assert (unpack_flags(host(flags), B, N) == flags_of(flat, B, N)).all()
    # every faulted position: the oracle's words there, the fault, Eq. 17-20
    grp, pos = flat // N, flat % N
    eps = oracle.entangle(c[grp], l)                                    # [F, M, N], the groups hit
    sig = (np.arange(len(flat))[:, None] * M + np.arange(M)[None, :]).reshape(-1)
    col = oracle.cconv_at(eps, g[grp], sig, np.repeat(pos, M)).reshape(len(flat), M, 1)
    col = inject(col, np.arange(len(flat)), strm, bit)
    want, wflags = oracle.extract(col, l, 0)
    assert wflags.all()
    assert (got[grp, :, pos] == want[:, :, 0]).all()
    # a sample of the other outputs against the direct convolution
    rng = np.random.default_rng(2)
    sg = rng.integers(0, B, 512)
    sp = rng.integers(0, N, 512)
    keep = ~np.isin(sg * N + sp, flat)
    sg, sp = sg[keep], sp[keep]
    sig = (sg[:, None] * M + np.arange(M)[None, :]).reshape(-1)
    want = oracle.cconv_at(c.astype(np.int64), g, sig, np.repeat(sp, M)).reshape(-1, M)
    assert (got[sg, :, sp] == want).all()


def test_config3_size_gemm_flags_exactly_the_injected_faults(ne):
    """M = 4 streams of 4096 x 4096 times a shared 4096 x 4096 operator, l = 16,
    fused epilogue, one flip per 10^4 output words."""
    M, n, l = 4, 4096, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    c = inputs.streams(0, (M, n, n))
    G = inputs.operator_int8(0, (n, n))
    cd = dev(c)
    planes = ne.ne_entangle_digits(p, dg, cd.reshape(M, n * n)).reshape(M, dg.S, n, n)
    del cd
    flat, strm, bit = fault_set(1, 1, n * n, M, M * n * n // 10 ** 4)
    fl = dev_faults(flat, strm, bit)
    flags = torch.zeros(ne.flag_words(1, n * n), dtype=torch.int32, device=DEV)
    nflag = torch.zeros(1, dtype=torch.int64, device=DEV)
    got = ne.ne_gemm_digits(p, dg, planes, dev(G), None, flags, nflag, ne.NE_FUSE_EXTRACT_CHECK, 0, faults=fl)
    assert int(nflag.item()) == len(flat)
    assert (unpack_flags(host(flags), 1, n * n)[0] == flags_of(flat, 1, n * n)[0]).all()
    rows, cols = flat // n, flat % n
    # the faulted outputs: eps rows of the oracle times G's columns, fault, extract
    take = np.arange(0, len(flat), 7)                                   # every 7th fault in full
    r_, c_ = rows[take], cols[take]
    got_f = host(got[:, torch.from_numpy(r_).to(DEV), torch.from_numpy(c_).to(DEV)])   # [M, F]
    col = np.empty((len(take), M, 1), np.int64)
    for t, (i, j) in enumerate(zip(r_, c_)):
        e = oracle.entangle(c[:, i, :], l)                              # [M, n]
        for m in range(M):
            col[t, m, 0] = oracle.gemm(e[m:m + 1], G[:, j:j + 1])[0, 0]
    col = inject(col, np.arange(len(take)), strm[take], bit[take])
    want, wflags = oracle.extract(col, l, 0)
    assert wflags.all() and (got_f.T == want[:, :, 0]).all()
    # a sample of the unflagged outputs against the direct product
    rng = np.random.default_rng(3)
    si, sj = rng.integers(0, n, 64), rng.integers(0, n, 64)
    keep = ~np.isin(si * n + sj, flat)
    si, sj = si[keep], sj[keep]
    got_s = host(got[:, torch.from_numpy(si).to(DEV), torch.from_numpy(sj).to(DEV)])
    for t, (i, j) in enumerate(zip(si, sj)):
        for m in range(M):
            assert got_s[m, t] == oracle.gemm(c[m, i:i + 1].astype(np.int64), G[:, j:j + 1])[0, 0]


# ---- fused recovery checks the lost stream's inputs --------------------------------------

@pytest.mark.parametrize("form", ["entangled", "ntt", "ntt_any"])
def test_recover_checks_the_lost_streams_inputs(ne, form):
    B, M, N, l = 3, 3, 1024, 16
    p = ne.params(M, l)
    dg = ne.ne_plan_digits(l, -128, 127)
    g = inputs.operator_int8(55, (B, N))
    for r in range(M):
        c = inputs.streams(55, (B, M, N))
        status = torch.zeros(1, dtype=torch.int32, device=DEV)
        run_cconv(ne, form, p, dg, c, g, ne.NE_FUSE_RECOVER, r, None, status=status)
        assert int(status.item()) == 0
        c[1, r, 333] = 128                       # one past the planned range, on the lost stream
        run_cconv(ne, form, p, dg, c, g, ne.NE_FUSE_RECOVER, r, None, status=status)
        assert int(status.item()) == ne.NE_ERANGE, (form, r)


def test_fault_lists_are_validated_on_the_host(ne):
    p = ne.params(3, 16)
    dg = ne.ne_plan_digits(16, -128, 127)
    c = torch.zeros((1, 3, 1024), dtype=torch.int32, device=DEV)
    g = torch.zeros((1, 1024), dtype=torch.int8, device=DEV)
    f = ne.ne_faults()
    f.count = 3                                  # entries but no lists
    with pytest.raises(ne.NEError):
        ne.ne_cconv_entangled(p, dg, c, g, faults=f)
    f.count = -1
    with pytest.raises(ne.NEError):
        ne.ne_cconv_entangled(p, dg, c, g, faults=f)
