"""GPU parity of the streaming kernels and the int64 CUDA-core operations
against the CPU oracle, bit-exact, through the C ABI."""
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


def codewords(M, l, shape, seed):
    """entangled outputs of valid data with outputs in the exact range"""
    rng = np.random.default_rng(seed)
    lim = min(2 ** ((M - 1) * l - 1) - 1, 2 ** 62 // (2 ** l + 1))
    d = rng.integers(-lim, lim + 1, shape[:-2] + (M, shape[-1]), dtype=np.int64)
    d[..., 0, :2] = lim
    d[..., 1, 2:4] = -lim
    delta = np.stack([d[..., m, :] + (d[..., (m - 1) % M, :] << l) for m in range(M)], axis=-2)
    return d, delta


# ---- entanglement -------------------------------------------------------------------

@pytest.mark.parametrize("M,l", [(3, 11), (3, 16), (4, 10), (5, 8), (8, 9), (7, 5), (12, 5)])
@pytest.mark.parametrize("shape", [(1, 1), (3, 4096), (5, 1000), (2, 7), (1, 33)])
def test_entangle_matches_oracle(ne, M, l, shape):
    batch, n = shape
    rng = np.random.default_rng(M * 1000 + l)
    c = rng.integers(-(2 ** 31), 2 ** 31 - 1, (batch, M, n), dtype=np.int64).astype(np.int32)
    if l > 20:
        c //= 2 ** (l - 20)
    want = oracle.entangle(c, l)
    got = host(ne.ne_entangle(ne.params(M, l), dev(c)))
    assert (got == want).all()


def test_entangle_unaligned_pointers(ne):
    M, l, n = 3, 13, 1024
    c = inputs.streams(3, (2, M, n + 1))
    cd = dev(c.reshape(-1))[1:1 + 2 * M * n].view(2, M, n)   # 4-byte offset: scalar path
    want = oracle.entangle(np.ascontiguousarray(c.reshape(-1)[1:1 + 2 * M * n]).reshape(2, M, n), l)
    assert (host(ne.ne_entangle(ne.params(M, l), cd)) == want).all()


def test_entangle_empty_is_noop(ne):
    c = torch.empty((0, 3, 16), dtype=torch.int32, device=DEV)
    assert ne.ne_entangle(ne.params(3, 11), c).shape == (0, 3, 16)


@pytest.mark.parametrize("M,l,lo,hi", [(3, 16, -128, 127), (3, 13, -128, 127), (4, 16, -128, 127),
                                       (5, 8, -128, 127), (3, 11, -1000, 1000), (4, 10, -128, 127)])
@pytest.mark.parametrize("shape", [(4, 1024), (1, 24), (3, 13)])
def test_entangle_digits_recombine_to_words(ne, M, l, lo, hi, shape):
    batch, n = shape
    c = inputs.int32_uniform(M + l, inputs.TAG_C, (batch, M, n), lo, hi)
    dg = ne.ne_plan_digits(l, lo, hi)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    planes = host(ne.ne_entangle_digits(ne.params(M, l), dg, dev(c), status=status))
    assert int(status.item()) == 0
    eps = oracle.entangle(c, l)
    rec = np.zeros_like(eps)
    for s, sh in enumerate(dg.shifts):
        assert planes[:, :, s].min() >= -128 and planes[:, :, s].max() <= 127
        rec += planes[:, :, s].astype(np.int64) << sh
    assert (rec == eps).all()


@pytest.mark.parametrize("M,l,lo,hi", [(3, 16, -128, 127), (4, 13, -128, 127), (5, 8, -100, 100), (3, 24, -128, 127)])
def test_entangle_digits_range_checked_path_equals_generic_path(ne, M, l, lo, hi):
    # a plan from ne_plan_digits carries its input range (checked per input,
    # 32-bit word arithmetic); the same digit set without a range checks
    # every word on the generic path.  Both must write the same planes.
    c = inputs.int32_uniform(l, inputs.TAG_C, (8, M, 1024), lo, hi)
    dg = ne.ne_plan_digits(l, lo, hi)
    dg_generic = ne.digits(dg.shifts)
    st1 = torch.zeros(1, dtype=torch.int32, device=DEV)
    st2 = torch.zeros(1, dtype=torch.int32, device=DEV)
    a = ne.ne_entangle_digits(ne.params(M, l), dg, dev(c), status=st1)
    b = ne.ne_entangle_digits(ne.params(M, l), dg_generic, dev(c), status=st2)
    assert (host(a) == host(b)).all() and int(st1.item()) == 0 and int(st2.item()) == 0
    bad = c.copy()
    bad[3, 1, 77] = hi + 1
    ne.ne_entangle_digits(ne.params(M, l), dg, dev(bad), status=st1)
    assert int(st1.item()) == ne.NE_ERANGE


def test_entangle_digits_reports_out_of_plan_words(ne):
    M, l = 3, 16
    dg = ne.ne_plan_digits(l, -128, 127)            # digits 0 and 2 only
    c = np.full((1, M, 64), 5, np.int32)
    c[0, 1, 7] = 300                                 # needs digit 1
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_entangle_digits(ne.params(M, l), dg, dev(c), status=status)
    assert int(status.item()) == ne.NE_ERANGE


# ---- extraction, check, recovery --------------------------------------------------

@pytest.mark.parametrize("M,l", [(3, 11), (3, 13), (3, 22), (4, 10), (4, 16), (5, 8), (6, 7), (7, 5), (8, 9),
                                 (12, 5), (32, 2)])
@pytest.mark.parametrize("shape", [(1, 4096), (4, 1000), (3, 33), (2, 64), (1, 1), (5, 31)])
def test_extract_check_recover_match_oracle(ne, M, l, shape):
    batch, n = shape
    d, delta = codewords(M, l, (batch, M, n), seed=M * 7 + l + n)
    # corrupt some positions: a single bit flip, arbitrary words, and two
    # co-located faults forming a valid codeword (undetectable by design)
    rng = np.random.default_rng(l)
    bad = delta.copy()
    for t in range(min(n, 5)):
        b, i, j = t % batch, rng.integers(n), rng.integers(M)
        bad[b, j, i] ^= np.int64(1) << np.int64(rng.integers(63))
    bad[0, M - 1, 0] = np.int64(-(2 ** 63))
    p = ne.params(M, l)
    for r in sorted({0, 1, M - 1}):
        want_d, want_f = oracle.extract(bad, l, r)
        wf = torch.zeros(batch * ((n + 31) // 32), dtype=torch.int32, device=DEV)
        nf = torch.zeros(1, dtype=torch.int64, device=DEV)
        got = host(ne.ne_extract(p, dev(bad), r=r, flags=wf, nflag=nf))
        assert (got == want_d).all(), f"extract r={r}"
        gf = unpack_flags(host(wf), batch, n)
        assert (gf == want_f).all(), f"flags r={r}"
        assert int(nf.item()) == int(want_f.sum())
        # check only
        wf2 = ne.ne_check(p, dev(bad), r=r)
        assert (unpack_flags(host(wf2), batch, n) == want_f).all()
        # fail-stop recovery: plane r poisoned, never read
        pois = delta.copy()
        pois[:, r, :] = np.int64(0x5A5A5A5A5A5A5A5A)
        assert (host(ne.ne_recover(p, dev(pois), r)) == d).all()
        # clean data: outputs equal the codeword data, no flags
        got_clean = host(ne.ne_extract(p, dev(delta), r=r, nflag=nf))
        assert (got_clean == d).all() and int(nf.item()) == 0


@pytest.mark.parametrize("M,l", [(3, 16), (3, 11), (4, 16), (5, 15), (6, 10), (8, 8)])
def test_staged_check_walks_many_units_per_block(ne, M, l):
    """The check with its reads staged in shared memory: enough groups that every
    block of the persistent launch goes round its ring of stages several times,
    n = 1000 so the second unit of every group is ragged, faults scattered over
    all streams; and the same data 8 bytes off alignment (the unstaged kernel)."""
    batch, n = (2600 if M == 3 else 700), 1000
    d, delta = codewords(M, l, (batch, M, n), seed=M * 31 + l)
    rng = np.random.default_rng(M + l)
    k = 3000
    gb, gi, gj = rng.integers(batch, size=k), rng.integers(n, size=k), rng.integers(M, size=k)
    bits = rng.integers(64, size=k).astype(np.uint64)
    np.bitwise_xor.at(delta.view(np.uint64), (gb, gj, gi), np.uint64(1) << bits)
    p = ne.params(M, l)
    for r in sorted({0, M - 1}):
        _, want_f = oracle.extract(delta, l, r)
        nf = torch.zeros(1, dtype=torch.int64, device=DEV)
        status = torch.zeros(1, dtype=torch.int32, device=DEV)
        wf = ne.ne_check(p, dev(delta), r=r, nflag=nf, status=status)
        assert (unpack_flags(host(wf), batch, n) == want_f).all(), f"r={r}"
        assert int(nf.item()) == int(want_f.sum()) and int(status.item()) == 0
        off = torch.empty(delta.size + 1, dtype=torch.int64, device=DEV)
        t = off[1:].view(batch, M, n)
        t.copy_(dev(delta))
        wf2 = ne.ne_check(p, t, r=r)
        assert (unpack_flags(host(wf2), batch, n) == want_f).all(), f"unaligned r={r}"


def test_every_single_bit_flip_flagged_on_gpu(ne):
    M, l, n = 4, 10, 256
    d, delta = codewords(M, l, (1, M, n), seed=11)
    p = ne.params(M, l)
    nf = torch.zeros(1, dtype=torch.int64, device=DEV)
    for j in range(M):
        for b in range(64):
            x = delta.copy()
            x[0, j, :] ^= np.int64(np.uint64(1 << b).view(np.int64))
            ne.ne_check(p, dev(x), r=(j + 1) % M, nflag=nf)
            assert int(nf.item()) == n, f"stream {j} bit {b}"


def test_inject_flips_listed_bits(ne):
    M, batch, n = 3, 4, 100
    delta = np.zeros((batch, M, n), np.int64)
    g, pos, j, b = inputs.fault_list(9, batch, n, M, 37)
    t = dev(delta)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ne.ne_inject(t, M, dev(g), dev(pos), dev(j), dev(b), status)
    want = delta.copy()
    for gi, pi, ji, bi in zip(g, pos, j, b):
        want[gi, ji, pi] ^= np.int64(np.uint64(1 << int(bi)).view(np.int64))
    assert (host(t) == want).all() and int(status.item()) == 0
    ne.ne_inject(t, M, *(dev(np.array([v], np.int64)) for v in (batch, 0, 0, 0)), status)
    assert int(status.item()) == ne.NE_EINVAL


# ---- int64 CUDA-core operations -----------------------------------------------------

@pytest.mark.parametrize("P,rows,cols,k", [(3, 64, 64, 64), (1, 1, 1, 1), (2, 65, 33, 17), (4, 100, 130, 250),
                                           (3, 7, 200, 96)])
def test_gemm_i64_matches_oracle(ne, P, rows, cols, k):
    rng = np.random.default_rng(rows + cols + k)
    x = rng.integers(-(2 ** 40), 2 ** 40, (P, rows, k), dtype=np.int64)
    G = rng.integers(-128, 128, (k, cols)).astype(np.int8)
    got = host(ne.ne_gemm(ne.planes_of(P), dev(x), dev(G), fuse=ne.NE_FUSE_NONE))
    for q in range(P):
        assert (got[q] == oracle.gemm(x[q], G)).all()


def test_gemm_i64_skip_mask_leaves_plane_untouched(ne):
    x = np.ones((3, 16, 16), np.int64)
    G = np.ones((16, 16), np.int8)
    out = torch.full((3, 16, 16), 7, dtype=torch.int64, device=DEV)
    ne.ne_gemm(ne.planes_of(3), dev(x), dev(G), out=out, fuse=ne.NE_FUSE_NONE, drop_mask=0b010)
    o = host(out)
    assert (o[1] == 7).all() and (o[0] == 16).all() and (o[2] == 16).all()


@pytest.mark.parametrize("batch,P,N", [(4, 3, 1024), (2, 4, 100), (1, 3, 1), (3, 5, 2048), (1, 3, 3000), (2, 3, 1500)])
def test_cconv_i64_matches_oracle(ne, batch, P, N):
    rng = np.random.default_rng(N + P)
    x = rng.integers(-(2 ** 35), 2 ** 35, (batch, P, N), dtype=np.int64)
    g = rng.integers(-128, 128, (batch, N)).astype(np.int8)
    got = host(ne.ne_cconv(ne.planes_of(P), dev(x), dev(g), fuse=ne.NE_FUSE_NONE))
    assert (got == oracle.cconv(x, g)).all()


# ---- full int64 pipelines -------------------------------------------------------------

def test_cconv_pipeline_int64(ne):
    B, M, N = 16, 3, 1024
    l, _ = ne.ne_choose_l(M, 64, N * 2 ** 14, ne.NE_L_SMALLEST)
    c = inputs.streams(0, (B, M, N))
    g = inputs.operator_int8(0, (B, N))
    p = ne.params(M, l)
    delta = ne.ne_cconv(p, ne.ne_entangle(p, dev(c)), dev(g), fuse=ne.NE_FUSE_NONE)
    nf = torch.zeros(1, dtype=torch.int64, device=DEV)
    dh = host(ne.ne_extract(p, delta, r=0, nflag=nf))
    assert (dh == oracle.cconv_direct(c, g)).all() and int(nf.item()) == 0


def test_gemm_pipeline_config1_int64(ne):
    # M = 3 streams of 64x64 int32 values, shared 64x64 int8, l from the K=64 bound,
    # one bit flip in one entangled output stream, one dropped stream.
    M = 3
    c = inputs.streams(0, (M, 64, 64))
    G = inputs.operator_int8(0, (64, 64))
    l, _ = ne.ne_choose_l(M, 64, 64 * 2 ** 14, ne.NE_L_SMALLEST)
    assert l == 11
    p = ne.params(M, l)
    eps = ne.ne_entangle(p, dev(c).reshape(M, 64 * 64)).reshape(M, 64, 64)
    delta = ne.ne_gemm(p, eps, dev(G), fuse=ne.NE_FUSE_NONE).reshape(1, M, 64 * 64)
    want = oracle.gemm_direct(c, G).reshape(1, M, -1)
    gi, pos, j, b = inputs.fault_list(1, 1, 64 * 64, M, 1)
    ne.ne_inject(delta, M, dev(gi), dev(pos), dev(j), dev(b))
    flags = ne.ne_check(p, delta, r=0)
    f = unpack_flags(host(flags), 1, 64 * 64)
    assert f.sum() == 1 and f[0, pos[0]] == 1
    rec = host(ne.ne_recover(p, delta, int(j[0])))
    assert (rec == want).all()


# ---- checksum ABFT -----------------------------------------------------------------

def test_abft_pipeline(ne):
    M, B, N = 3, 4, 512
    c = inputs.streams(5, (B, M, N))
    g = inputs.operator_int8(5, (B, N))
    x = ne.ne_abft_encode(M, dev(c))
    xh = host(x)
    for b in range(B):
        assert (xh[b, M] == oracle.abft_encode(c[b])).all()
    d = ne.ne_cconv(ne.planes_of(M + 1), x, dev(g), fuse=ne.NE_FUSE_NONE)
    nf = torch.zeros(1, dtype=torch.int64, device=DEV)
    ne.ne_abft_check(M, d, nflag=nf)
    assert int(nf.item()) == 0
    ne.ne_inject(d, M + 1, *(dev(np.array([v], np.int64)) for v in (2, 100, 1, 5)))
    flags = ne.ne_abft_check(M, d, nflag=nf)
    f = unpack_flags(host(flags), B, N)
    assert int(nf.item()) == 1 and f[2, 100] == 1
    for b in range(B):
        assert (f[b] == oracle.abft_check(host(d)[b])).all()
    ne.ne_abft_recover(M, d, 1)
    assert (host(d)[:, :M] == oracle.cconv_direct(c, g)).all()
