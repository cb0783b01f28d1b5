"""Pins for the oracle's LSB operations, the ABFT comparator and the composed
pipelines: textbook/library routines (numpy matmul, an explicit circulant
matrix, numpy FFT), Python big-integer brute force and the invariant that
disentangled outputs equal the direct outputs (Prop. 3-4)."""
import numpy as np
import pytest

import oracle
from paper_1604_04740_gb300 import inputs


def test_gemm_matches_numpy_matmul():
    rng = np.random.default_rng(0)
    for m, n, k in [(1, 1, 1), (7, 5, 3), (33, 17, 65), (64, 64, 64)]:
        A = rng.integers(-(2 ** 20), 2 ** 20, (m, k), dtype=np.int64)
        G = rng.integers(-128, 128, (k, n)).astype(np.int8)
        assert (oracle.gemm(A, G) == A @ G.astype(np.int64)).all()


def test_gemm_big_int_brute_force_and_overflow():
    A = np.array([[2 ** 55, -(2 ** 55)], [3, 4]], np.int64)
    G = np.array([[127, -128], [127, 127]], np.int8)
    want = [[sum(int(A[i, t]) * int(G[t, j]) for t in range(2)) for j in range(2)] for i in range(2)]
    assert oracle.gemm(A, G).tolist() == want
    # a partial sum beyond int64 is reported even if the final sum would fit
    A2 = np.array([[2 ** 62, -(2 ** 62)]], np.int64)
    G2 = np.array([[2], [2]], np.int8)
    with pytest.raises(oracle.OracleError):
        oracle.gemm(A2, G2)


def test_cconv_matches_circulant_matrix_and_fft():
    rng = np.random.default_rng(1)
    for N in (1, 2, 5, 16, 100, 256):
        x = rng.integers(-(2 ** 20), 2 ** 20, (2, 3, N), dtype=np.int64)
        g = rng.integers(-128, 128, (2, N)).astype(np.int8)
        y = oracle.cconv(x, g)
        for b in range(2):
            C = np.array([[int(g[b, (i - j) % N]) for j in range(N)] for i in range(N)], np.int64)
            for s in range(3):
                assert (y[b, s] == C @ x[b, s]).all()
        # FFT route on small-magnitude data (exact after rounding)
        xs = rng.integers(-100, 100, (1, 1, N), dtype=np.int64)
        ys = oracle.cconv(xs, g[:1])
        f = np.fft.ifft(np.fft.fft(xs[0, 0].astype(float)) * np.fft.fft(g[0].astype(float))).real
        assert (ys[0, 0] == np.rint(f).astype(np.int64)).all()


def test_cconv_tiny_brute_force():
    x = np.array([[[1, 2, 3]]], np.int64)
    g = np.array([[1, 0, -1]], np.int8)
    # y[n] = sum_j x[j] g[(n-j) mod 3]:  y0 = 1*1 + 2*g[2] + 3*g[1] = 1 - 2 = -1
    #                                     y1 = 1*g[1] + 2*g[0] + 3*g[2] = 2 - 3 = -1
    #                                     y2 = 1*g[2] + 2*g[1] + 3*g[0] = -1 + 3 = 2
    assert oracle.cconv(x, g)[0, 0].tolist() == [-1, -1, 2]


def test_elementwise_and_self_entangled_kernel():
    rng = np.random.default_rng(2)
    x = rng.integers(-(2 ** 30), 2 ** 30, 50, dtype=np.int64)
    g = rng.integers(-(2 ** 20), 2 ** 20, 50, dtype=np.int64)
    assert (oracle.elementwise(oracle.OP_ADD, x, g) == x + g).all()
    assert (oracle.elementwise(oracle.OP_SUB, x, g) == x - g).all()
    assert (oracle.elementwise(oracle.OP_MUL, x, g) == x * g).all()
    assert (oracle.entangle_kernel_self(g, 9) == g * 513).all()


def test_elementwise_add_pipeline_uses_self_entangled_kernel():
    # Footnote to Eq. 10: with g <- S_l{g} + g the entangled sum decodes to c + g.
    M, l, n = 3, 12, 64
    rng = np.random.default_rng(5)
    c = rng.integers(-500, 500, (M, n)).astype(np.int32)
    g = rng.integers(-500, 500, n, dtype=np.int64)
    eps = oracle.entangle(c, l)
    ge = oracle.entangle_kernel_self(g, l)
    for op, want in ((oracle.OP_ADD, c + g), (oracle.OP_SUB, c - g)):
        delta = np.stack([oracle.elementwise(op, eps[m], ge) for m in range(M)])
        dh, fl = oracle.extract(delta, l, 0)
        assert (dh == want).all() and not fl.any()
    delta = np.stack([oracle.elementwise(oracle.OP_MUL, eps[m], g) for m in range(M)])
    dh, fl = oracle.extract(delta, l, 1)
    assert (dh == c * g).all() and not fl.any()


def test_abft_encode_check_recover():
    rng = np.random.default_rng(3)
    M, n = 4, 100
    c = rng.integers(-(2 ** 31), 2 ** 31 - 1, (M, n)).astype(np.int32)
    r = oracle.abft_encode(c)
    assert (r == c.astype(np.int64).sum(axis=0)).all()
    # op = elementwise x g on M+1 streams (Eq. 5)
    g = rng.integers(-128, 128, n, dtype=np.int64)
    d = np.concatenate([c.astype(np.int64) * g, (r * g)[None]])
    assert not oracle.abft_check(d).any()
    bad = d.copy()
    bad[2, 17] ^= 1 << 40
    f = oracle.abft_check(bad)
    assert f[17] and f.sum() == 1
    lost = d.copy()
    lost[1] = 999
    assert (oracle.abft_recover(lost, 1) == d).all()


@pytest.mark.parametrize("M,l", [(3, 11), (3, 22), (4, 10), (4, 16), (5, 8)])
def test_gemm_pipeline_equals_direct(M, l):
    c = inputs.streams(0, (M, 24, 40))
    G = inputs.operator_int8(0, (40, 19))
    direct = oracle.gemm_direct(c, G)
    for r in range(M):
        dh, fl, delta = oracle.gemm_entangled(c, G, l, r)
        assert (dh == direct).all() and not fl.any()
        assert (oracle.recover(delta.reshape(M, -1), l, r).reshape(dh.shape) == direct).all()


@pytest.mark.parametrize("M,l,N", [(3, 13, 64), (3, 16, 100), (4, 16, 33), (5, 8, 50)])
def test_cconv_pipeline_equals_direct(M, l, N):
    c = inputs.streams(1, (3, M, N))
    g = inputs.operator_int8(1, (3, N))
    direct = oracle.cconv_direct(c, g)
    dh, fl, delta = oracle.cconv_entangled(c, g, l, 0)
    assert (dh == direct).all() and not fl.any()


def test_inputs_generator_is_stable():
    # The generator is the published SplitMix64 output function on a counter;
    # the first value for key 0 + GAMMA is the well-known SplitMix64 first
    # output for seed 0.
    z = inputs._fin(np.array([0x9E3779B97F4A7C15], np.uint64))[0]
    assert int(z) == 0xE220A8397B1DCDAF
    a = inputs.int8_uniform(0, inputs.TAG_C, (1000,))
    assert a.min() >= -128 and a.max() <= 127 and a.dtype == np.int8
    assert (a == inputs.int8_uniform(0, inputs.TAG_C, (1000,))).all()
    assert (a[500:] == inputs.int8_uniform(0, inputs.TAG_C, (500,), start=500)).all()
    gi, pos, j, b = inputs.fault_list(1, 10, 100, 3, 50)
    assert len(set(zip(gi.tolist(), pos.tolist()))) == 50
    assert j.max() < 3 and b.max() < 64


# ---- the remaining LSB operators of Eq. 2 ----------------------------------

def test_inner_matches_einsum_and_big_int():
    rng = np.random.default_rng(7)
    for B, S, n in [(1, 1, 1), (2, 3, 17), (3, 4, 256)]:
        x = rng.integers(-(2 ** 30), 2 ** 30, (B, S, n), dtype=np.int64)
        g = rng.integers(-(2 ** 20), 2 ** 20, (B, n), dtype=np.int64)
        assert (oracle.inner(x, g) == np.einsum("bsi,bi->bs", x, g)).all()
    x = np.array([[[2 ** 40, -3, 5]]], np.int64)
    g = np.array([[2 ** 20, 7, -(2 ** 21)]], np.int64)
    assert oracle.inner(x, g).tolist() == [[2 ** 60 - 21 - 5 * 2 ** 21]]
    with pytest.raises(oracle.OracleError):       # a partial sum leaves int64
        oracle.inner(np.array([[[2 ** 62, 2 ** 62]]], np.int64), np.array([[2, -2]], np.int64))


def test_outer_matches_einsum():
    rng = np.random.default_rng(8)
    x = rng.integers(-(2 ** 30), 2 ** 30, (2, 3, 7), dtype=np.int64)
    g = rng.integers(-(2 ** 20), 2 ** 20, (2, 5), dtype=np.int64)
    assert (oracle.outer(x, g) == np.einsum("bsi,bj->bsij", x, g)).all()
    assert oracle.outer(np.array([[[2, -3]]], np.int64), np.array([[5, 7, -1]], np.int64)).tolist() == \
        [[[[10, 14, -2], [-15, -21, 3]]]]


def test_permute_gathers_and_composes():
    rng = np.random.default_rng(9)
    n = 37
    x = rng.integers(-(2 ** 40), 2 ** 40, (2, 3, n), dtype=np.int64)
    p, q = rng.permutation(n), rng.permutation(n)
    assert (oracle.permute(x, p) == x[..., p]).all()
    assert (oracle.permute(x, np.arange(n)) == x).all()
    # gathering by p then by q is gathering by p[q]
    assert (oracle.permute(oracle.permute(x, p), q) == oracle.permute(x, p[q])).all()
    # the inverse permutation undoes it
    assert (oracle.permute(oracle.permute(x, p), np.argsort(p)) == x).all()
    assert oracle.permute(np.array([[[10, 20, 30]]], np.int64), np.array([2, 0, 1])).tolist() == [[[30, 10, 20]]]
    for bad in ([0, 0, 1], [0, 1, 3], [-1, 0, 1]):   # not a bijection of {0, 1, 2}
        with pytest.raises(oracle.OracleError):
            oracle.permute(np.zeros((1, 1, 3), np.int64), np.array(bad))


def test_cxcorr_matches_numpy_correlate_and_brute_force():
    rng = np.random.default_rng(10)
    for N in (1, 2, 5, 64, 129):
        x = rng.integers(-(2 ** 20), 2 ** 20, (2, 2, N), dtype=np.int64)
        g = rng.integers(-128, 128, (2, N)).astype(np.int8)
        y = oracle.cxcorr(x, g)
        for b in range(2):
            for s in range(2):
                # linear correlation of the doubled signal, first N lags
                want = np.correlate(np.concatenate([x[b, s], x[b, s]]), g[b].astype(np.int64), "valid")[:N]
                assert (y[b, s] == want).all()
    # y[i] = sum_j x[(i + j) mod 3] g[j] with g = (1, 0, -1):  y_i = x_i - x_{i+2}
    x = np.array([[[1, 2, 4]]], np.int64)
    assert oracle.cxcorr(x, np.array([[1, 0, -1]], np.int8))[0, 0].tolist() == [1 - 4, 2 - 1, 4 - 2]


def lsb_operand(op, B, n, seed):
    rng = np.random.default_rng(seed)
    if op == "outer":
        return rng.integers(-128, 128, (B, 9), dtype=np.int64)
    if op == "permute":
        return rng.permutation(n)
    if op == "cxcorr":
        return rng.integers(-128, 128, (B, n)).astype(np.int8)
    return rng.integers(-128, 128, (B, n), dtype=np.int64)


@pytest.mark.parametrize("op", oracle.LSB_OPS)
@pytest.mark.parametrize("M,l", [(3, 16), (4, 16), (5, 12)])
def test_lsb_pipeline_equals_direct_flags_and_recovers(op, M, l):
    B, n = 2, 40
    c = inputs.streams(2, (B, M, n))
    g = lsb_operand(op, B, n, M)
    direct = oracle.lsb_direct(op, c, g)
    for r in range(M):
        dh, fl, delta = oracle.lsb_entangled(op, c, g, l, r)
        assert (dh == direct).all() and not fl.any()
        flat = delta.reshape(B, M, -1)
        # Prop. 3: any one stream rebuilt from the others
        assert (oracle.recover(flat, l, (r + 1) % M).reshape(dh.shape) == direct).all()
        # Prop. 4: a bit flip in any one stream is flagged at exactly that position
        bad = flat.copy()
        pos = flat.shape[-1] // 2
        bad[1, (r + 2) % M, pos] ^= np.int64(1) << np.int64(5 + r)
        _, f2 = oracle.extract(bad, l, r)
        assert f2[1, pos] and f2.sum() == 1


# ---- row/column checksum ABFT of a product (ABFT RC-check) -----------------

def test_gemm64_matches_numpy():
    rng = np.random.default_rng(12)
    X = rng.integers(-(2 ** 20), 2 ** 20, (9, 13), dtype=np.int64)
    Y = rng.integers(-(2 ** 20), 2 ** 20, (13, 7), dtype=np.int64)
    assert (oracle.gemm64(X, Y) == X @ Y).all()
    with pytest.raises(oracle.OracleError):
        oracle.gemm64(np.array([[2 ** 40]], np.int64), np.array([[2 ** 30]], np.int64))


def test_rc_full_checksum_matrix_borders_the_product():
    rng = np.random.default_rng(13)
    m, k, n = 17, 23, 11
    A = rng.integers(-128, 128, (m, k), dtype=np.int64)
    B = rng.integers(-128, 128, (k, n)).astype(np.int8)
    ac, br = oracle.rc_encode(A, B)
    assert (ac[:m] == A).all() and (ac[m] == A.sum(0)).all()
    assert (br[:, :n] == B).all() and (br[:, n] == B.astype(np.int64).sum(1)).all()
    Cf = oracle.rc_full(A, B)
    C = A @ B.astype(np.int64)
    assert (Cf[:m, :n] == C).all()
    assert (Cf[:m, n] == C.sum(1)).all() and (Cf[m, :n] == C.sum(0)).all() and Cf[m, n] == C.sum()
    rb, cb = oracle.rc_check(Cf)
    assert not rb.any() and not cb.any()


def test_rc_single_error_is_located_and_corrected_anywhere():
    rng = np.random.default_rng(14)
    m, k, n = 6, 9, 5
    A = rng.integers(-128, 128, (m, k), dtype=np.int64)
    B = rng.integers(-128, 128, (k, n)).astype(np.int8)
    Cf = oracle.rc_full(A, B)
    for i in range(m + 1):
        for j in range(n + 1):
            bad = Cf.copy()
            bad[i, j] ^= np.int64(1) << np.int64((3 * i + j) % 60)
            rb, cb = oracle.rc_check(bad)
            assert np.flatnonzero(rb).tolist() == [i] and np.flatnonzero(cb).tolist() == [j]
            fixed, done = oracle.rc_correct(bad)
            assert done and (fixed == Cf).all()


def test_rc_two_errors_are_detected_not_corrected():
    rng = np.random.default_rng(15)
    A = rng.integers(-128, 128, (8, 8), dtype=np.int64)
    B = rng.integers(-128, 128, (8, 8)).astype(np.int8)
    Cf = oracle.rc_full(A, B)
    bad = Cf.copy()
    bad[1, 2] += 5
    bad[4, 6] -= 3
    rb, cb = oracle.rc_check(bad)
    assert np.flatnonzero(rb).tolist() == [1, 4] and np.flatnonzero(cb).tolist() == [2, 6]
    fixed, done = oracle.rc_correct(bad)
    assert not done and (fixed == bad).all()


def test_cconv_at_equals_full_cconv_at_every_requested_output():
    rng = np.random.default_rng(16)
    B, S, N = 3, 2, 37
    x = rng.integers(-(2 ** 20), 2 ** 20, (B, S, N), dtype=np.int64)
    g = rng.integers(-128, 128, (B, N)).astype(np.int8)
    full = oracle.cconv(x, g)
    sig = rng.integers(0, B * S, 50)
    pos = rng.integers(0, N, 50)
    assert (oracle.cconv_at(x, g, sig, pos) == full.reshape(B * S, N)[sig, pos]).all()
    # y[0] of a delta signal is the filter's first entry
    e = np.zeros((1, 1, 8), np.int64)
    e[0, 0, 0] = 1
    gg = np.arange(8, dtype=np.int8).reshape(1, 8)
    assert oracle.cconv_at(e, gg, [0, 0], [0, 5]).tolist() == [0, 5]


# ---- linear convolution of long streams (Sec. IV-A blocking, Sec. V second experiment) ----

def test_lconv_matches_numpy_convolve_and_brute_force():
    rng = np.random.default_rng(31)
    for n, K in [(1, 1), (5, 1), (1, 7), (37, 5), (200, 64), (1000, 129), (300, 450)]:
        x = rng.integers(-(2 ** 30), 2 ** 30, (2, 3, n), dtype=np.int64)
        g = rng.integers(-128, 128, (2, K)).astype(np.int8)
        y = oracle.lconv(x, g)
        assert y.shape == (2, 3, n + K - 1)
        for b in range(2):
            for s in range(3):
                assert (y[b, s] == np.convolve(x[b, s], g[b].astype(np.int64))).all()
        if n * K <= 400:     # the definition on Python integers
            for b in range(2):
                for i in range(n + K - 1):
                    want = sum(int(g[b, t]) * int(x[b, 0, i - t]) for t in range(K) if 0 <= i - t < n)
                    assert int(y[b, 0, i]) == want


def test_lconv_is_a_zero_padded_circular_convolution_and_blocks_overlap_save():
    # (i) the full linear convolution is the circular convolution of length
    # L >= n + K - 1 of the zero-padded stream and kernel; (ii) overlap-save:
    # blocks of L inputs that overlap by K - 1, each convolved circularly,
    # reproduce the outputs from their position K - 1 on (Sec. IV-A)
    rng = np.random.default_rng(32)
    n, K, L = 500, 40, 128
    x = rng.integers(-(2 ** 20), 2 ** 20, (1, 2, n), dtype=np.int64)
    g = rng.integers(-128, 128, (1, K)).astype(np.int8)
    y = oracle.lconv(x, g)
    Lf = n + K - 1
    xp = np.zeros((1, 2, Lf), np.int64)
    xp[..., :n] = x
    gp = np.zeros((1, Lf), np.int8)
    gp[:, :K] = g
    assert (oracle.cconv(xp, gp) == y).all()
    B = L - K + 1
    gL = np.zeros((1, L), np.int8)
    gL[:, :K] = g
    out = np.zeros_like(y)
    for j0 in range(0, Lf, B):
        seg = np.zeros((1, 2, L), np.int64)
        lo = j0 - (K - 1)
        for q in range(L):
            if 0 <= lo + q < n:
                seg[..., q] = x[..., lo + q]
        blk = oracle.cconv(seg, gL)
        take = min(B, Lf - j0)
        out[..., j0:j0 + take] = blk[..., K - 1:K - 1 + take]
    assert (out == y).all()


@pytest.mark.parametrize("M,l", [(3, 16), (4, 16), (8, 8)])
def test_lconv_pipeline_equals_direct_flags_and_recovers(M, l):
    rng = np.random.default_rng(33 + M)
    n, K = 700, 90
    c = rng.integers(-128, 128, (2, M, n)).astype(np.int32)
    g = rng.integers(-128, 128, (2, K)).astype(np.int8)
    direct = oracle.lconv_direct(c, g)
    dhat, flags, delta = oracle.lconv_entangled(c, g, l, r=M - 1)
    assert (dhat == direct).all() and not flags.any()
    bad = delta.copy()
    bad[1, 2, 333] ^= np.int64(1 << 37)
    _, f = oracle.extract(bad, l, 0)
    assert f.sum() == 1 and f[1, 333] == 1
    assert (oracle.recover(bad, l, 2) == direct).all()


def test_lconv_at_equals_full_lconv_at_every_requested_output():
    rng = np.random.default_rng(34)
    n, K = 400, 77
    x = rng.integers(-(2 ** 30), 2 ** 30, (3, 2, n), dtype=np.int64)
    g = rng.integers(-128, 128, (3, K)).astype(np.int8)
    y = oracle.lconv(x, g)
    sig = rng.integers(0, 6, 300)
    pos = rng.integers(0, n + K - 1, 300)
    pos[:3] = [0, n + K - 2, n - 1]
    got = oracle.lconv_at(x, g, sig, pos)
    assert (got == y.reshape(6, -1)[sig, pos]).all()
