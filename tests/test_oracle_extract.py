"""Pins for the oracle's entanglement, extraction, check and recovery.

Each pin is independent of the oracle's own code: the M = 3 equations of the
paper written out as printed (Eq. 7, Eq. 11, Eq. 23), the circulant-matrix
form of Eq. 15-16, exhaustive enumeration of small codes, the invariants of
Prop. 1-4 and the two-fault escape the proofs of Prop. 2 and 4 allow.
"""
import itertools

import numpy as np
import pytest

import oracle


def sl(x, s):
    """S_s{x} on Python integers (Eq. 9): x << s for s >= 0, floor shift else."""
    return x << s if s >= 0 else x >> (-s)     # Python >> on ints is floor division


# ---- entanglement ------------------------------------------------------------

def test_entangle_m3_as_printed():
    # Eq. 7, three statements as printed.
    rng = np.random.default_rng(1)
    for l in (1, 11, 22, 31):
        c = rng.integers(-(2 ** 30), 2 ** 30, (3, 50)).astype(np.int32)
        eps = oracle.entangle(c, l)
        for n in range(50):
            c0, c1, c2 = (int(c[m, n]) for m in range(3))
            assert eps[0, n] == sl(c2, l) + c0
            assert eps[1, n] == sl(c0, l) + c1
            assert eps[2, n] == sl(c1, l) + c2


@pytest.mark.parametrize("M", [3, 4, 5, 8])
def test_entangle_matches_circulant_operator(M):
    # Eq. 15-16: eps = E c, E the M x M circulant of [1 0 ... 0 S_l].
    l = 7
    E = np.zeros((M, M), dtype=object)
    first_row = [1] + [0] * (M - 2) + [2 ** l]
    for i in range(M):
        for j in range(M):
            E[i, j] = first_row[(j - i) % M]
    rng = np.random.default_rng(M)
    c = rng.integers(-1000, 1000, (M, 40)).astype(np.int32)
    want = E.dot(c.astype(object))
    assert (oracle.entangle(c, l) == want.astype(np.int64)).all()


def test_entangle_overflow_is_reported():
    c = np.full((3, 4), 2 ** 31 - 1, np.int32)
    with pytest.raises(oracle.OracleError):
        oracle.entangle(c, 40)


# ---- the M = 3 disentanglement exactly as printed ----------------------------

def eq11_and_eq23(delta0, delta1, delta2, l):
    """Eq. 11 (r = 0) and the check of Eq. 23, on Python integers."""
    dtemp = delta2 - sl(delta1, l)
    P = 1 << (2 * l)
    d2 = ((dtemp % P) + (P >> 1)) % P - (P >> 1)   # S_{-2(w-l)}{S_{2(w-l)}{dtemp}}
    d0 = sl(-(dtemp - d2), -2 * l)
    d1 = delta1 - sl(d0, l)
    flag = (delta0 - (sl(d2, l) + d0)) != 0
    return d0, d1, d2, flag


def wrap64(x):
    return ((x + 2 ** 63) % 2 ** 64) - 2 ** 63


@pytest.mark.parametrize("l", [3, 11, 13, 16, 22, 31])
def test_general_extract_reduces_to_eq11_at_m3(l):
    rng = np.random.default_rng(l)
    n = 400
    # half valid codewords, half arbitrary 64-bit words (corrupted data)
    lim = 2 ** (2 * l - 1) - 1
    d = rng.integers(-lim, lim + 1, (3, n // 2), dtype=np.int64)
    valid = np.stack([d[m] + (d[(m - 1) % 3] << l) for m in range(3)]) if 3 * l < 62 else None
    if valid is None:
        valid = rng.integers(-(2 ** 40), 2 ** 40, (3, n // 2), dtype=np.int64)
    junk = rng.integers(-(2 ** 63), 2 ** 63 - 1, (3, n // 2), dtype=np.int64)
    delta = np.concatenate([valid, junk], axis=1)
    dh, fl = oracle.extract(delta, l, 0)
    for i in range(n):
        d0, d1, d2, f = eq11_and_eq23(*(int(delta[m, i]) for m in range(3)), l)
        assert (int(dh[0, i]), int(dh[1, i]), int(dh[2, i])) == (wrap64(d0), wrap64(d1), wrap64(d2))
        assert bool(fl[i]) == f


def test_worked_example_m3_l4():
    # Hand-evaluated: c = (3, -2, 5), l = 4, op = x with g = 1 (Sec. II: the
    # streams "left in their native state").
    # Eq. 7:  eps0 = 16*5 + 3 = 83, eps1 = 16*3 - 2 = 46, eps2 = 16*(-2) + 5 = -27
    eps = oracle.entangle(np.array([[3], [-2], [5]], np.int32), 4)
    assert eps[:, 0].tolist() == [83, 46, -27]
    # Eq. 11: dtemp = -27 - 16*46 = -763; low 8 bits sign-extended = 5 = d2;
    #         d0 = -(-763 - 5) >> 8 = 3; d1 = 46 - 16*3 = -2.  Eq. 23: 83 - (80 + 3) = 0.
    dh, fl = oracle.extract(eps, 4, 0)
    assert dh[:, 0].tolist() == [3, -2, 5] and fl[0] == 0


# ---- exhaustive round trip, check and recovery -------------------------------

def _all_codes(M, l):
    lim = 2 ** ((M - 1) * l - 1) - 1
    vals = np.arange(-lim, lim + 1, dtype=np.int64)
    d = np.array(np.meshgrid(*([vals] * M), indexing="ij")).reshape(M, -1)
    delta = np.stack([d[m] + (d[(m - 1) % M] << l) for m in range(M)])
    return d, delta


@pytest.mark.parametrize("M,l", [(3, 1), (3, 2), (3, 3), (4, 1), (5, 1), (4, 2)])
def test_exhaustive_round_trip_every_r(M, l):
    # Prop. 3: every code in the exact range decodes from any M-1 streams.
    d, delta = _all_codes(M, l)
    if d.shape[1] > 300000:
        idx = np.random.default_rng(0).choice(d.shape[1], 300000, replace=False)
        d, delta = d[:, idx], delta[:, idx]
    for r in range(M):
        dh, fl = oracle.extract(delta, l, r)
        assert (dh == d).all()
        assert not fl.any()
        # fail-stop: plane r replaced by garbage is never read
        poisoned = delta.copy()
        poisoned[r] = np.int64(-0x5A5A5A5A5A5A5A5A)
        assert (oracle.recover(poisoned, l, r) == d).all()


@pytest.mark.parametrize("M,l", [(3, 2), (4, 1), (3, 5), (5, 2), (8, 3)])
def test_every_single_bit_flip_is_flagged(M, l):
    # Prop. 2 / Prop. 4: any fault confined to one stream of a position is
    # detected.  Every stream, every one of the 64 bits, every r.
    d, delta = _all_codes(M, l) if (M, l) in [(3, 2), (4, 1)] else (None, None)
    if delta is None:
        rng = np.random.default_rng(M * 100 + l)
        lim = 2 ** ((M - 1) * l - 1) - 1
        d = rng.integers(-lim, lim + 1, (M, 300), dtype=np.int64)
        delta = np.stack([d[m] + (d[(m - 1) % M] << l) for m in range(M)])
    n = delta.shape[1]
    cols = []
    for j, b in itertools.product(range(M), range(64)):
        x = delta.copy()
        x[j] ^= np.int64(np.uint64(1 << b).view(np.int64))
        cols.append(x)
    big = np.concatenate(cols, axis=1)
    for r in range(M):
        _, fl = oracle.extract(big, l, r)
        assert fl.all(), f"undetected single-bit flip (M={M}, l={l}, r={r})"
    assert big.shape[1] == n * M * 64


@pytest.mark.parametrize("M,l", [(3, 11), (4, 10), (5, 8)])
def test_two_colocated_faults_can_escape(M, l):
    # The proofs of Prop. 2 and 4 guarantee detection only for a single faulty
    # stream: delta_j += t together with delta_{j+1} += 2^l t is the code of
    # d_j + t, so the check passes and d_j silently moves by t.
    rng = np.random.default_rng(7)
    lim = 2 ** ((M - 1) * l - 2)
    d = rng.integers(-lim, lim, (M, 64), dtype=np.int64)
    delta = np.stack([d[m] + (d[(m - 1) % M] << l) for m in range(M)])
    j, t = 1, 12345
    delta[j] += t
    delta[(j + 1) % M] += t << l
    for r in range(M):
        dh, fl = oracle.extract(delta, l, r)
        assert not fl.any()
        want = d.copy()
        want[j] += t
        assert (dh == want).all()


def test_extract_of_random_words_never_overflows_128_bits():
    # Any 64-bit corruption stays representable in the 2w-bit temporaries.
    rng = np.random.default_rng(3)
    for M, l in [(3, 21), (3, 31), (4, 20), (5, 15), (8, 9), (16, 4), (32, 2)]:
        delta = rng.integers(-(2 ** 63), 2 ** 63 - 1, (M, 200), dtype=np.int64, endpoint=True)
        delta[:, :4] = np.int64(-(2 ** 63))
        delta[:, 4:8] = np.int64(2 ** 63 - 1)
        for r in range(M):
            oracle.extract(delta, l, r)            # raises on any overflow
