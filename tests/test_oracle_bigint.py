"""Pins for the oracle's outputs at flagged positions for general M.

On corrupted words the outputs are defined by Eq. 17-20 with the chosen
unused stream r (their low 64 bits) and the flag by Eq. 24.  Two pins that do
not go through the oracle's C code:

1. Eq. 17-20 and Eq. 24 restated on unbounded Python integers (no 128-bit
   temporaries, true floor division, low 64 bits taken only at the end), on
   random 64-bit words for M in {4, 5, 8} and every r.
2. Structure every output of Eq. 17-20 has, whatever the input words:
   re-entangling the outputs (Eq. 16, wrapping 64-bit) reproduces every input
   word but delta_r; d_{r-1} lies in the sign-extension range of (M-1) l
   bits; the flag is set exactly when delta_r differs from d_r + 2^l d_{r-1};
   and a single-word error on a codeword is flagged (Prop. 4).
"""
import numpy as np
import pytest

import oracle


def wrap64(x):
    return ((x + 2 ** 63) % 2 ** 64) - 2 ** 63


def extract_bigint(delta, M, l, r):
    """Eq. 17-20 and Eq. 24 on Python integers for one position.
    delta: M ints.  Returns (outputs as wrapped int64, flag)."""
    L = (M - 1) * l
    # Eq. 17 with the (-1)^M factor (the reading that reduces to Eq. 11 at M = 3)
    T = 0
    for m in range(M - 1):
        T += (-1) ** m * 2 ** ((M - 2 - m) * l) * delta[(r + 1 + m) % M]
    T *= (-1) ** M
    # Eq. 18: the low L bits of T, sign-extended
    low = T % 2 ** L
    d_prev = low - 2 ** L if low >= 2 ** (L - 1) else low
    # Eq. 19 (index r - 1 in place of the r = 0 case's M - 1): an exact division
    num = (-1) ** M * (T - d_prev)
    assert num % 2 ** L == 0
    d_r = num // 2 ** L
    d = [None] * M
    d[r] = d_r
    d[(r - 1) % M] = d_prev
    # Eq. 20, m = 1 .. M - 2
    prev = d_r
    for m in range(1, M - 1):
        cur = delta[(r + m) % M] - 2 ** l * prev
        d[(r + m) % M] = cur
        prev = cur
    # Eq. 24
    flag = delta[r] != d_r + 2 ** l * d_prev
    return [wrap64(v) for v in d], flag


def random_words(rng, M, n):
    """n arbitrary 64-bit words per stream (the worst kind of corruption)."""
    return rng.integers(-(2 ** 63), 2 ** 63 - 1, (M, n), dtype=np.int64, endpoint=True)


CASES = [(4, 8), (4, 16), (4, 21), (5, 8), (5, 13), (8, 4), (8, 9)]


@pytest.mark.parametrize("M,l", CASES)
def test_oracle_outputs_on_arbitrary_words_match_bigint_restatement(M, l):
    rng = np.random.default_rng(1000 * M + l)
    n = 64
    delta = random_words(rng, M, n)
    for r in range(M):
        dhat, flags = oracle.extract(delta, l, r)
        for i in range(n):
            col = [int(delta[m, i]) for m in range(M)]
            want, fl = extract_bigint(col, M, l, r)
            assert [int(dhat[m, i]) for m in range(M)] == want, (M, l, r, i)
            assert bool(flags[i]) == fl


@pytest.mark.parametrize("M,l", CASES)
def test_oracle_outputs_have_the_structure_of_eq17_to_20(M, l):
    rng = np.random.default_rng(77 * M + l)
    n = 200
    delta = random_words(rng, M, n)
    L = (M - 1) * l
    for r in range(M):
        dhat, flags = oracle.extract(delta, l, r)
        for i in range(n):
            d = [int(dhat[m, i]) for m in range(M)]
            dl = [int(delta[m, i]) for m in range(M)]
            # every stream but r is re-entangled exactly (mod 2^64)
            for m in range(M):
                if m != r:
                    assert wrap64(d[m] + 2 ** l * d[(m - 1) % M]) == dl[m], (M, l, r, m, i)
            # d_{r-1} is a sign-extended L-bit value
            assert -(2 ** (L - 1)) <= d[(r - 1) % M] < 2 ** (L - 1)
            # the flag compares delta_r with the untruncated d_r + 2^l d_{r-1};
            # d_r is exact in 64 bits (|d_r| < 2^(64 - l))
            assert abs(d[r]) < 2 ** (64 - l)
            assert bool(flags[i]) == (dl[r] != d[r] + 2 ** l * d[(r - 1) % M])


@pytest.mark.parametrize("M,l", [(4, 16), (5, 8), (8, 5)])
def test_single_word_errors_on_codewords_are_flagged_for_every_r(M, l):
    # Prop. 4 on the oracle with random in-range outputs and a random error
    # (not a single bit) added to one stream
    rng = np.random.default_rng(5 * M + l)
    L = (M - 1) * l
    lim = 2 ** (L - 1) - 1
    lim = min(lim, (2 ** 62) // (2 ** l + 1))
    n = 300
    d = rng.integers(-lim, lim + 1, (M, n), dtype=np.int64)
    # delta_m = d_m + 2^l d_{m-1}: Eq. 16 applied to outputs (linearity, Eq. 10)
    delta = np.empty_like(d)
    for m in range(M):
        delta[m] = [int(d[m, i]) + 2 ** l * int(d[(m - 1) % M, i]) for i in range(n)]
    j = rng.integers(0, M, n)
    e = rng.integers(1, 2 ** 40, n) * rng.choice([-1, 1], n)
    bad = delta.copy()
    bad[j, np.arange(n)] += e
    for r in range(M):
        dhat, flags = oracle.extract(delta, l, r)
        assert (dhat == d).all() and not flags.any()
        _, flags = oracle.extract(bad, l, r)
        assert flags.all(), (M, l, r)
