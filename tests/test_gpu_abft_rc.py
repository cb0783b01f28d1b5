"""GPU parity of the row/column checksum ABFT comparator (ABFT RC-check of
Sec. V) against the CPU oracle, bit-exact: the encoding, the border of the
full-checksum matrix, the row/column flags on clean data, single-error
location and correction, and detection without correction of two errors."""
import numpy as np
import pytest

import oracle
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


def case(batch, m, k, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-128, 128, (batch, m, k)).astype(np.int32)
    B = rng.integers(-128, 128, (k, n)).astype(np.int8)
    C = np.stack([A[b].astype(np.int64) @ B.astype(np.int64) for b in range(batch)])
    return A, B, C


@pytest.mark.parametrize("batch,m,k,n", [(3, 37, 50, 29), (2, 300, 700, 260), (1, 1, 1, 1), (4, 64, 64, 256)])
def test_rc_check_and_correct_match_oracle(ne, batch, m, k, n):
    A, B, C = case(batch, m, k, n, m + k + n)
    Ad, Bd, Cd = dev(A), dev(B), dev(C)
    ac, br = ne.ne_abft_rc_encode(Ad, Bd)
    full = [oracle.rc_full(A[b].astype(np.int64), B) for b in range(batch)]
    for b in range(batch):
        want_ac, want_br = oracle.rc_encode(A[b].astype(np.int64), B)
        assert (host(ac)[b] == want_ac[m]).all()
        assert (host(br) == want_br[:, n]).all()
    nbad = torch.full((2,), 9, dtype=torch.int64, device=DEV)
    work, rb, cb = ne.ne_abft_rc_check(Cd, Ad, Bd, ac, br, nbad=nbad)
    w = host(work)
    for b in range(batch):
        Cf = full[b]
        assert (w[b, :m] == Cf[:m, n]).all() and (w[b, m:m + n] == Cf[m, :n]).all() and w[b, m + n] == Cf[m, n]
        assert (w[b, m + n + 1:m + n + 1 + m] == C[b].sum(1)).all()
        assert (w[b, 2 * m + n + 1:2 * m + 2 * n + 1] == C[b].sum(0)).all()
    assert not unpack_flags(host(rb), batch, m + 1).any() and not unpack_flags(host(cb), batch, n + 1).any()
    assert host(nbad).tolist() == [0, 0]
    # one fault per product: located exactly where the oracle locates it, then corrected
    rng = np.random.default_rng(7)
    bad = C.copy()
    pos = [(int(rng.integers(m)), int(rng.integers(n))) for _ in range(batch)]
    for b, (i, j) in enumerate(pos):
        bad[b, i, j] ^= np.int64(1) << np.int64(int(rng.integers(0, 62)))
    Cd = dev(bad)
    work, rb, cb = ne.ne_abft_rc_check(Cd, Ad, Bd, ac, br, nbad=nbad)
    grb, gcb = unpack_flags(host(rb), batch, m + 1), unpack_flags(host(cb), batch, n + 1)
    for b, (i, j) in enumerate(pos):
        Cf = full[b].copy()
        Cf[i, j] = bad[b, i, j]
        orb, ocb = oracle.rc_check(Cf)
        assert (grb[b] == orb).all() and (gcb[b] == ocb).all()
        assert np.flatnonzero(orb).tolist() == [i] and np.flatnonzero(ocb).tolist() == [j]
    assert host(nbad).tolist() == [batch, batch]
    ncor = torch.zeros(1, dtype=torch.int64, device=DEV)
    ne.ne_abft_rc_correct(Cd, work, rb, cb, ncor)
    assert (host(Cd) == C).all() and int(ncor.item()) == batch


def test_rc_two_errors_detected_not_corrected(ne):
    batch, m, k, n = 2, 40, 33, 70
    A, B, C = case(batch, m, k, n, 99)
    Ad, Bd = dev(A), dev(B)
    ac, br = ne.ne_abft_rc_encode(Ad, Bd)
    bad = C.copy()
    bad[1, 3, 5] += 1000
    bad[1, 17, 60] -= 7
    Cd = dev(bad)
    work, rb, cb = ne.ne_abft_rc_check(Cd, Ad, Bd, ac, br)
    grb, gcb = unpack_flags(host(rb), batch, m + 1), unpack_flags(host(cb), batch, n + 1)
    assert not grb[0].any() and not gcb[0].any()
    assert np.flatnonzero(grb[1]).tolist() == [3, 17] and np.flatnonzero(gcb[1]).tolist() == [5, 60]
    ncor = torch.zeros(1, dtype=torch.int64, device=DEV)
    ne.ne_abft_rc_correct(Cd, work, rb, cb, ncor)
    assert (host(Cd) == bad).all() and int(ncor.item()) == 0

