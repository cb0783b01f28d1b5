"""Pins for the oracle's parameter choice (Eq. 13, Eq. 14, Table II)."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_w32.txt")


def _table2():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    return rows


@pytest.mark.parametrize("row", _table2())
def test_table2_paper_rule(row):
    # Table II: l, k and the two bitwidth columns at w = 32.
    M, l, k, bw_prop, bw_abft = row
    assert oracle.choose_l(M, 32, 0, oracle.POLICY_PAPER) == (l, k)
    assert (M - 2) * l + k == bw_prop
    assert 32 - math.ceil(math.log2(M)) == bw_abft


def test_m3_w32_instance():
    # Sec. III-A: "w = 32, l = 11 and k = 10" for M = 3, and Eq. 8 is tight.
    l, k = oracle.choose_l(3, 32, 0, oracle.POLICY_PAPER)
    assert (l, k) == (11, 10) and 2 * l + k == 32


@pytest.mark.parametrize("w", [32, 64])
def test_m4_k_equals_l_equals_w_over_4(w):
    # Caption of Fig. 5: for M = 4 and w in {32, 64}, k = l = w / 4.
    assert oracle.choose_l(4, w, 0, oracle.POLICY_PAPER) == (w // 4, w // 4)


def test_eq14_closed_form_values():
    # Hand-evaluated Eq. 14: 2^((M-3)l+k) (2^(l-1) - 1)
    assert oracle.range_eq14(3, 11, 10) == 2 ** 10 * 1023           # 1047552
    assert oracle.range_eq14(4, 8, 8) == 65536 * 127                 # 8323072
    assert oracle.range_eq14(5, 7, 4) == 2 ** 18 * 63
    assert oracle.range_eq14(3, 40, 40) == -1                        # >= 2^63


def _extract_exact_at(M, l, B):
    """Brute consequence check: outputs at the corners of [-B, B]^M survive the
    whole encode/extract round trip for every unused stream r."""
    corners = np.array(np.meshgrid(*([[-B, B, 0, B - 1]] * M), indexing="ij")).reshape(M, -1)
    d = corners.astype(object)
    delta = np.array([[int(d[m, i]) + (int(d[(m - 1) % M, i]) << l) for i in range(d.shape[1])]
                      for m in range(M)], dtype=object)
    if any(abs(int(v)) >= 2 ** 63 for v in delta.ravel()):
        return False
    for r in range(M):
        dh, fl = oracle.extract(delta.astype(np.int64), l, r)
        if not (dh == corners).all() or fl.any():
            return False
    return True


@pytest.mark.parametrize("M,B", [(3, 64 * 2 ** 14), (3, 1024 * 2 ** 14), (4, 4096 * 2 ** 14),
                                 (5, 2048 * 2 ** 14), (3, 2 ** 16 * 2 ** 14)])
@pytest.mark.parametrize("policy", [oracle.POLICY_SMALLEST, oracle.POLICY_BYTE])
def test_bound_policies_are_sufficient_and_eq14_minimal(M, B, policy):
    l, k = oracle.choose_l(M, 64, B, policy)
    # Eq. 13 and k <= l
    assert (M - 1) * l + k <= 64 and 1 <= k <= l
    # Eq. 14 covers the bound ...
    assert oracle.range_eq14(M, l, k) >= B
    # ... and the round trip is exact at the extreme outputs
    assert _extract_exact_at(M, l, B)
    if policy == oracle.POLICY_BYTE:
        assert l % 8 == 0
    else:
        # no smaller l has any admissible k whose Eq. 14 range covers B
        for l2 in range(1, l):
            for k2 in range(1, l2 + 1):
                if (M - 1) * l2 + k2 <= 64:
                    D = oracle.range_eq14(M, l2, k2)
                    assert 0 <= D < B


def test_tight_l_of_the_configured_workloads():
    # |c| <= 128, |g| <= 128: the output bound is K * 2^14.
    assert oracle.choose_l(3, 64, 64 * 2 ** 14, oracle.POLICY_SMALLEST)[0] == 11
    assert oracle.choose_l(3, 64, 1024 * 2 ** 14, oracle.POLICY_SMALLEST)[0] == 13
    assert oracle.choose_l(4, 64, 4096 * 2 ** 14, oracle.POLICY_SMALLEST)[0] == 10
