"""CPU tests of the C ABI: the library builds and loads, exports every symbol
include/ne.h declares, and its host-side logic (planning, argument checks)
behaves as documented.  No device computation runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04740_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ne_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in include/ but not exported"


def test_measurement_probes_live_outside_the_library_abi(lib):
    from paper_1604_04740_gb300 import build
    src = open(os.path.join(build.PROBE, "ne_probe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    probes = set(re.findall(r"\b(ne_probe_[a-z0-9_]+)\s*\(", src))
    assert len(probes) == 4
    plib = ctypes.CDLL(build.PROBE_LIB)
    for s in probes:
        assert hasattr(plib, s), s
        assert not hasattr(lib, s), f"{s} is exported by the library"
        assert s not in declared_symbols()


def _choose(lib, M, w, B, policy):
    l, k = ctypes.c_int32(), ctypes.c_int32()
    st = lib.ne_choose_l(M, w, ctypes.c_int64(B), policy, ctypes.byref(l), ctypes.byref(k))
    return st, l.value, k.value


@pytest.mark.parametrize("M", [3, 4, 5, 8, 11, 16, 32])
@pytest.mark.parametrize("w", [32, 64])
def test_choose_l_agrees_with_oracle(lib, M, w):
    for policy, B in [(0, 0), (1, 2 ** 20), (1, 2 ** 26), (2, 2 ** 24)]:
        st, l, k = _choose(lib, M, w, B, policy)
        try:
            want = oracle.choose_l(M, w, B, policy)
        except oracle.OracleError:
            assert st == 2
            continue
        assert st == 0 and (l, k) == want


class Digits(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("shift", ctypes.c_int32 * 8), ("l", ctypes.c_int32),
                ("lo", ctypes.c_int32), ("hi", ctypes.c_int32)]


def _brute_digits(l, lo, hi):
    used = set()
    for a in range(lo, hi + 1):
        for b in range(lo, hi + 1):
            x = a + (b << l)
            t = 0
            while x != 0:
                d = ((x + 128) % 256) - 128
                if d:
                    used.add(8 * t)
                x = (x - d) // 256
                t += 1
    return sorted(used) or [0]


@pytest.mark.parametrize("l,lo,hi", [(16, -128, 127), (13, -128, 127), (8, -128, 127), (11, -20, 20),
                                     (24, -128, 127), (16, -128, 128), (10, 0, 255)])
def test_plan_digits_matches_brute_force(lib, l, lo, hi):
    d = Digits()
    assert lib.ne_plan_digits(l, lo, hi, ctypes.byref(d)) == 0
    assert [d.shift[i] for i in range(d.S)] == _brute_digits(l, lo, hi)
    assert (d.l, d.lo, d.hi) == (l, lo, hi)


def test_byte_aligned_l_gives_two_digits_for_int8_streams(lib):
    d = Digits()
    assert lib.ne_plan_digits(16, -128, 127, ctypes.byref(d)) == 0
    assert (d.S, d.shift[0], d.shift[1]) == (2, 0, 16)


class Params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("l", ctypes.c_int32), ("w", ctypes.c_int32)]


def test_host_argument_checks_reject_before_any_launch(lib):
    lib.ne_last_error.restype = ctypes.c_char_p
    P = ctypes.c_void_p
    lib.ne_entangle.argtypes = [Params, P, P, ctypes.c_int64, ctypes.c_int64, P]
    lib.ne_extract.argtypes = [Params, P, P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, P, P, P]
    fake = ctypes.c_void_p(0x1000)
    # M < 3
    assert lib.ne_entangle(Params(2, 5, 64), fake, fake, 1, 8, None) == 1
    # w != 64
    assert lib.ne_entangle(Params(3, 5, 32), fake, fake, 1, 8, None) == 1
    # Eq. 13 violated: (M-1) l = 64
    assert lib.ne_entangle(Params(3, 32, 64), fake, fake, 1, 8, None) == 2
    assert b"Eq. 13" in lib.ne_last_error()
    # r out of range
    assert lib.ne_extract(Params(3, 11, 64), fake, fake, 1, 8, 3, None, None, None) == 1
    # null pointer
    assert lib.ne_entangle(Params(3, 11, 64), None, fake, 1, 8, None) == 1
    # empty problem is a no-op
    assert lib.ne_entangle(Params(3, 11, 64), None, None, 0, 0, None) == 0


def test_lsb_operator_argument_checks(lib):
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.ne_elementwise.argtypes = [Params, i32, P, P, i64, P, P, P, i64, i64, i32, i32, P]
    lib.ne_outer.argtypes = [Params, P, P, i64, P, P, P, i64, i64, i64, i32, i32, P]
    lib.ne_permute.argtypes = [Params, P, P, P, P, P, i64, i64, i32, i32, P, P]
    lib.ne_inner.argtypes = [Params, P, P, i64, P, P, P, i64, i64, i32, i32, P]
    lib.ne_entangle_kernel_self.argtypes = [i32, P, P, i64, P]
    lib.ne_reverse_operand.argtypes = [P, P, i64, i64, P]
    fake = ctypes.c_void_p(0x1000)
    ok = Params(3, 16, 64)
    # unknown operator, negative operand stride, unknown epilogue, r out of range
    assert lib.ne_elementwise(ok, 3, fake, fake, 0, fake, None, None, 1, 8, 0, 0, None) == 1
    assert lib.ne_elementwise(ok, 0, fake, fake, -1, fake, None, None, 1, 8, 0, 0, None) == 1
    assert lib.ne_elementwise(ok, 0, fake, fake, 0, fake, None, None, 1, 8, 7, 0, None) == 1
    assert lib.ne_elementwise(ok, 0, fake, fake, 0, fake, None, None, 1, 8, 1, 3, None) == 1
    # Eq. 13 still applies
    assert lib.ne_inner(Params(3, 32, 64), fake, fake, 0, fake, None, None, 1, 8, 0, 0, None) == 2
    # null operand / index set
    assert lib.ne_outer(ok, fake, None, 0, fake, None, None, 1, 8, 4, 0, 0, None) == 1
    assert lib.ne_permute(ok, fake, None, fake, None, None, 1, 8, 0, 0, None, None) == 1
    # n * k beyond the supported output size
    assert lib.ne_outer(ok, fake, fake, 0, fake, None, None, 1, 1 << 30, 1 << 30, 0, 0, None) == 1
    # operand preparations: bad l, aliasing
    assert lib.ne_entangle_kernel_self(0, fake, fake, 8, None) == 1
    assert lib.ne_reverse_operand(fake, fake, 1, 8, None) == 1
    # empty problems are no-ops
    assert lib.ne_elementwise(ok, 0, None, None, 0, None, None, None, 0, 0, 0, 0, None) == 0
    assert lib.ne_inner(ok, None, None, 0, None, None, None, 0, 0, 0, 0, None) == 0


def test_cconv_split_accepts_exactly_the_documented_variants(lib):
    # ne.h lists the tensor / dp4a splits: -1 (default), 0 (tensor pipe only),
    # HR = 8 tensor warps and H dp4a warps of R outputs per thread, and 4HR the
    # same with 4 tensor warps; anything else is refused
    lib.ne_set_cconv_split.argtypes = [ctypes.c_int32]
    header = re.sub(r"\s*\n\s*\*\s*", " ", open(os.path.join(ROOT, "include", "ne.h")).read())
    hr = re.search(r"HR in \{([0-9, ]+)\}", header)
    twhr = re.search(r"4HR in \{([0-9, ]+)\}", header)
    assert hr and twhr, "ne.h documents the accepted splits"
    documented = {int(v) for v in hr.group(1).split(",")} | {int(v) for v in twhr.group(1).split(",")}
    try:
        for v in sorted(documented | {-1, 0}):
            assert lib.ne_set_cconv_split(v) == 0, v
        for v in range(-3, 500):
            if v not in documented | {-1, 0}:
                assert lib.ne_set_cconv_split(v) == 1, v
        # every accepted code puts whole 64-output blocks on the dp4a warps and
        # keeps a CTA of 32 (TW + H) threads within 384
        for v in documented:
            TW = 4 if v >= 100 else 8
            H, R = divmod(v % 100, 10)
            assert (32 * H * R) % 64 == 0 and 2 <= R <= 4 and 32 * (TW + H) <= 384, v
    finally:
        assert lib.ne_set_cconv_split(-1) == 0
