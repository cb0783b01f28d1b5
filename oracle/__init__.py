"""CPU oracle for numerical entanglement -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  The product library never imports it and
shares no code with it.  The arithmetic lives in ``ne_oracle.c`` (plain C,
every intermediate in ``__int128`` with overflow checks); this module only
marshals numpy arrays and composes the paper's steps:

  entangle (Eq. 7 / Eq. 16)  ->  op on each entangled stream (Eq. 10)
  ->  extract + check with an unused stream r (Eq. 17-20, Eq. 24)

and the checksum-ABFT comparator (Eq. 3-6).  All functions take and return
C-contiguous numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ne_oracle.c")
_LIB = os.path.join(_HERE, "libne_oracle.so")

POLICY_PAPER = 0        # maximise (M-2)l+k under Eq. 13 with k <= l (Table II rule)
POLICY_SMALLEST = 1     # smallest l whose Eq. 14 range covers the output bound
POLICY_BYTE = 2         # smallest multiple-of-8 l whose Eq. 14 range covers the bound


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ne_oracle.c into libne_oracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i32, i64, p = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        lib.or_threads.restype = i32
        lib.or_set_threads.argtypes = [i32]
        lib.or_set_threads.restype = None
        lib.or_range_eq14.argtypes = [i32, i32, i32]
        lib.or_range_eq14.restype = i64
        lib.or_choose_l.argtypes = [i32, i32, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.or_entangle.argtypes = [i32, i32, p, p, i64]
        lib.or_gemm.argtypes = [p, p, p, i32, i32, i32]
        lib.or_cconv.argtypes = [p, p, p, i64, i64, i64]
        lib.or_elementwise.argtypes = [i32, p, p, p, i64]
        lib.or_entangle_kernel_self.argtypes = [i32, p, p, i64]
        lib.or_extract.argtypes = [i32, i32, p, i64, i32, p, p]
        lib.or_inner.argtypes = [p, p, p, i64, i64, i64]
        lib.or_cconv_at.argtypes = [p, p, i64, i64, p, p, i64, p]
        lib.or_lconv.argtypes = [p, p, p, i64, i64, i64, i64]
        lib.or_lconv_at.argtypes = [p, p, i64, i64, i64, p, p, i64, p]
        lib.or_rc_encode.argtypes = [p, p, i64, i64, i64, p, p]
        lib.or_gemm64.argtypes = [p, p, p, i64, i64, i64]
        lib.or_rc_check.argtypes = [p, i64, i64, p, p]
        lib.or_rc_correct.argtypes = [p, i64, i64, ctypes.POINTER(i32)]
        lib.or_outer.argtypes = [p, p, p, i64, i64, i64, i64]
        lib.or_permute.argtypes = [p, p, p, i64, i64, i64]
        lib.or_cxcorr.argtypes = [p, p, p, i64, i64, i64]
        lib.or_abft_encode.argtypes = [i32, p, i64, p]
        lib.or_abft_check.argtypes = [i32, p, i64, p]
        lib.or_abft_recover.argtypes = [i32, p, i64, i32]
        for f in ("or_entangle", "or_gemm", "or_cconv", "or_lconv", "or_lconv_at", "or_elementwise", "or_entangle_kernel_self",
                  "or_extract", "or_cconv_at", "or_rc_encode", "or_gemm64", "or_rc_check", "or_rc_correct", "or_inner", "or_outer", "or_permute", "or_cxcorr", "or_abft_encode", "or_abft_check", "or_abft_recover", "or_choose_l"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


_ERR = {1: "overflow: an intermediate left the int64 word (checked in __int128)",
        2: "invalid argument", 3: "no feasible (l, k)"}


def _chk(code: int, what: str):
    if code != 0:
        raise OracleError(f"{what}: {_ERR.get(code, code)}")


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_L().or_threads())


def set_threads(n: int) -> None:
    """OpenMP threads for the following calls (for timing; results are the same)."""
    _L().or_set_threads(int(n))


# ---- parameters (Eq. 13, Eq. 14, Table II) --------------------------------

def range_eq14(M: int, l: int, k: int) -> int:
    """Eq. 14 output range bound 2^((M-3)l+k) (2^(l-1)-1); -1 if >= 2^63."""
    return int(_L().or_range_eq14(M, l, k))


def choose_l(M: int, w: int = 64, out_bound: int = 0, policy: int = POLICY_PAPER):
    l, k = ctypes.c_int(), ctypes.c_int()
    _chk(_L().or_choose_l(M, w, int(out_bound), policy, ctypes.byref(l), ctypes.byref(k)), "choose_l")
    return l.value, k.value


# ---- entanglement ----------------------------------------------------------

def entangle(c, l: int):
    """c: int32 [M, n] (or [..., M, n]); returns int64 eps of the same shape (Eq. 16)."""
    c, pc = _arr(c, np.int32)
    M, n = c.shape[-2], c.shape[-1]
    out = np.empty(c.shape, np.int64)
    batch = int(np.prod(c.shape[:-2], dtype=np.int64)) if c.ndim > 2 else 1
    for b in range(batch):
        _chk(_L().or_entangle(M, l, pc + b * M * n * 4, out.ctypes.data + b * M * n * 8, n), "entangle")
    return out


# ---- LSB operations (Eq. 2 / Eq. 10) ---------------------------------------

def gemm(A, G):
    """D = A @ G exactly; A int64 [m, k], G int8 [k, n]."""
    A, pa = _arr(A, np.int64)
    G, pg = _arr(G, np.int8)
    m, k = A.shape
    k2, n = G.shape
    assert k == k2
    D = np.empty((m, n), np.int64)
    _chk(_L().or_gemm(pa, pg, D.ctypes.data, m, n, k), "gemm")
    return D


def cconv(x, g):
    """Circular convolution y[.., n] = sum_j x[.., j] g[(n - j) mod N].

    x: int64 [B, S, N]; g: int8 [B, N] (kernel b serves the S signals of group b).
    """
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int8)
    B, S, N = x.shape
    assert g.shape == (B, N)
    y = np.empty_like(x)
    _chk(_L().or_cconv(px, pg, y.ctypes.data, B, S, N), "cconv")
    return y


def cconv_at(x, g, signal, pos):
    """Selected outputs y[signal[t], pos[t]] of cconv(x, g), one by one (x int64
    [B, S, N], g int8 [B, N], signal = b * S + s)."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int8)
    B, S, N = x.shape
    sig, ps = _arr(signal, np.int64)
    pos, pp = _arr(pos, np.int64)
    y = np.empty(sig.size, np.int64)
    _chk(_L().or_cconv_at(px, pg, S, N, ps, pp, sig.size, y.ctypes.data), "cconv_at")
    return y


def lconv(x, g):
    """Full linear convolution y[.., i] = sum_t g[.., t] x[.., i - t], i < n + K - 1
    (x zero outside [0, n)); x int64 [B, S, n], g int8 [B, K]."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int8)
    B, S, n = x.shape
    K = g.shape[1]
    assert g.shape == (B, K)
    y = np.empty((B, S, n + K - 1), np.int64)
    _chk(_L().or_lconv(px, pg, y.ctypes.data, B, S, n, K), "lconv")
    return y


def lconv_at(x, g, signal, pos):
    """Selected outputs y[signal[t], pos[t]] of lconv(x, g), one by one
    (signal = b * S + s)."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int8)
    B, S, n = x.shape
    K = g.shape[1]
    sig, ps = _arr(signal, np.int64)
    pos, pp = _arr(pos, np.int64)
    y = np.empty(sig.size, np.int64)
    _chk(_L().or_lconv_at(px, pg, S, n, K, ps, pp, sig.size, y.ctypes.data), "lconv_at")
    return y


OP_ADD, OP_SUB, OP_MUL = 0, 1, 2


def elementwise(op: int, x, g):
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int64)
    assert x.shape == g.shape
    y = np.empty_like(x)
    _chk(_L().or_elementwise(op, px, pg, y.ctypes.data, x.size), "elementwise")
    return y


def entangle_kernel_self(g, l: int):
    """Footnote to Eq. 10: g <- S_l{g} + g (for op in {+, -})."""
    g, pg = _arr(g, np.int64)
    out = np.empty_like(g)
    _chk(_L().or_entangle_kernel_self(l, pg, out.ctypes.data, g.size), "entangle_kernel_self")
    return out


def inner(x, g):
    """Inner products y[b, s] = sum_i x[b, s, i] g[b, i]; x int64 [B, S, n], g int64 [B, n]."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int64)
    B, S, n = x.shape
    assert g.shape == (B, n)
    y = np.empty((B, S), np.int64)
    _chk(_L().or_inner(px, pg, y.ctypes.data, B, S, n), "inner")
    return y


def outer(x, g):
    """Outer products y[b, s, i, j] = x[b, s, i] g[b, j]; x int64 [B, S, n], g int64 [B, k]."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int64)
    B, S, n = x.shape
    k = g.shape[1]
    assert g.shape[0] == B
    y = np.empty((B, S, n, k), np.int64)
    _chk(_L().or_outer(px, pg, y.ctypes.data, B, S, n, k), "outer")
    return y


def permute(x, g):
    """y[b, s, i] = x[b, s, g[i]]; x int64 [B, S, n], g a permutation of range(n)."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int64)
    B, S, n = x.shape
    assert g.shape == (n,)
    y = np.empty_like(x)
    _chk(_L().or_permute(px, pg, y.ctypes.data, B, S, n), "permute")
    return y


def cxcorr(x, g):
    """Circular cross-correlation y[.., i] = sum_j x[.., (i + j) mod N] g[.., j];
    x int64 [B, S, N], g int8 [B, N]."""
    x, px = _arr(x, np.int64)
    g, pg = _arr(g, np.int8)
    B, S, N = x.shape
    assert g.shape == (B, N)
    y = np.empty_like(x)
    _chk(_L().or_cxcorr(px, pg, y.ctypes.data, B, S, N), "cxcorr")
    return y


# ---- extraction / check / recovery (Eq. 17-20, Eq. 24) ---------------------

def extract(delta, l: int, r: int = 0, check: bool = True):
    """delta: int64 [M, n] (or [..., M, n]).  Returns (dhat, flags) where flags
    is a uint8 array of the positions (None when check is False, in which case
    delta[r] is not read: this is the fail-stop recovery of Prop. 3)."""
    delta, pd = _arr(delta, np.int64)
    M, n = delta.shape[-2], delta.shape[-1]
    batch = int(np.prod(delta.shape[:-2], dtype=np.int64)) if delta.ndim > 2 else 1
    dhat = np.empty(delta.shape, np.int64)
    flags = np.zeros(delta.shape[:-2] + (n,), np.uint8) if check else None
    for b in range(batch):
        fp = flags.ctypes.data + b * n if check else None
        _chk(_L().or_extract(M, l, pd + b * M * n * 8, n, r, dhat.ctypes.data + b * M * n * 8, fp), "extract")
    return dhat, flags


def recover(delta, l: int, r_lost: int):
    """Prop. 3: all M outputs from the M-1 planes other than r_lost."""
    return extract(delta, l, r_lost, check=False)[0]


# ---- checksum ABFT (Eq. 3-6) ----------------------------------------------

def abft_encode(c):
    """Eq. 4: r = sum_m c_m; c int32 [M, n] -> int64 [n]."""
    c, pc = _arr(c, np.int32)
    M, n = c.shape
    r = np.empty(n, np.int64)
    _chk(_L().or_abft_encode(M, pc, n, r.ctypes.data), "abft_encode")
    return r


def abft_check(d):
    """Eq. 6 per position; d int64 [M+1, n] (last plane is e)."""
    d, pd = _arr(d, np.int64)
    M = d.shape[0] - 1
    n = d.shape[1]
    f = np.zeros(n, np.uint8)
    _chk(_L().or_abft_check(M, pd, n, f.ctypes.data), "abft_check")
    return f


def abft_recover(d, j: int):
    """Sec. II-A: rebuild plane j of d [M+1, n] from e and the others."""
    d = np.array(d, dtype=np.int64, order="C", copy=True)
    M = d.shape[0] - 1
    _chk(_L().or_abft_recover(M, d.ctypes.data, d.shape[1], j), "abft_recover")
    return d


# ---- row/column checksum ABFT of a product (ABFT RC-check, Sec. V) ----------

def rc_encode(A, B):
    """Column-checksum matrix of A [m, k] and row-checksum matrix of B (int8 [k, n]):
    returns (ac [m+1, k], br [k, n+1]), int64."""
    A, pa = _arr(A, np.int64)
    B, pb = _arr(B, np.int8)
    m, k = A.shape
    n = B.shape[1]
    ac = np.empty((m + 1, k), np.int64)
    br = np.empty((k, n + 1), np.int64)
    _chk(_L().or_rc_encode(pa, pb, m, k, n, ac.ctypes.data, br.ctypes.data), "rc_encode")
    return ac, br


def gemm64(X, Y):
    """Z = X Y exactly for int64 matrices."""
    X, px = _arr(X, np.int64)
    Y, py = _arr(Y, np.int64)
    m, k = X.shape
    n = Y.shape[1]
    Z = np.empty((m, n), np.int64)
    _chk(_L().or_gemm64(px, py, Z.ctypes.data, m, k, n), "gemm64")
    return Z


def rc_full(A, B):
    """The full-checksum matrix of C = A B, [m+1, n+1]."""
    ac, br = rc_encode(A, B)
    return gemm64(ac, br)


def rc_check(Cf):
    """(rowbad [m+1], colbad [n+1]) of a full-checksum matrix."""
    Cf, pc = _arr(Cf, np.int64)
    m, n = Cf.shape[0] - 1, Cf.shape[1] - 1
    rb = np.zeros(m + 1, np.uint8)
    cb = np.zeros(n + 1, np.uint8)
    _chk(_L().or_rc_check(pc, m, n, rb.ctypes.data, cb.ctypes.data), "rc_check")
    return rb, cb


def rc_correct(Cf):
    """Single-error correction; returns (corrected copy, whether an entry was replaced)."""
    Cf = np.array(Cf, dtype=np.int64, order="C", copy=True)
    done = ctypes.c_int(0)
    _chk(_L().or_rc_correct(Cf.ctypes.data, Cf.shape[0] - 1, Cf.shape[1] - 1, ctypes.byref(done)), "rc_correct")
    return Cf, bool(done.value)


# ---- the pipelines composed from the steps ---------------------------------

def gemm_direct(c, G):
    """d_m = c_m G for every stream (Eq. 2, inner products); c int32 [M, m, k]."""
    return np.stack([gemm(np.asarray(cm, np.int64), G) for cm in c])


def gemm_entangled(c, G, l: int, r: int = 0):
    """entangle -> delta_m = eps_m G -> extract/check.  Returns (dhat, flags, delta)."""
    M, m, k = c.shape
    eps = entangle(c.reshape(M, m * k), l).reshape(M, m, k)
    delta = np.stack([gemm(eps[i], G) for i in range(M)])
    n = G.shape[1]
    dhat, flags = extract(delta.reshape(M, m * n), l, r)
    return dhat.reshape(M, m, n), flags.reshape(m, n), delta


def cconv_direct(c, g):
    """c int32 [B, M, N], g int8 [B, N] -> int64 [B, M, N]."""
    return cconv(np.asarray(c, np.int64), g)


def cconv_entangled(c, g, l: int, r: int = 0):
    """entangle each group -> circular convolution per stream -> extract/check.
    Returns (dhat [B, M, N], flags [B, N], delta [B, M, N])."""
    eps = entangle(c, l)
    delta = cconv(eps, g)
    dhat, flags = extract(delta, l, r)
    return dhat, flags, delta


def lconv_direct(c, g):
    """c int32 [B, M, n], g int8 [B, K] -> int64 [B, M, n + K - 1]."""
    return lconv(np.asarray(c, np.int64), g)


def lconv_entangled(c, g, l: int, r: int = 0):
    """entangle each group -> linear convolution per stream -> extract/check.
    Returns (dhat [B, M, n + K - 1], flags [B, n + K - 1], delta)."""
    eps = entangle(c, l)
    delta = lconv(eps, g)
    dhat, flags = extract(delta, l, r)
    return dhat, flags, delta


LSB_OPS = ("add", "sub", "mul", "inner", "outer", "permute", "cxcorr")


def lsb_apply(op: str, x, g):
    """The operator of Eq. 2 on every signal of x (int64 [B, S, n]).  g: int64
    [B, n] (add/sub/mul/inner), int64 [B, k] (outer), a permutation of
    range(n) (permute) or int8 [B, n] (cxcorr)."""
    x = np.asarray(x, np.int64)
    if op in ("add", "sub", "mul"):
        code = {"add": OP_ADD, "sub": OP_SUB, "mul": OP_MUL}[op]
        return elementwise(code, x, np.broadcast_to(np.asarray(g, np.int64)[:, None, :], x.shape))
    return {"inner": inner, "outer": outer, "permute": permute, "cxcorr": cxcorr}[op](x, g)


def lsb_direct(op: str, c, g):
    """The operator on the raw streams c (int32 [B, M, n])."""
    return lsb_apply(op, np.asarray(c, np.int64), g)


def lsb_entangled(op: str, c, g, l: int, r: int = 0):
    """entangle (Eq. 16) -> the operator on every entangled stream (Eq. 10;
    for + and - the kernel is first entangled with itself, the footnote to
    Eq. 10) -> extract/check (Eq. 17-20, Eq. 24).  Returns (dhat, flags,
    delta); delta is [B, M, ...] and flags cover each group's output
    positions in row-major order."""
    B, M = np.asarray(c).shape[:2]
    eps = entangle(c, l)
    if op in ("add", "sub"):
        g = entangle_kernel_self(np.asarray(g, np.int64), l)
    delta = lsb_apply(op, eps, g)
    dhat, flags = extract(delta.reshape(B, M, -1), l, r)
    return dhat.reshape(delta.shape), flags, delta
