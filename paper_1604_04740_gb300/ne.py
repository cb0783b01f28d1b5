"""Thin Python binding of the C ABI in include/ne.h (argument marshalling only).

Every function here has the name of the C entry point it calls, takes torch
tensors that already live on the GPU, checks dtype/device/contiguity/shape,
passes raw device pointers and the current CUDA stream, and raises NEError
on a non-zero status.  No computation happens in Python: if libne.so cannot
be built or loaded, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

NE_OK, NE_EINVAL, NE_ERANGE, NE_ECUDA, NE_ETIMEOUT, NE_ENOMEM = range(6)
NE_L_PAPER, NE_L_SMALLEST, NE_L_BYTE = 0, 1, 2
NE_FUSE_NONE, NE_FUSE_EXTRACT_CHECK, NE_FUSE_RECOVER = 0, 1, 2
NE_MODE_I64, NE_MODE_S8SLICE = 0, 1
NE_MAX_DIGITS = 8


class NEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class ne_params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("l", ctypes.c_int32), ("w", ctypes.c_int32)]


class ne_digits(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int32), ("shift", ctypes.c_int32 * NE_MAX_DIGITS),
                ("l", ctypes.c_int32), ("lo", ctypes.c_int32), ("hi", ctypes.c_int32)]

    @property
    def shifts(self):
        return tuple(self.shift[i] for i in range(self.S))

    def __repr__(self):
        return f"ne_digits(S={self.S}, shift={self.shifts})"


class ne_faults(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("bit", ctypes.c_void_p),
                ("count", ctypes.c_int64)]


def faults(pos: torch.Tensor | None = None, stream: torch.Tensor | None = None,
           bit: torch.Tensor | None = None) -> ne_faults:
    """The ne_faults of three device tensors (pos int64, stream int32, bit
    int32, equal lengths; pos ascending).  No arguments: no faults.  The
    caller keeps the tensors alive until the call that uses them has run."""
    f = ne_faults()
    if pos is None:
        if stream is not None or bit is not None:
            raise ValueError("fault lists need pos, stream and bit together")
        return f
    n = pos.numel()
    if stream.numel() != n or bit.numel() != n:
        raise ValueError("fault lists differ in length")
    f.pos = _ptr(pos, torch.int64, "fault pos")
    f.stream = _ptr(stream, torch.int32, "fault stream")
    f.bit = _ptr(bit, torch.int32, "fault bit")
    f.count = n
    return f


def _faults_arg(fl) -> ne_faults:
    if fl is None:
        return ne_faults()
    if isinstance(fl, ne_faults):
        return fl
    return faults(*fl)


NE_JOB_GEMM, NE_JOB_CCONV = 0, 1
NE_ORDER_JOB, NE_ORDER_LPT = 0, 1


class ne_job(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("kind", "M", "l", "rows", "cols", "k", "N", "r", "fuse", "cmin", "cmax",
                                              "plain")] + \
               [(n, ctypes.c_int64) for n in ("c_off", "op_off", "out_off", "flag_off", "fault_begin", "fault_end")]


class ne_batch_config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("ctas_per_sm", "order", "cconv_blocks", "l_policy", "ntt_min_n")]


class ne_batch_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("njobs", "ntiles", "nsegs", "grid", "ngemm_tiles", "gemm_grid")] + \
               [(n, ctypes.c_int64) for n in ("flag_words", "workspace_bytes", "mma_ops", "useful_ops")] + \
               [(n, ctypes.c_int32) for n in ("ntransform", "ntt_max_logL", "ntt_max_M", "ntt_min_logL")] + \
               [(n, ctypes.c_int64) for n in ("ntt_table_off", "ntt_ws_off", "ntt_units", "table_bytes")]


def params(M: int, l: int, w: int = 64) -> ne_params:
    return ne_params(M, l, w)


def digits(shifts) -> ne_digits:
    """A digit set without a known input range (every word is checked)."""
    d = ne_digits()
    d.S = len(shifts)
    for i, s in enumerate(shifts):
        d.shift[i] = s
    d.l, d.lo, d.hi = 0, 1, 0
    return d


def raw_digits(lo: int = -128, hi: int = 127) -> ne_digits:
    """One digit at shift 0 for raw streams with values in [lo, hi] (the plain
    operation of the fused kernels)."""
    d = digits((0,))
    d.lo, d.hi = lo, hi
    return d


def _load():
    path = _build.LIB
    if not os.path.exists(path) or os.environ.get("NE_REBUILD") == "1":
        _build.build()
    lib = ctypes.CDLL(path)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "ne_choose_l": [i32, i32, i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "ne_plan_digits": [i32, i32, i32, ctypes.POINTER(ne_digits)],
        "ne_entangle": [ne_params, P, P, i64, i64, P],
        "ne_entangle_digits": [ne_params, ne_digits, P, P, i64, i64, P, P],
        "ne_gemm": [ne_params, P, P, P, P, P, i32, i32, i32, i32, ne_digits, i32, i32, u32, ne_faults, P, P],
        "ne_gemm_digits": [ne_params, ne_digits, P, P, P, P, P, i32, i32, i32, i32, i32, ne_faults, P],
        "ne_cconv": [ne_params, P, P, P, P, P, i64, i64, i32, ne_digits, i32, i32, u32, ne_faults, P, P],
        "ne_cconv_digits": [ne_params, ne_digits, P, P, P, P, P, i64, i64, i32, i32, ne_faults, P],
        "ne_extract": [ne_params, P, P, i64, i64, i32, P, P, P],
        "ne_check": [ne_params, P, i64, i64, i32, P, P, P, P],
        "ne_recover": [ne_params, P, P, i64, i64, i32, P],
        "ne_check_set_wait_limit": [u32],
        "ne_inject": [P, i32, i64, i64, P, P, P, P, i64, P, P],
        "ne_abft_encode": [i32, P, P, i64, i64, P],
        "ne_abft_check": [i32, P, i64, i64, P, P, P],
        "ne_abft_recover": [i32, P, i64, i64, i32, P],
        "ne_split_digits": [ne_digits, P, P, i64, i32, i64, P, P],
        "ne_split_digits_raw": [ne_params, ne_digits, P, P, i64, i64, P, P],
        "ne_batch_plan": [ctypes.POINTER(ne_job), i32, ne_batch_config, P, i64, ctypes.POINTER(ne_batch_info), P],
        "ne_batch_plan_staged": [ctypes.POINTER(ne_job), i32, ne_batch_config, P, i64, P, i64,
                                 ctypes.POINTER(ne_batch_info), P],
        "ne_batch_run": [ne_batch_info, P, P, P, P, P, P, P, P, P, P, P],
        "ne_batch_run_static": [ctypes.POINTER(ne_job), i32, ne_batch_config, P, P, P, P, P, P, P, P, P, P],
        "ne_copy_regions_h2d": [P, P, P, P, P, i64, P],
        "ne_cconv_entangled": [ne_params, ne_digits, P, P, P, P, P, i64, i64, i32, i32, i32, ne_faults, P, P],
        "ne_set_cconv_split": [i32],
        "ne_lconv": [ne_params, ne_digits, P, P, P, P, P, i64, i64, i64, i32, i32, i32, ne_faults, P, P],
        "ne_cconv_ntt_any": [ne_params, i32, i32, P, P, P, P, P, i64, i64, i32, i32, i32, ne_faults, P, P, i64, P],
        "ne_cconv_ntt": [ne_params, ne_digits, P, P, P, P, P, i64, i64, i32, i32, i32, ne_faults, P, P],
        "ne_abft_rc_encode": [P, P, P, P, i64, i64, i64, i64, P],
        "ne_abft_rc_check": [P, P, P, P, P, P, P, P, P, i64, i64, i64, i64, P],
        "ne_abft_rc_correct": [P, P, P, P, P, i64, i64, i64, P],
        "ne_elementwise": [ne_params, i32, P, P, i64, P, P, P, i64, i64, i32, i32, P],
        "ne_entangle_kernel_self": [i32, P, P, i64, P],
        "ne_outer": [ne_params, P, P, i64, P, P, P, i64, i64, i64, i32, i32, P],
        "ne_permute": [ne_params, P, P, P, P, P, i64, i64, i32, i32, P, P],
        "ne_inner": [ne_params, P, P, i64, P, P, P, i64, i64, i32, i32, P],
        "ne_reverse_operand": [P, P, i64, i64, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ne_cconv_ntt_any_workspace.argtypes = [i32, i64, i64]
    lib.ne_cconv_ntt_any_workspace.restype = i64
    lib.ne_last_error.restype = ctypes.c_char_p
    lib.ne_version.restype = ctypes.c_char_p
    return lib


_lib = _load()
LIB_PATH = _build.LIB


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call(name: str, *args):
    st = getattr(_lib, name)(*args)
    if st != NE_OK:
        raise NEError(st, _lib.ne_last_error().decode())


def _ptr(t, dtype, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def ne_version() -> str:
    return _lib.ne_version().decode()


# ---- planning ----------------------------------------------------------------

def ne_choose_l(M: int, w: int = 64, out_bound: int = 0, policy: int = NE_L_PAPER):
    l, k = ctypes.c_int32(), ctypes.c_int32()
    _call("ne_choose_l", M, w, int(out_bound), policy, ctypes.byref(l), ctypes.byref(k))
    return l.value, k.value


def ne_plan_digits(l: int, cmin: int = -128, cmax: int = 127) -> ne_digits:
    d = ne_digits()
    _call("ne_plan_digits", l, cmin, cmax, ctypes.byref(d))
    return d


# ---- entanglement --------------------------------------------------------------

def _bmn(t, M):
    """(batch, n) of a [.., M, n] plane tensor."""
    if t.dim() < 2 or t.shape[-2] != M:
        raise ValueError(f"expected [..., {M}, n] planes, got {tuple(t.shape)}")
    n = t.shape[-1]
    batch = t.numel() // (M * n) if n else 0
    return batch, n


def ne_entangle(p: ne_params, c: torch.Tensor, eps: torch.Tensor | None = None) -> torch.Tensor:
    batch, n = _bmn(c, p.M)
    if eps is None:
        eps = torch.empty(c.shape, dtype=torch.int64, device=c.device)
    if eps.shape != c.shape:
        raise ValueError("eps must have the shape of c")
    _call("ne_entangle", p, _ptr(c, torch.int32, "c"), _ptr(eps, torch.int64, "eps"), batch, n, _stream())
    return eps


def ne_entangle_digits(p: ne_params, dg: ne_digits, c: torch.Tensor, planes: torch.Tensor | None = None,
                       status: torch.Tensor | None = None) -> torch.Tensor:
    """planes: int8 [..., M, S, n] (the shape of c with S inserted)."""
    batch, n = _bmn(c, p.M)
    shape = tuple(c.shape[:-1]) + (dg.S, n)
    if planes is None:
        planes = torch.empty(shape, dtype=torch.int8, device=c.device)
    if tuple(planes.shape) != shape:
        raise ValueError(f"planes must be {shape}")
    _call("ne_entangle_digits", p, dg, _ptr(c, torch.int32, "c"), _ptr(planes, torch.int8, "planes"), batch, n,
          _ptr(status, torch.int32, "status", True), _stream())
    return planes


def ne_split_digits_raw(p: ne_params, dg: ne_digits, c: torch.Tensor, planes: torch.Tensor | None = None,
                        status: torch.Tensor | None = None) -> torch.Tensor:
    """The raw streams c int32 [..., M, n] as digit planes int8 [..., M, S, n]
    with an entangled plan's digit set (the plain operation's operand)."""
    batch, n = _bmn(c, p.M)
    shape = tuple(c.shape[:-1]) + (dg.S, n)
    if planes is None:
        planes = torch.empty(shape, dtype=torch.int8, device=c.device)
    if tuple(planes.shape) != shape:
        raise ValueError(f"planes must be {shape}")
    _call("ne_split_digits_raw", p, dg, _ptr(c, torch.int32, "c"), _ptr(planes, torch.int8, "planes"), batch, n,
          _ptr(status, torch.int32, "status", True), _stream())
    return planes


def ne_split_digits(dg: ne_digits, x: torch.Tensor, P: int, planes: torch.Tensor | None = None,
                    status: torch.Tensor | None = None) -> torch.Tensor:
    """x int64 [..., P, n] -> planes int8 [..., P, S, n]."""
    batch, n = _bmn(x, P)
    shape = tuple(x.shape[:-1]) + (dg.S, n)
    if planes is None:
        planes = torch.empty(shape, dtype=torch.int8, device=x.device)
    if tuple(planes.shape) != shape:
        raise ValueError(f"planes must be {shape}")
    _call("ne_split_digits", dg, _ptr(x, torch.int64, "x"), _ptr(planes, torch.int8, "planes"), batch, P, n,
          _ptr(status, torch.int32, "status", True), _stream())
    return planes


# ---- operations ----------------------------------------------------------------

def ne_gemm(p: ne_params, eps: torch.Tensor, G: torch.Tensor, out: torch.Tensor | None = None,
            flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None, mode: int = NE_MODE_I64,
            dg: ne_digits | None = None, fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, drop_mask: int = 0,
            faults=None, status: torch.Tensor | None = None) -> torch.Tensor:
    """eps int64 [M, rows, k] @ G int8 [k, cols] -> int64 [M, rows, cols]: delta
    (NE_FUSE_NONE) or d_hat.  mode NE_MODE_I64 (CUDA cores) or NE_MODE_S8SLICE
    (int8 tensor path, the words split into the digits of dg in the kernel).
    faults: None, an ne_faults or (pos, stream, bit) device tensors."""
    M, rows, k = eps.shape
    if M != p.M:
        raise ValueError("eps must be [M, rows, k]")
    k2, cols = G.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((M, rows, cols), dtype=torch.int64, device=eps.device)
    if tuple(out.shape) != (M, rows, cols):
        raise ValueError("out shape")
    _call("ne_gemm", p, _ptr(eps, torch.int64, "eps"), _ptr(G, torch.int8, "G"), _ptr(out, torch.int64, "out"),
          _ptr(flags, torch.int32, "flags", True), _ptr(nflag, torch.int64, "nflag", True), rows, cols, k, mode,
          dg if dg is not None else ne_digits(), fuse, r, drop_mask, _faults_arg(faults),
          _ptr(status, torch.int32, "status", True), _stream())
    return out


def ne_gemm_digits(p: ne_params, dg: ne_digits, planes: torch.Tensor, G: torch.Tensor,
                   out: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                   nflag: torch.Tensor | None = None, fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0,
                   faults=None) -> torch.Tensor:
    """planes int8 [M, S, rows, k]; G int8 [k, cols] -> int64 [M, rows, cols].
    faults: None, an ne_faults, or (pos, stream, bit) device tensors
    (positions i * cols + j, ascending)."""
    M, S, rows, k = planes.shape
    if M != p.M or S != dg.S:
        raise ValueError("planes shape does not match (M, S)")
    k2, cols = G.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if out is None:
        out = torch.empty((M, rows, cols), dtype=torch.int64, device=planes.device)
    _call("ne_gemm_digits", p, dg, _ptr(planes, torch.int8, "planes"), _ptr(G, torch.int8, "G"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), rows, cols, k, fuse, r, _faults_arg(faults), _stream())
    return out


def ne_cconv(p: ne_params, eps: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
             flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None, mode: int = NE_MODE_I64,
             dg: ne_digits | None = None, fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, drop_mask: int = 0,
             faults=None, status: torch.Tensor | None = None) -> torch.Tensor:
    """eps int64 [batch, M, N], g int8 [batch, N] -> int64 [batch, M, N]:
    delta (NE_FUSE_NONE) or d_hat; modes and faults as for ne_gemm."""
    batch, M, N = eps.shape
    if M != p.M or tuple(g.shape) != (batch, N):
        raise ValueError("eps must be [batch, M, N] and g [batch, N]")
    if out is None:
        out = torch.empty_like(eps)
    _call("ne_cconv", p, _ptr(eps, torch.int64, "eps"), _ptr(g, torch.int8, "g"), _ptr(out, torch.int64, "out"),
          _ptr(flags, torch.int32, "flags", True), _ptr(nflag, torch.int64, "nflag", True), batch, N, mode,
          dg if dg is not None else ne_digits(), fuse, r, drop_mask, _faults_arg(faults),
          _ptr(status, torch.int32, "status", True), _stream())
    return out


def planes_of(M: int) -> ne_params:
    """The parameters of the bare operation on M planes (NE_FUSE_NONE, NE_MODE_I64:
    l is not used): the plain operation or the checksum comparator."""
    return ne_params(M, 1, 64)


def ne_cconv_digits(p: ne_params, dg: ne_digits, planes: torch.Tensor, g: torch.Tensor,
                    out: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                    nflag: torch.Tensor | None = None, fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0,
                    faults=None) -> torch.Tensor:
    """planes int8 [batch, M, S, N]; g int8 [batch, N] -> int64 [batch, M, N].
    faults as for ne_gemm_digits (positions group * N + i)."""
    batch, M, S, N = planes.shape
    if M != p.M or S != dg.S or tuple(g.shape) != (batch, N):
        raise ValueError("planes / g shapes")
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.int64, device=planes.device)
    _call("ne_cconv_digits", p, dg, _ptr(planes, torch.int8, "planes"), _ptr(g, torch.int8, "g"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, N, fuse, r, _faults_arg(faults), _stream())
    return out


def ne_set_cconv_split(variant: int = -1):
    """The tensor / dp4a split of the convolution tile (-1: the default)."""
    _call("ne_set_cconv_split", variant)


def ne_cconv_entangled(p: ne_params, dg: ne_digits, c: torch.Tensor, g: torch.Tensor,
                       out: torch.Tensor | None = None, flags: torch.Tensor | None = None,
                       nflag: torch.Tensor | None = None, fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0,
                       plain: bool = False, status: torch.Tensor | None = None, faults=None) -> torch.Tensor:
    """c int32 [batch, M, N] (raw streams); g int8 [batch, N] -> int64 [batch, M, N] (tensor path, one launch).
    faults as for ne_cconv_digits."""
    batch, M, N = c.shape
    if M != p.M or tuple(g.shape) != (batch, N):
        raise ValueError("c / g shapes")
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.int64, device=c.device)
    _call("ne_cconv_entangled", p, dg, _ptr(c, torch.int32, "c"), _ptr(g, torch.int8, "g"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, N, fuse, r, 1 if plain else 0, _faults_arg(faults),
          _ptr(status, torch.int32, "status", True), _stream())
    return out


def ne_lconv(p: ne_params, dg: ne_digits, c: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
             flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
             fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, plain: bool = False,
             status: torch.Tensor | None = None, faults=None) -> torch.Tensor:
    """Full linear convolution of long streams: c int32 [batch, M, n] (raw),
    g int8 [batch, K] -> int64 [batch, M, n + K - 1]."""
    batch, M, n = c.shape
    if M != p.M or g.dim() != 2 or g.shape[0] != batch:
        raise ValueError("c must be [batch, M, n] and g [batch, K]")
    K = g.shape[1]
    if out is None:
        out = torch.empty((batch, M, n + K - 1), dtype=torch.int64, device=c.device)
    if tuple(out.shape) != (batch, M, n + K - 1):
        raise ValueError("out must be [batch, M, n + K - 1]")
    _call("ne_lconv", p, dg, _ptr(c, torch.int32, "c"), _ptr(g, torch.int8, "g"), _ptr(out, torch.int64, "out"),
          _ptr(flags, torch.int32, "flags", True), _ptr(nflag, torch.int64, "nflag", True), batch, n, K, fuse, r,
          1 if plain else 0, _faults_arg(faults), _ptr(status, torch.int32, "status", True), _stream())
    return out


def ne_cconv_ntt_any(p: ne_params, c: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                     flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
                     fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, plain: bool = False,
                     status: torch.Tensor | None = None, cmin: int = -128, cmax: int = 127,
                     workspace: torch.Tensor | None = None, faults=None) -> torch.Tensor:
    """c int32 [batch, M, N] (raw streams, any N in [2, 65536]); g int8 [batch, N] -> int64 [batch, M, N].
    faults as for ne_cconv_digits."""
    batch, M, N = c.shape
    if M != p.M or tuple(g.shape) != (batch, N):
        raise ValueError("c / g shapes")
    need = int(_lib.ne_cconv_ntt_any_workspace(M, N, batch))
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=c.device)
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.int64, device=c.device)
    _call("ne_cconv_ntt_any", p, cmin, cmax, _ptr(c, torch.int32, "c"), _ptr(g, torch.int8, "g"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, N, fuse, r, 1 if plain else 0, _faults_arg(faults),
          _ptr(status, torch.int32, "status", True), _ptr(workspace, torch.uint8, "workspace"),
          workspace.numel(), _stream())
    return out


def ne_cconv_ntt(p: ne_params, dg: ne_digits, c: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                 flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
                 fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, plain: bool = False,
                 status: torch.Tensor | None = None, faults=None) -> torch.Tensor:
    """c int32 [batch, M, N] (raw streams); g int8 [batch, N] -> int64 [batch, M, N].
    faults as for ne_cconv_digits."""
    batch, M, N = c.shape
    if M != p.M or tuple(g.shape) != (batch, N):
        raise ValueError("c / g shapes")
    if out is None:
        out = torch.empty((batch, M, N), dtype=torch.int64, device=c.device)
    _call("ne_cconv_ntt", p, dg, _ptr(c, torch.int32, "c"), _ptr(g, torch.int8, "g"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, N, fuse, r, 1 if plain else 0, _faults_arg(faults),
          _ptr(status, torch.int32, "status", True), _stream())
    return out


# ---- row/column checksum ABFT of a product (ABFT RC-check) ---------------------------

def ne_abft_rc_encode(A: torch.Tensor, B: torch.Tensor, ac: torch.Tensor | None = None,
                      br: torch.Tensor | None = None):
    """A int32 [batch, m, k], B int8 [k, n] -> (ac int64 [batch, k], br int64 [k])."""
    batch, m, k = A.shape
    n = B.shape[1]
    if ac is None:
        ac = torch.empty((batch, k), dtype=torch.int64, device=A.device)
    if br is None:
        br = torch.empty(k, dtype=torch.int64, device=A.device)
    _call("ne_abft_rc_encode", _ptr(A, torch.int32, "A"), _ptr(B, torch.int8, "B"), _ptr(ac, torch.int64, "ac"),
          _ptr(br, torch.int64, "br"), batch, m, k, n, _stream())
    return ac, br


def rc_flag_words(batch: int, m: int, n: int):
    return batch * ((m + 1 + 31) // 32), batch * ((n + 1 + 31) // 32)


def ne_abft_rc_check(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, ac: torch.Tensor, br: torch.Tensor,
                     work: torch.Tensor | None = None, row_bad: torch.Tensor | None = None,
                     col_bad: torch.Tensor | None = None, nbad: torch.Tensor | None = None):
    """C int64 [batch, m, n] -> (work, row_bad, col_bad)."""
    batch, m, k = A.shape
    n = B.shape[1]
    if tuple(C.shape) != (batch, m, n):
        raise ValueError("C must be [batch, m, n]")
    if work is None:
        work = torch.empty((batch, 2 * (m + n + 1)), dtype=torch.int64, device=C.device)
    rw, cw = rc_flag_words(batch, m, n)
    if row_bad is None:
        row_bad = torch.empty(rw, dtype=torch.int32, device=C.device)
    if col_bad is None:
        col_bad = torch.empty(cw, dtype=torch.int32, device=C.device)
    _call("ne_abft_rc_check", _ptr(C, torch.int64, "C"), _ptr(A, torch.int32, "A"), _ptr(B, torch.int8, "B"),
          _ptr(ac, torch.int64, "ac"), _ptr(br, torch.int64, "br"), _ptr(work, torch.int64, "work"),
          _ptr(row_bad, torch.int32, "row_bad"), _ptr(col_bad, torch.int32, "col_bad"),
          _ptr(nbad, torch.int64, "nbad", True), batch, m, k, n, _stream())
    return work, row_bad, col_bad


def ne_abft_rc_correct(C: torch.Tensor, work: torch.Tensor, row_bad: torch.Tensor, col_bad: torch.Tensor,
                       ncorrected: torch.Tensor | None = None) -> torch.Tensor:
    batch, m, n = C.shape
    _call("ne_abft_rc_correct", _ptr(C, torch.int64, "C"), _ptr(work, torch.int64, "work"),
          _ptr(row_bad, torch.int32, "row_bad"), _ptr(col_bad, torch.int32, "col_bad"),
          _ptr(ncorrected, torch.int64, "ncorrected", True), batch, m, n, _stream())
    return C


# ---- the other LSB operators of Eq. 2 ----------------------------------------------

NE_OP_ADD, NE_OP_SUB, NE_OP_MUL = 0, 1, 2


def _operand_stride(g: torch.Tensor, batch: int, length: int) -> int:
    """g is one operand [length] shared by every group, or [batch, length]."""
    if g.dim() == 1 and g.shape[0] == length:
        return 0
    if tuple(g.shape) == (batch, length):
        return length
    raise ValueError(f"operand must be [{length}] or [{batch}, {length}], got {tuple(g.shape)}")


def ne_elementwise(p: ne_params, op: int, eps: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
                   flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
                   fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0) -> torch.Tensor:
    """eps int64 [..., M, n]; g int64 [n] or [batch, n] -> int64 like eps."""
    batch, n = _bmn(eps, p.M)
    gs = _operand_stride(g, batch, n)
    if out is None:
        out = torch.empty_like(eps)
    _call("ne_elementwise", p, op, _ptr(eps, torch.int64, "eps"), _ptr(g, torch.int64, "g"), gs,
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, n, fuse, r, _stream())
    return out


def ne_entangle_kernel_self(l: int, g: torch.Tensor, ge: torch.Tensor | None = None) -> torch.Tensor:
    if ge is None:
        ge = torch.empty_like(g)
    _call("ne_entangle_kernel_self", l, _ptr(g, torch.int64, "g"), _ptr(ge, torch.int64, "ge"), g.numel(),
          _stream())
    return ge


def ne_outer(p: ne_params, eps: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
             flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
             fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0) -> torch.Tensor:
    """eps int64 [batch, M, n]; g int64 [k] or [batch, k] -> int64 [batch, M, n, k]."""
    batch, M, n = eps.shape
    if M != p.M:
        raise ValueError("eps must be [batch, M, n]")
    k = g.shape[-1]
    gs = _operand_stride(g, batch, k)
    if out is None:
        out = torch.empty((batch, M, n, k), dtype=torch.int64, device=eps.device)
    _call("ne_outer", p, _ptr(eps, torch.int64, "eps"), _ptr(g, torch.int64, "g"), gs,
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, n, k, fuse, r, _stream())
    return out


def ne_permute(p: ne_params, eps: torch.Tensor, perm: torch.Tensor, out: torch.Tensor | None = None,
               flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
               fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0, status: torch.Tensor | None = None) -> torch.Tensor:
    """eps int64 [..., M, n]; perm int32 [n] -> int64 like eps (out[..., i] = eps[..., perm[i]])."""
    batch, n = _bmn(eps, p.M)
    if tuple(perm.shape) != (n,):
        raise ValueError("perm must be [n]")
    if out is None:
        out = torch.empty_like(eps)
    _call("ne_permute", p, _ptr(eps, torch.int64, "eps"), _ptr(perm, torch.int32, "perm"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, n, fuse, r, _ptr(status, torch.int32, "status", True),
          _stream())
    return out


def ne_inner(p: ne_params, eps: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None,
             flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None,
             fuse: int = NE_FUSE_EXTRACT_CHECK, r: int = 0) -> torch.Tensor:
    """eps int64 [..., M, n]; g int64 [n] or [batch, n] -> int64 [..., M]."""
    batch, n = _bmn(eps, p.M)
    gs = _operand_stride(g, batch, n)
    if out is None:
        out = torch.empty(tuple(eps.shape[:-1]), dtype=torch.int64, device=eps.device)
    _call("ne_inner", p, _ptr(eps, torch.int64, "eps"), _ptr(g, torch.int64, "g"), gs,
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), batch, n, fuse, r, _stream())
    return out


def ne_reverse_operand(g: torch.Tensor, g_rev: torch.Tensor | None = None) -> torch.Tensor:
    """g int8 [batch, N] -> g_rev[b, j] = g[b, (N - j) mod N]."""
    batch, N = g.shape
    if g_rev is None:
        g_rev = torch.empty_like(g)
    _call("ne_reverse_operand", _ptr(g, torch.int8, "g"), _ptr(g_rev, torch.int8, "g_rev"), batch, N, _stream())
    return g_rev


# ---- extraction / check / recovery ---------------------------------------------

def flag_words(batch: int, n: int) -> int:
    return batch * ((n + 31) // 32)


def ne_extract(p: ne_params, delta: torch.Tensor, d_hat: torch.Tensor | None = None, r: int = 0,
               flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None) -> torch.Tensor:
    batch, n = _bmn(delta, p.M)
    if d_hat is None:
        d_hat = torch.empty_like(delta)
    _call("ne_extract", p, _ptr(delta, torch.int64, "delta"), _ptr(d_hat, torch.int64, "d_hat"), batch, n, r,
          _ptr(flags, torch.int32, "flags", True), _ptr(nflag, torch.int64, "nflag", True), _stream())
    return d_hat


def ne_check(p: ne_params, delta: torch.Tensor, r: int = 0, flags: torch.Tensor | None = None,
             nflag: torch.Tensor | None = None, status: torch.Tensor | None = None):
    batch, n = _bmn(delta, p.M)
    if flags is None:
        flags = torch.empty(flag_words(batch, n), dtype=torch.int32, device=delta.device)
    _call("ne_check", p, _ptr(delta, torch.int64, "delta"), batch, n, r, _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), _ptr(status, torch.int32, "status", True), _stream())
    return flags


def ne_check_set_wait_limit(polls: int = 1 << 22):
    """Test support: polls of the first wait of each block of ne_check's staged kernel."""
    _call("ne_check_set_wait_limit", polls)


def ne_recover(p: ne_params, delta: torch.Tensor, r_lost: int, d_hat: torch.Tensor | None = None) -> torch.Tensor:
    batch, n = _bmn(delta, p.M)
    if d_hat is None:
        d_hat = torch.empty_like(delta)
    _call("ne_recover", p, _ptr(delta, torch.int64, "delta"), _ptr(d_hat, torch.int64, "d_hat"), batch, n, r_lost,
          _stream())
    return d_hat


def ne_inject(delta: torch.Tensor, P: int, group, pos, stream, bit, status: torch.Tensor | None = None):
    """delta int64 [batch, P, n]; fault lists int64 device tensors of equal length."""
    batch, n = _bmn(delta, P)
    count = group.numel()
    for t in (pos, stream, bit):
        if t.numel() != count:
            raise ValueError("fault lists differ in length")
    _call("ne_inject", _ptr(delta, torch.int64, "delta"), P, batch, n, _ptr(group, torch.int64, "group"),
          _ptr(pos, torch.int64, "pos"), _ptr(stream, torch.int64, "stream"), _ptr(bit, torch.int64, "bit"),
          count, _ptr(status, torch.int32, "status", True), _stream())


# ---- checksum ABFT ---------------------------------------------------------------

def ne_abft_encode(M: int, c: torch.Tensor, x: torch.Tensor | None = None) -> torch.Tensor:
    batch, n = _bmn(c, M)
    shape = tuple(c.shape[:-2]) + (M + 1, n)
    if x is None:
        x = torch.empty(shape, dtype=torch.int64, device=c.device)
    _call("ne_abft_encode", M, _ptr(c, torch.int32, "c"), _ptr(x, torch.int64, "x"), batch, n, _stream())
    return x


def ne_abft_check(M: int, d: torch.Tensor, flags: torch.Tensor | None = None, nflag: torch.Tensor | None = None):
    batch, n = _bmn(d, M + 1)
    if flags is None:
        flags = torch.empty(flag_words(batch, n), dtype=torch.int32, device=d.device)
    _call("ne_abft_check", M, _ptr(d, torch.int64, "d"), batch, n, _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), _stream())
    return flags


def ne_abft_recover(M: int, d: torch.Tensor, j: int) -> torch.Tensor:
    batch, n = _bmn(d, M + 1)
    _call("ne_abft_recover", M, _ptr(d, torch.int64, "d"), batch, n, j, _stream())
    return d


# ---- ragged batches -------------------------------------------------------------------

JOB_DTYPE = None   # numpy structured dtype with the layout of ne_job (set below)


def _job_array(jobs):
    """(pointer, count) of a ctypes ne_job array or a numpy JOB_DTYPE array."""
    if isinstance(jobs, ctypes.Array):
        return jobs, len(jobs)
    import numpy as np
    a = np.ascontiguousarray(jobs)
    if a.dtype != JOB_DTYPE:
        raise TypeError("jobs must be ne_job structures or a JOB_DTYPE array")
    return ctypes.cast(a.ctypes.data, ctypes.POINTER(ne_job)), len(a)


def ne_batch_plan(jobs, cfg: ne_batch_config, workspace: torch.Tensor | None = None,
                  staging: torch.Tensor | None = None) -> ne_batch_info:
    """jobs: a ctypes array of ne_job or a numpy JOB_DTYPE array (host).
    With workspace None only sizes the plan (info.workspace_bytes,
    info.table_bytes); otherwise writes the tables into it (uint8 device
    tensor, 256-byte aligned) by a copy ordered on the current stream: run the
    batch on the same stream.  staging: a pinned uint8 host tensor of at least
    info.table_bytes bytes to build the tables in and upload them from without
    the host waiting (keep it untouched until the run on the stream is done)."""
    info = ne_batch_info()
    ws_ptr, ws_bytes = None, 0
    if workspace is not None:
        ws_ptr = _ptr(workspace, torch.uint8, "workspace")
        ws_bytes = workspace.numel()
    ptr, n = _job_array(jobs)
    if staging is None:
        _call("ne_batch_plan", ptr, n, cfg, ws_ptr, ws_bytes, ctypes.byref(info), _stream())
    else:
        if staging.is_cuda or not staging.is_pinned() or staging.dtype != torch.uint8 or not staging.is_contiguous():
            raise ValueError("staging must be a contiguous pinned uint8 host tensor")
        _call("ne_batch_plan_staged", ptr, n, cfg, ws_ptr, ws_bytes, ctypes.c_void_p(staging.data_ptr()),
              staging.numel(), ctypes.byref(info), _stream())
    return info


def ne_copy_regions_h2d(dst: torch.Tensor, src: torch.Tensor, dst_off, src_off, nbytes):
    """Byte regions of the pinned host tensor src into the device tensor dst
    (offsets and sizes in bytes, int64 numpy arrays)."""
    import numpy as np
    if not dst.is_cuda or src.is_cuda or not src.is_pinned():
        raise ValueError("dst must be a CUDA tensor and src a pinned host tensor")
    d = np.ascontiguousarray(dst_off, np.int64)
    s_ = np.ascontiguousarray(src_off, np.int64)
    b = np.ascontiguousarray(nbytes, np.int64)
    if not (len(d) == len(s_) == len(b)):
        raise ValueError("region lists differ in length")
    if len(b) and (int((d + b).max()) > dst.numel() * dst.element_size() or
                   int((s_ + b).max()) > src.numel() * src.element_size()):
        raise ValueError("a region lies outside its tensor")
    _call("ne_copy_regions_h2d", ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(src.data_ptr()),
          ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(s_.ctypes.data), ctypes.c_void_p(b.ctypes.data),
          len(b), _stream())


def ne_batch_run(info: ne_batch_info, c: torch.Tensor, ops: torch.Tensor, out: torch.Tensor,
                 flags: torch.Tensor | None, nflag: torch.Tensor | None, workspace: torch.Tensor,
                 fault_pos: torch.Tensor | None = None, fault_stream: torch.Tensor | None = None,
                 fault_bit: torch.Tensor | None = None, status: torch.Tensor | None = None):
    _call("ne_batch_run", info, _ptr(c, torch.int32, "c"), _ptr(ops, torch.int8, "ops"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), _ptr(fault_pos, torch.int64, "fault_pos", True),
          _ptr(fault_stream, torch.int32, "fault_stream", True), _ptr(fault_bit, torch.int32, "fault_bit", True),
          _ptr(workspace, torch.uint8, "workspace"), _ptr(status, torch.int32, "status", True), _stream())


def ne_batch_run_static(jobs, cfg: ne_batch_config, c: torch.Tensor, ops: torch.Tensor, out: torch.Tensor,
                        flags: torch.Tensor | None, nflag: torch.Tensor | None,
                        fault_pos: torch.Tensor | None = None, fault_stream: torch.Tensor | None = None,
                        fault_bit: torch.Tensor | None = None, status: torch.Tensor | None = None):
    """Plan and run a batch with the library's static scratch array (no device
    memory is allocated); see include/ne.h for the size limit and sharing."""
    _call("ne_batch_run_static", jobs, len(jobs), cfg, _ptr(c, torch.int32, "c"), _ptr(ops, torch.int8, "ops"),
          _ptr(out, torch.int64, "out"), _ptr(flags, torch.int32, "flags", True),
          _ptr(nflag, torch.int64, "nflag", True), _ptr(fault_pos, torch.int64, "fault_pos", True),
          _ptr(fault_stream, torch.int32, "fault_stream", True), _ptr(fault_bit, torch.int32, "fault_bit", True),
          _ptr(status, torch.int32, "status", True), _stream())


def _make_job_dtype():
    import numpy as np
    fields = [(name, np.int32 if t is ctypes.c_int32 else np.int64) for name, t in ne_job._fields_]
    dt = np.dtype(fields, align=True)
    assert dt.itemsize == ctypes.sizeof(ne_job), "ne_job layout"
    return dt


JOB_DTYPE = _make_job_dtype()
