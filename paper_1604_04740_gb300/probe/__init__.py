"""Binding of the benchmark's throughput probes (libne_probe.so, declared in
probe/ne_probe.h): each launches on the current CUDA stream and returns the
operations it issues; the caller times it with events."""
from __future__ import annotations

import ctypes
import os

import torch

from .. import build as _build

_lib = None


def _L():
    global _lib
    if _lib is None:
        path = _build.PROBE_LIB
        if not os.path.exists(path):
            _build.build()
        lib = ctypes.CDLL(path)
        i32, i64, P = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        for name, args in {"ne_probe_mma_peak": [i32, ctypes.POINTER(i64), P],
                           "ne_probe_dp4a_peak": [i32, ctypes.POINTER(i64), P],
                           "ne_probe_imad_peak": [i32, ctypes.POINTER(i64), P],
                           "ne_probe_mixed_peak": [i32, i32, i32, i32, i32, ctypes.POINTER(i64), P]}.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = i32
        _lib = lib
    return _lib


def _run(name, *args):
    ops = ctypes.c_int64(0)
    st = getattr(_L(), name)(*args, ctypes.byref(ops), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError(f"{name}: status {st}")
    return ops.value


def mma_peak(iters: int) -> int:
    return _run("ne_probe_mma_peak", iters)


def dp4a_peak(iters: int) -> int:
    return _run("ne_probe_dp4a_peak", iters)


def imad_peak(iters: int) -> int:
    return _run("ne_probe_imad_peak", iters)


def mixed_peak(iters_mma: int, iters_dp4a: int, mma_warps: int, dp4a_warps: int, blocks_per_sm: int) -> int:
    return _run("ne_probe_mixed_peak", iters_mma, iters_dp4a, mma_warps, dp4a_warps, blocks_per_sm)
