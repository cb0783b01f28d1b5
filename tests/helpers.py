"""Shared test helpers (no method arithmetic)."""
import numpy as np


def unpack_flags(words, batch, n):
    """uint32 bitmap words [batch * ceil(n/32)] -> uint8 [batch, n]."""
    w = np.ascontiguousarray(np.asarray(words).view(np.uint32))
    wpr = (n + 31) // 32
    bits = np.unpackbits(w.view(np.uint8), bitorder="little").reshape(batch, wpr * 32)
    return bits[:, :n]


def pack_flags(flags):
    """uint8 [batch, n] -> uint32 words [batch * ceil(n/32)] (bits past n are 0)."""
    flags = np.asarray(flags, np.uint8)
    batch, n = flags.shape
    wpr = (n + 31) // 32
    pad = np.zeros((batch, wpr * 32), np.uint8)
    pad[:, :n] = flags
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint32).reshape(-1)
