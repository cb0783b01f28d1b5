"""Autotuner of the ragged batch runner.

Searches the launch configuration of a batch -- resident blocks per SM of
the persistent launch, tile order (job order or costliest first), the width
of the convolution tiles, the l policy that sets each job's digit count
(the "slice count": byte-aligned l gives two digits for int8 streams, the
smallest l may need three), and the length from which convolutions run as
exact transforms instead of tensor tiles -- by timing each candidate on the
GPU with CUDA events, and caches the winner per job-mix signature in a JSON
file.
"""
from __future__ import annotations

import hashlib
import itertools
import json
import os

import torch

from . import batch as B
from . import ne

CACHE = os.environ.get("NE_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ne_gb300", "autotune.json"))


SEARCH_SPACE = "v2: ctas 1-2, order, blocks 8/16, l policy, transform from N"


def signature(b: B.Batch) -> str:
    h = hashlib.sha256()
    h.update(SEARCH_SPACE.encode())
    for s in b.specs:
        h.update(f"{s.kind},{s.M},{s.rows},{s.cols},{s.k},{s.N},{s.fuse},{s.l};".encode())
    dev = torch.cuda.get_device_name(b.device)
    h.update(dev.encode())
    return h.hexdigest()[:20]


def candidates():
    # the tile shape and order first (tensor path only), then the transform threshold
    # on the best of them: 0 keeps every convolution on the tensor tiles
    for ctas, order, blocks, pol in itertools.product((1, 2), (ne.NE_ORDER_LPT, ne.NE_ORDER_JOB), (16, 8),
                                                      (ne.NE_L_BYTE, ne.NE_L_SMALLEST)):
        yield B.default_config(ctas_per_sm=ctas, order=order, cconv_blocks=blocks, l_policy=pol)


NTT_THRESHOLDS = (2048, 4096, 8192, 16384)


def _time(b: B.Batch, iters: int) -> float:
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        b.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / iters


def tune(b: B.Batch, iters: int = 2, use_cache: bool = True, verbose: bool = False):
    """Returns (best config, {config-string: ms}).  Leaves b planned with the best."""
    key = signature(b)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        try:
            cache = json.load(open(CACHE))
        except Exception:
            cache = {}
    if use_cache and key in cache:
        cfg = B.default_config(**cache[key]["config"])
        b.plan(cfg)
        return cfg, cache[key].get("trials", {})
    trials = {}
    best = None
    for cfg in candidates():
        name = json.dumps(B.config_dict(cfg), sort_keys=True)
        try:
            b.plan(cfg)
        except ne.NEError as e:
            trials[name] = f"infeasible: {e}"
            continue
        ms = _time(b, iters)
        trials[name] = ms
        if verbose:
            print(f"autotune {name}: {ms:.3f} ms", flush=True)
        if best is None or ms < best[0]:
            best = (ms, cfg)
    if best is None:
        raise RuntimeError("no feasible batch configuration")
    base = B.config_dict(best[1])
    for thr in NTT_THRESHOLDS:
        cfg = B.default_config(**{**base, "ntt_min_n": thr})
        name = json.dumps(B.config_dict(cfg), sort_keys=True)
        try:
            b.plan(cfg)
        except ne.NEError as e:
            trials[name] = f"infeasible: {e}"
            continue
        ms = _time(b, iters)
        trials[name] = ms
        if verbose:
            print(f"autotune {name}: {ms:.3f} ms", flush=True)
        if ms < best[0]:
            best = (ms, cfg)
    b.plan(best[1])
    if use_cache:
        cache[key] = {"config": B.config_dict(best[1]), "ms": best[0], "trials": trials}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    return best[1], trials
