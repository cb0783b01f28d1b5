"""Autotuner of the ragged batch runner.

Searches the launch configuration of a batch -- resident blocks per SM of
the persistent launch, tile order (job order or costliest first), the width
of the convolution tiles, and the l policy that sets each job's digit count
(the "slice count": byte-aligned l gives two digits for int8 streams, the
smallest l may need three) -- by timing each candidate on the GPU with CUDA
events, and caches the winner per job-mix signature in a JSON file.
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


def signature(b: B.Batch) -> str:
    h = hashlib.sha256()
    for s in b.specs:
        h.update(f"{s.kind},{s.M},{s.rows},{s.cols},{s.k},{s.N},{s.fuse},{s.l};".encode())
    dev = torch.cuda.get_device_name(b.device)
    h.update(dev.encode())
    return h.hexdigest()[:20]


def candidates():
    for ctas, order, blocks, pol in itertools.product((1, 2), (ne.NE_ORDER_LPT, ne.NE_ORDER_JOB), (16, 8),
                                                      (ne.NE_L_BYTE, ne.NE_L_SMALLEST)):
        yield B.default_config(ctas_per_sm=ctas, order=order, cconv_blocks=blocks, l_policy=pol)


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
    b.plan(best[1])
    if use_cache:
        cache[key] = {"config": B.config_dict(best[1]), "ms": best[0], "trials": trials}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    return best[1], trials
