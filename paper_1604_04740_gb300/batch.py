"""Ragged batches of entangled jobs through the C ABI (ne_batch_plan /
ne_batch_run): job-mix generation, arena packing, seeded inputs, transient
fault lists, planning, running and CUDA-graph capture.

A batch is a list of independent jobs -- matrix products and circular
convolutions of M entangled streams with their own sizes -- executed by one
entangle launch and ONE persistent launch over all tiles.  This module only
prepares memory and calls the library; no job arithmetic happens here.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np
import torch

from . import inputs
from . import ne


@dataclasses.dataclass
class JobSpec:
    kind: int                 # ne.NE_JOB_GEMM or ne.NE_JOB_CCONV
    M: int
    rows: int = 0
    cols: int = 0
    k: int = 0
    N: int = 0
    fuse: int = ne.NE_FUSE_EXTRACT_CHECK
    r: int = 0
    l: int = 0                # 0: the plan chooses l from the job's bound
    plain: int = 0            # 1: the plain operation on the raw streams (fuse must be NONE)

    @property
    def positions_in(self) -> int:
        return self.rows * self.k if self.kind == ne.NE_JOB_GEMM else self.N

    @property
    def positions_out(self) -> int:
        return self.rows * self.cols if self.kind == ne.NE_JOB_GEMM else self.N

    @property
    def op_bytes(self) -> int:
        return self.k * self.cols if self.kind == ne.NE_JOB_GEMM else self.N

    @property
    def useful_ops(self) -> int:
        if self.kind == ne.NE_JOB_GEMM:
            return 2 * self.M * self.rows * self.cols * self.k
        return 2 * self.M * self.N * self.N


def mixed_jobs(seed: int, njobs: int = 2048, mnk=(32, 2048), conv=(256, 65536), recover_frac: float = 0.0):
    """The ragged job mix: M uniform in {3, 4, 5}; half products with m, n, k
    log-uniform in [mnk], half circular convolutions with N log-uniform in
    [conv], every size used exactly as drawn.  A fraction recover_frac of
    jobs loses one stream (uniform)."""
    T = inputs.TAG_JOBS
    Ms = (inputs.u64(seed, T, 0, njobs) % np.uint64(3)).astype(np.int64) + 3
    keys = inputs.u64(seed, T, njobs, njobs)
    kinds = np.zeros(njobs, np.int64)
    kinds[np.argsort(keys, kind="stable")[: njobs // 2]] = ne.NE_JOB_CCONV
    rows = inputs.log_uniform_int(seed, T, 2 * njobs, njobs, *mnk)
    cols = inputs.log_uniform_int(seed, T, 3 * njobs, njobs, *mnk)
    ks = inputs.log_uniform_int(seed, T, 4 * njobs, njobs, *mnk)
    Ns = inputs.log_uniform_int(seed, T, 5 * njobs, njobs, *conv)
    lost = inputs.unit_float(seed, T, 6 * njobs, njobs) < recover_frac
    lost_r = inputs.u64(seed, T, 7 * njobs, njobs)
    specs = []
    for i in range(njobs):
        M = int(Ms[i])
        fuse = ne.NE_FUSE_RECOVER if lost[i] else ne.NE_FUSE_EXTRACT_CHECK
        r = int(lost_r[i] % np.uint64(M)) if lost[i] else 0
        if kinds[i] == ne.NE_JOB_GEMM:
            specs.append(JobSpec(ne.NE_JOB_GEMM, M, rows=int(rows[i]), cols=int(cols[i]), k=int(ks[i]), fuse=fuse,
                                 r=r))
        else:
            specs.append(JobSpec(ne.NE_JOB_CCONV, M, N=int(Ns[i]), fuse=fuse, r=r))
    return specs


def _align(x, q):
    return (x + q - 1) // q * q


class Batch:
    """Device arenas, job table, inputs and optional faults of one batch.

    Arenas: c int32 (streams [M][positions] per job), ops int8 (G [k][cols] or
    g [N]), out int64 (d_hat [M][positions]), flags int32 (one bitmap per job).
    Inputs are the seeded streams/operators of `seed` (values in [-128, 127]);
    job j's streams are the counters c_off .. of TAG_C, its operator the
    counters op_off .. of TAG_G.
    """

    def __init__(self, specs, seed: int = 0, fault_rate: float = 0.0, fault_seed: int = 1,
                 device="cuda", cmin: int = -128, cmax: int = 127, generate: bool = True):
        self.specs = list(specs)
        self.seed = seed
        self.device = torch.device(device)
        self.cmin, self.cmax = cmin, cmax
        n = len(self.specs)
        self.jobs = (ne.ne_job * n)()
        c_off = op_off = out_off = flag_off = 0
        for j, s in enumerate(self.specs):
            jb = self.jobs[j]
            jb.kind, jb.M, jb.l = s.kind, s.M, s.l
            jb.rows, jb.cols, jb.k, jb.N = s.rows, s.cols, s.k, s.N
            jb.r, jb.fuse, jb.cmin, jb.cmax, jb.plain = s.r, s.fuse, cmin, cmax, s.plain
            jb.c_off, jb.op_off, jb.out_off, jb.flag_off = c_off, op_off, out_off, flag_off
            c_off = _align(c_off + s.M * s.positions_in, 4)
            op_off = _align(op_off + s.op_bytes, 16)
            out_off += s.M * s.positions_out
            flag_off += (s.positions_out + 31) // 32
        self.sizes = dict(c=c_off, ops=op_off, out=out_off, flags=flag_off)
        dev = self.device
        self.c = torch.zeros(max(c_off, 4), dtype=torch.int32, device=dev)
        self.ops = torch.zeros(max(op_off, 16), dtype=torch.int8, device=dev)
        self.out = torch.empty(max(out_off, 1), dtype=torch.int64, device=dev)
        self.flags = torch.empty(max(flag_off, 1), dtype=torch.int32, device=dev)
        self.nflag = torch.zeros(1, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        if generate:
            self._generate()
        self.faults = None
        if fault_rate > 0:
            self._faults(fault_rate, fault_seed)
        self.workspace = None
        self.info = None
        self.graph = None

    # -- data ------------------------------------------------------------------------
    def _generate(self):
        if self.cmin == -128 and self.cmax == 127:
            # int8-valued streams: one pass over the arena, widened on the device
            self.c.copy_(inputs.int8_uniform_device(self.seed, inputs.TAG_C, self.c.numel(), 0, self.device))
        else:
            for j, s in enumerate(self.specs):
                jb = self.jobs[j]
                n = s.M * s.positions_in
                v = inputs.int32_uniform(self.seed, inputs.TAG_C, (n,), self.cmin, self.cmax, start=jb.c_off)
                self.c[jb.c_off:jb.c_off + n].copy_(torch.from_numpy(v))
        self.ops.copy_(inputs.int8_uniform_device(self.seed, inputs.TAG_G, self.ops.numel(), 0, self.device))

    def job_inputs(self, j):
        """Host copies of job j's streams ([M, rows, k] or [1, M, N]) and operator."""
        s, jb = self.specs[j], self.jobs[j]
        c = self.c[jb.c_off:jb.c_off + s.M * s.positions_in].cpu().numpy()
        op = self.ops[jb.op_off:jb.op_off + s.op_bytes].cpu().numpy()
        if s.kind == ne.NE_JOB_GEMM:
            return c.reshape(s.M, s.rows, s.k), op.reshape(s.k, s.cols)
        return c.reshape(1, s.M, s.N), op.reshape(1, s.N)

    def job_output(self, j):
        s, jb = self.specs[j], self.jobs[j]
        o = self.out[jb.out_off:jb.out_off + s.M * s.positions_out]
        if s.kind == ne.NE_JOB_GEMM:
            return o.view(s.M, s.rows, s.cols)
        return o.view(1, s.M, s.N)

    def job_flags(self, j):
        s, jb = self.specs[j], self.jobs[j]
        return self.flags[jb.flag_off:jb.flag_off + (s.positions_out + 31) // 32]

    # -- transient faults --------------------------------------------------------------
    def _faults(self, rate, seed):
        """One bit flip per 1/rate output words: distinct (job, position)
        pairs, uniform stream and bit; only jobs that are checked get faults."""
        checked = [j for j, s in enumerate(self.specs) if s.fuse == ne.NE_FUSE_EXTRACT_CHECK]
        sizes = np.array([self.specs[j].positions_out for j in checked], np.int64)
        words = int(sum(self.specs[j].M * self.specs[j].positions_out for j in checked))
        count = int(words * rate)
        if count == 0 or not checked:
            return
        starts = np.concatenate([[0], np.cumsum(sizes)])
        g, pos, _, bit = inputs.fault_list(seed, 1, int(starts[-1]), 1, count)
        flat = pos
        jidx = np.searchsorted(starts, flat, side="right") - 1
        local = flat - starts[jidx]
        extra = inputs.u64(seed, inputs.TAG_FAULT + 2000, 0, count)
        Ms = np.array([self.specs[checked[i]].M for i in jidx], np.int64)
        stream = (extra % Ms.astype(np.uint64)).astype(np.int64)
        jobs = np.array([checked[i] for i in jidx], np.int64)
        order = np.lexsort((local, jobs))
        jobs, local, stream, bit = jobs[order], local[order], stream[order], bit[order]
        for j in range(len(self.specs)):
            self.jobs[j].fault_begin = self.jobs[j].fault_end = 0
        b = np.searchsorted(jobs, np.arange(len(self.specs)), side="left")
        e = np.searchsorted(jobs, np.arange(len(self.specs)), side="right")
        for j in range(len(self.specs)):
            self.jobs[j].fault_begin, self.jobs[j].fault_end = int(b[j]), int(e[j])
        self.faults = dict(job=jobs, pos=local, stream=stream, bit=bit)
        self.fault_dev = (torch.from_numpy(local).to(self.device),
                          torch.from_numpy(stream.astype(np.int32)).to(self.device),
                          torch.from_numpy(bit.astype(np.int32)).to(self.device))

    # -- plan / run ----------------------------------------------------------------------
    def plan(self, cfg: ne.ne_batch_config):
        info = ne.ne_batch_plan(self.jobs, cfg)
        need = info.workspace_bytes
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        ws = self.workspace
        off = (-ws.data_ptr()) % 256
        self.ws_view = ws[off:off + need]
        self.info = ne.ne_batch_plan(self.jobs, cfg, self.ws_view)
        self.graph = None
        return self.info

    def run(self):
        fp = self.fault_dev if self.faults is not None else (None, None, None)
        ne.ne_batch_run(self.info, self.c, self.ops, self.out, self.flags, self.nflag, self.ws_view, *fp,
                        status=self.status)

    def capture(self):
        """Capture run() into a CUDA graph (after one eager run)."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def useful_ops(self) -> int:
        return sum(s.useful_ops for s in self.specs)


def default_config(**kw) -> ne.ne_batch_config:
    cfg = ne.ne_batch_config()
    cfg.ctas_per_sm = kw.get("ctas_per_sm", 2)
    cfg.order = kw.get("order", ne.NE_ORDER_LPT)
    cfg.cconv_blocks = kw.get("cconv_blocks", 16)
    cfg.l_policy = kw.get("l_policy", ne.NE_L_BYTE)
    cfg.ntt_min_n = kw.get("ntt_min_n", 0)
    return cfg


def config_dict(cfg: ne.ne_batch_config) -> dict:
    return {f: getattr(cfg, f) for f, _ in cfg._fields_}


def expected_flags(batch: Batch, j: int):
    """uint8 [positions] with 1 where a fault was injected into job j."""
    s = batch.specs[j]
    f = np.zeros(s.positions_out, np.uint8)
    if batch.faults is not None:
        sel = batch.faults["job"] == j
        f[batch.faults["pos"][sel]] = 1
    return f


def log2_ceil(x):
    return int(math.ceil(math.log2(max(1, x))))
