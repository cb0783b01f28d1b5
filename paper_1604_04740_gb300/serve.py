"""Continuous-batching serving loop for entangled jobs on one GPU.

Requests (jobs of the ragged-batch distribution) arrive over time.  The
server admits them in arrival order whenever their device memory fits in the
free part of an HBM budget, and launches the admitted requests as a
micro-batch (ne_batch_plan + ne_batch_run) on the next free executor lane (a
CUDA stream) -- so requests that arrive while others are running are
admitted as soon as a lane and memory free up, and their work overlaps on
the device with the batches already in flight.  Entangled state (digit
planes, outputs, check bitmaps) lives in device memory carved from one
pre-allocated pool; a micro-batch's region returns to the pool when it
completes.  A request that lost one stream (fail-stop) runs with the fused
recovery and needs only the other M-1 streams.

Per micro-batch the host work is vectorised (numpy job tables handed to the
C planner, one native call issuing the requests' host->device copies), so
the loop keeps up with tens of thousands of requests per second.

Latency of a request = completion of its micro-batch, observed on the host,
minus its arrival time.  Outputs stay in device memory (the device-resident
result); only the batch status and flag count return to the host.

A serving process should start CUDA with CUDA_MODULE_LOADING=EAGER: with
lazy loading, the first launch of each kernel the warm-up did not reach
loads its module inside the loop and stalls that micro-batch.
"""
from __future__ import annotations

import bisect
import dataclasses
import gc
import time

import numpy as np
import torch

from . import batch as B
from . import inputs
from . import ne


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate: cumulative
    exponential gaps -ln(1 - U) / rate."""
    u = inputs.unit_float(seed, inputs.TAG_ARRIVAL, 0, n)
    return np.cumsum(-np.log1p(-u) / rate)


class Pool:
    """First-fit allocator over one device buffer (offsets aligned to 256)."""

    def __init__(self, nbytes: int, device):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.base = (-self.buf.data_ptr()) % 256
        self.size = nbytes - self.base
        self.free = [(0, self.size)]      # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes: int):
        nbytes = (nbytes + 255) // 256 * 256
        for i, (off, ln) in enumerate(self.free):
            if ln >= nbytes:
                if ln == nbytes:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + nbytes, ln - nbytes)
                self.used += nbytes
                return off, nbytes
        return None

    def release(self, off: int, nbytes: int):
        self.used -= nbytes
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, nbytes))
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)

    def view(self, off: int, nbytes: int, dtype):
        a = self.base + off
        return self.buf[a:a + nbytes].view(dtype)


def _a(x, q=256):
    return (x + q - 1) // q * q


@dataclasses.dataclass
class Request:
    idx: int
    spec: B.JobSpec
    arrival: float
    c_pool: int = 0           # offset of its streams in the host input pool (int32 elements)
    op_pool: int = 0          # offset of its operator in the host operator pool (bytes)
    done: float = -1.0


def work_estimate(T, ntt_min_n: int) -> np.ndarray:
    """Rough device work of each request of table T, in int8 tensor-op
    equivalents: 2 M S m n k for a product and 2 M S N^2 for a convolution on
    tensor tiles (S = 2 digit planes per stream for the entangled form, 1 for
    the plain one), and 280 (2 M + 1) N log2 N for a convolution on the
    transform path (N >= ntt_min_n, or N not a multiple of 64) (the factor from the ragged batch, where
    528 such convolutions take as long as 4.1e11 tile ops)."""
    S = np.where(T.plain != 0, 1.0, 2.0)
    M = T.M.astype(np.float64)
    N = T.N.astype(np.float64)
    gemm = 2.0 * M * S * T.rows * T.cols * T.k
    tiles = 2.0 * M * S * N * N
    ntt = 280.0 * (2.0 * M + 1.0) * N * np.log2(np.maximum(N, 2.0))
    conv = np.where(((ntt_min_n > 0) & (T.N >= ntt_min_n)) | (T.N % 64 != 0), ntt, tiles)
    return np.where(T.kind == ne.NE_JOB_GEMM, gemm, conv)


class _Table:
    """Per-request numpy columns of one run()."""

    def __init__(self, specs, c_pool, op_pool, ntt_min_n: int = 0):
        G = ne.NE_JOB_GEMM
        self.kind = np.array([s.kind for s in specs], np.int32)
        self.M = np.array([s.M for s in specs], np.int32)
        self.l = np.array([s.l for s in specs], np.int32)
        self.rows = np.array([s.rows for s in specs], np.int32)
        self.cols = np.array([s.cols for s in specs], np.int32)
        self.k = np.array([s.k for s in specs], np.int32)
        self.N = np.array([s.N for s in specs], np.int32)
        self.r = np.array([s.r for s in specs], np.int32)
        self.fuse = np.array([s.fuse for s in specs], np.int32)
        self.plain = np.array([s.plain for s in specs], np.int32)
        gemm = self.kind == G
        pin = np.where(gemm, self.rows.astype(np.int64) * self.k, self.N.astype(np.int64))
        pout = np.where(gemm, self.rows.astype(np.int64) * self.cols, self.N.astype(np.int64))
        self.c_elems = self.M * pin
        self.op_bytes = np.where(gemm, self.k.astype(np.int64) * self.cols, self.N.astype(np.int64))
        self.out_elems = self.M * pout
        self.flag_words = (pout + 31) // 32
        # rough device work per request (work_estimate), cumulated for the admission cap
        self.cum_work = np.concatenate([[0.0], np.cumsum(work_estimate(self, ntt_min_n))])
        self.c_pool = np.asarray(c_pool, np.int64)
        self.op_pool = np.asarray(op_pool, np.int64)


class Server:
    def __init__(self, budget_bytes: int, lanes: int = 4, max_batch: int = 256, device="cuda",
                 cfg: ne.ne_batch_config | None = None, host_pool_elems: int = 1 << 27, seed: int = 0,
                 keep_outputs: bool = False, max_batch_work: float | None = None):
        self.device = torch.device(device)
        self.pool = Pool(budget_bytes, self.device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(lanes)]
        self.max_batch = max_batch
        # admission also stops once a micro-batch's estimated work (work_estimate)
        # would pass this: the persistent launches of a long micro-batch fill every
        # SM, so the ones behind it on other lanes wait for all of it
        self.max_batch_work = max_batch_work
        self.cfg = cfg or B.default_config()
        self.keep_outputs = keep_outputs
        # pinned host pools the requests' inputs come from
        self.c_host = torch.from_numpy(inputs.int32_uniform_int8range(seed, inputs.TAG_C, (host_pool_elems,))).pin_memory()
        self.op_host = torch.from_numpy(inputs.int8_uniform(seed, inputs.TAG_G, (host_pool_elems // 4,))).pin_memory()
        self.outputs = {}
        # per-lane pinned words for the batch status and flag count (read without touching
        # the default stream, which would wait for every lane)
        self.status_h = [torch.zeros(1, dtype=torch.int32).pin_memory() for _ in range(lanes)]
        # pinned per-lane staging for the plan tables: their upload never waits for the
        # copy engines (a lane plans again only after its previous batch is done).  8 MiB
        # holds the tables of about half a million tiles, so the loop itself rarely has
        # to pin a larger buffer (a pinned allocation can take tens of milliseconds)
        self.staging = [torch.empty(8 << 20, dtype=torch.uint8).pin_memory() for _ in range(lanes)]
        self.nflag_h = [torch.zeros(1, dtype=torch.int64).pin_memory() for _ in range(lanes)]
        self.flagged = 0
        # host-side timing of the last run: the longest loop iteration and the
        # longest micro-batch launch (plan, copies, kernel launches), in seconds
        self.max_iter_s = 0.0
        self.max_launch_s = 0.0
        self.max_phase_s = {"plan": 0.0, "copy": 0.0, "run": 0.0}
        # the longest device span of a micro-batch (events on its lane, from before its
        # input copies to after its status read) and how many requests it held, and
        # the longest input-copy and kernel parts of a micro-batch
        self.max_device_s = 0.0
        self.max_device_requests = 0
        self.max_copy_span_s = 0.0
        self.max_kernel_span_s = 0.0

    # -- one micro-batch: requests [a, b) ------------------------------------------------
    def _launch(self, T: _Table, a: int, b: int, lane: int):
        n = b - a
        jobs = np.zeros(n, ne.JOB_DTYPE)
        for f in ("kind", "M", "l", "rows", "cols", "k", "N", "r", "fuse", "plain"):
            jobs[f] = getattr(T, f)[a:b]
        jobs["cmin"], jobs["cmax"] = -128, 127
        c_sz = (T.c_elems[a:b] + 3) // 4 * 4
        op_sz = (T.op_bytes[a:b] + 15) // 16 * 16
        c_off = np.concatenate([[0], np.cumsum(c_sz)[:-1]])
        op_off = np.concatenate([[0], np.cumsum(op_sz)[:-1]])
        out_off = np.concatenate([[0], np.cumsum(T.out_elems[a:b])[:-1]])
        flag_off = np.concatenate([[0], np.cumsum(T.flag_words[a:b])[:-1]])
        jobs["c_off"], jobs["op_off"], jobs["out_off"], jobs["flag_off"] = c_off, op_off, out_off, flag_off
        n_c, n_op = int(c_sz.sum()), int(op_sz.sum())
        n_out, n_fl = int(T.out_elems[a:b].sum()), int(T.flag_words[a:b].sum())
        t_p = time.perf_counter()
        info = ne.ne_batch_plan(jobs, self.cfg)
        parts = [_a(n_c * 4 + 16), _a(n_op + 16), _a(max(n_out, 1) * 8), _a(max(n_fl, 1) * 4), 256, 256,
                 _a(info.workspace_bytes)]
        got = self.pool.alloc(sum(parts))
        if got is None:
            return None
        off, nb = got
        starts = np.concatenate([[off], off + np.cumsum(parts)[:-1]])
        v = self.pool.view
        c = v(int(starts[0]), parts[0], torch.int32)
        ops = v(int(starts[1]), parts[1], torch.int8)
        out = v(int(starts[2]), parts[2], torch.int64)
        flags = v(int(starts[3]), parts[3], torch.int32)
        nflag = v(int(starts[4]), 256, torch.int64)[:1]
        status = v(int(starts[5]), 256, torch.int32)[:1]
        ws = v(int(starts[6]), parts[6], torch.uint8)
        stream = self.streams[lane]
        if self.staging[lane].numel() < info.table_bytes:
            self.staging[lane] = torch.empty(2 * info.table_bytes, dtype=torch.uint8).pin_memory()
        ev0 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            info = ne.ne_batch_plan(jobs, self.cfg, ws, staging=self.staging[lane])
            t_c = time.perf_counter()
            ne.ne_copy_regions_h2d(c, self.c_host, c_off * 4, T.c_pool[a:b] * 4, T.c_elems[a:b] * 4)
            ne.ne_copy_regions_h2d(ops, self.op_host, op_off, T.op_pool[a:b], T.op_bytes[a:b])
            evc = torch.cuda.Event(enable_timing=True)
            evc.record(stream)
            t_r = time.perf_counter()
            status.zero_()
            ne.ne_batch_run(info, c, ops, out, flags, nflag, ws, status=status)
            self.status_h[lane].copy_(status, non_blocking=True)
            self.nflag_h[lane].copy_(nflag, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        t_e = time.perf_counter()
        for phase, dt in (("plan", t_c - t_p), ("copy", t_r - t_c), ("run", t_e - t_r)):
            self.max_phase_s[phase] = max(self.max_phase_s[phase], dt)
        return dict(ev0=ev0, evc=evc, ev=ev, region=(off, nb), a=a, b=b, out=out, out_off=out_off, lane=lane)

    def _finish(self, fl, T: _Table, reqs, t):
        for i in range(fl["a"], fl["b"]):
            reqs[i].done = t
        lane = fl["lane"]
        dev_s = fl["ev0"].elapsed_time(fl["ev"]) * 1e-3
        if dev_s > self.max_device_s:
            self.max_device_s, self.max_device_requests = dev_s, fl["b"] - fl["a"]
        self.max_copy_span_s = max(self.max_copy_span_s, fl["ev0"].elapsed_time(fl["evc"]) * 1e-3)
        self.max_kernel_span_s = max(self.max_kernel_span_s, fl["evc"].elapsed_time(fl["ev"]) * 1e-3)
        if int(self.status_h[lane][0]) != 0:
            raise RuntimeError("a request's inputs left the planned value range")
        self.flagged += int(self.nflag_h[lane][0])
        if self.keep_outputs:
            with torch.cuda.stream(self.streams[lane]):
                for j, i in enumerate(range(fl["a"], fl["b"])):
                    o = int(fl["out_off"][j])
                    self.outputs[reqs[i].idx] = fl["out"][o:o + int(T.out_elems[i])].cpu().numpy()
        self.pool.release(*fl["region"])

    # -- the loop -------------------------------------------------------------------------
    def run(self, specs, arrivals, seed: int = 0, offsets=None, timeout_s: float = 600.0):
        """Serve the requests; returns the list of Request with their times.
        Request i takes its inputs from the host pools at seeded offsets, or
        at offsets[i] = (stream offset, operator offset) when given."""
        n = len(specs)
        rng_c = inputs.u64(seed, inputs.TAG_ARRIVAL + 1, 0, n)
        reqs = []
        for i, s in enumerate(specs):
            span_c = self.c_host.numel() - s.M * s.positions_in
            span_o = self.op_host.numel() - s.op_bytes
            if span_c < 0 or span_o < 0:
                raise ValueError(f"request {i} is larger than the host input pool")
            if offsets is not None:
                co, oo = offsets[i]
            else:
                co, oo = int(rng_c[i] % np.uint64(span_c + 1)), int(rng_c[i] % np.uint64(span_o + 1))
            reqs.append(Request(i, s, float(arrivals[i]), c_pool=co, op_pool=oo))
        T = _Table(specs, [rq.c_pool for rq in reqs], [rq.op_pool for rq in reqs], self.cfg.ntt_min_n)
        # no cyclic garbage collection inside the loop: a full collection can
        # stall the host for tens of milliseconds, which shows up as latency
        gc_on = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return self._loop(T, reqs, arrivals, n, timeout_s)
        finally:
            if gc_on:
                gc.enable()

    def _loop(self, T, reqs, arrivals, n, timeout_s):
        inflight = []
        free_lanes = list(range(len(self.streams)))
        head = nxt = done = 0          # requests [head, nxt) have arrived and wait for admission
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        arr = np.asarray(arrivals, np.float64) + t0
        for i, rq in enumerate(reqs):
            rq.arrival = float(arr[i])
        self.max_iter_s = self.max_launch_s = 0.0
        self.max_phase_s = {"plan": 0.0, "copy": 0.0, "run": 0.0}
        self.max_device_s, self.max_device_requests = 0.0, 0
        self.max_copy_span_s = self.max_kernel_span_s = 0.0
        last = time.perf_counter()
        while done < n:
            now = time.perf_counter()
            self.max_iter_s = max(self.max_iter_s, now - last)
            last = now
            nxt = int(np.searchsorted(arr, now, side="right"))
            still = []
            for fl in inflight:
                if fl["ev"].query():
                    self._finish(fl, T, reqs, time.perf_counter())
                    done += fl["b"] - fl["a"]
                    free_lanes.append(fl["lane"])
                else:
                    still.append(fl)
            inflight = still
            if head < nxt and free_lanes:
                b = min(nxt, head + self.max_batch)
                if self.max_batch_work:
                    # the longest prefix within the work cap, at least one request
                    cap = T.cum_work[head] + self.max_batch_work
                    j = int(np.searchsorted(T.cum_work, cap, side="right")) - 1
                    b = max(head + 1, min(b, j))
                fl = None
                while b > head:
                    t_l = time.perf_counter()
                    fl = self._launch(T, head, b, free_lanes[0])
                    self.max_launch_s = max(self.max_launch_s, time.perf_counter() - t_l)
                    if fl is not None:
                        break
                    b = head + (b - head) // 2          # does not fit the free budget: admit fewer
                if fl is not None:
                    free_lanes.pop(0)
                    inflight.append(fl)
                    head = b
                elif not inflight:
                    raise RuntimeError(f"request {head} does not fit the HBM budget even alone")
            elif not inflight and head == nxt and nxt < n:
                dt = arr[nxt] - time.perf_counter()
                if dt > 2e-4:
                    time.sleep(dt - 1e-4)
            if time.perf_counter() - t0 > timeout_s:
                raise RuntimeError(f"serving did not finish within {timeout_s} s ({done} of {n} done)")
        torch.cuda.synchronize(self.device)
        return reqs


def summarize(reqs):
    lat = np.array([rq.done - rq.arrival for rq in reqs])
    first = min(rq.arrival for rq in reqs)
    last = max(rq.done for rq in reqs)
    useful = sum(rq.spec.useful_ops for rq in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "jobs_per_s": len(reqs) / (last - first), "useful_Gop_s": useful / (last - first) / 1e9,
            "lost_stream_requests": sum(1 for rq in reqs if rq.spec.fuse == ne.NE_FUSE_RECOVER)}


def plain_copy(specs):
    """The same requests without entanglement (the unprotected comparison)."""
    return [dataclasses.replace(s, fuse=ne.NE_FUSE_NONE, plain=1, r=0) for s in specs]
