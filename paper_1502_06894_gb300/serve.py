"""Many scans at once on one GPU: batched launches and a serving loop.

Batch.  The next integration of every open scan is recorded as parallel
branches of one CUDA graph and launched once (corr_batch_run).  Scans of
different station count, band layout, channel count and length share the
launch; each keeps its own work buffers, so its result does not depend on
what else is in the batch.

Serve.  A request loop admits correlation jobs while the sum of their device
working sets (corr_device_bytes plus the output slot) stays inside an HBM
budget, puts every admitted job into the very next batch (continuous
batching: a job that arrives while others are on the GPU joins them as soon
as memory allows), hands each integration's visibilities to the host as it
completes, and records every job's latency from arrival to its last result.

The scheduling logic is plain host code over an executor interface
(job_bytes / open / step / close), so it runs without a GPU against a fake
executor; GpuExecutor is the one that drives the library.  Station samples of
served jobs come from a device-resident pool of random 2-bit bytes that every
station of every job reads at its own offset (a replayed chunk: the reads
cost what fresh data would).
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Job:
    """One correlation request: a scan description (synth.Scan or anything
    with the same fields) and its arrival time in seconds from the start of
    the run."""
    jid: int
    scan: object
    arrival: float = 0.0
    precision: int = 0
    # set by the scheduler
    nint: int = 0
    done: int = 0
    nbytes: int = 0
    admitted: Optional[float] = None
    finished: Optional[float] = None

    @property
    def station_samples(self) -> float:
        sc = self.scan
        return float(sc.stations * sc.nsub * sc.npol * round(sc.fs * sc.tint) * self.nint)


def integrations_of(scan) -> int:
    return max(1, int(round(scan.duration / scan.tint)))


class Admission:
    """HBM budget: admit while used + need <= cap - reserve - fixed, where
    fixed is memory held for every job (a shared sample pool)."""

    def __init__(self, cap: float, reserve: float, fixed: float = 0.0):
        self.limit = int(cap - reserve - fixed)
        if self.limit <= 0:
            raise ValueError("HBM budget leaves no room for jobs")
        self.used = 0
        self.peak = 0

    def fits(self, n: int) -> bool:
        return self.used + n <= self.limit

    def take(self, n: int) -> None:
        if not self.fits(n):
            raise RuntimeError("admission over budget")
        self.used += n
        self.peak = max(self.peak, self.used)

    def give(self, n: int) -> None:
        self.used -= n
        if self.used < 0:
            raise RuntimeError("admission released more than it took")


def percentile(xs: Sequence[float], q: float) -> Optional[float]:
    """Nearest-rank percentile (q in 0..100)."""
    if not xs:
        return None
    s = sorted(xs)
    k = max(1, int(math.ceil(q / 100.0 * len(s))))
    return float(s[k - 1])


class Scheduler:
    """Continuous batching over an executor.

    Every round of the loop: move jobs whose arrival time has passed into the
    queue; admit queued jobs in arrival order while they fit the budget (and
    max_active, if set); run one step, which advances every active job by one
    integration; retire finished jobs and free their memory.  A job larger
    than the whole budget is rejected.  With virtual=True the clock is the
    executor's (no sleeping): arrivals are compared against the sum of step
    durations the executor reports, which makes runs reproducible."""

    def __init__(self, executor, cap: float, reserve: float, fixed: float = 0.0,
                 max_active: Optional[int] = None, virtual: bool = False):
        self.ex = executor
        self.adm = Admission(cap, reserve, fixed)
        self.max_active = max_active
        self.virtual = virtual
        self.vnow = 0.0
        self.steps = 0
        self.max_batch = 0
        self.rejected: List[Job] = []

    def _now(self, t0: float) -> float:
        return self.vnow if self.virtual else time.perf_counter() - t0

    def run(self, jobs: Sequence[Job]) -> Dict:
        pending = collections.deque(sorted(jobs, key=lambda j: (j.arrival, j.jid)))
        queue: collections.deque = collections.deque()
        active: List[Job] = []
        done: List[Job] = []
        t0 = time.perf_counter()
        busy = 0.0
        while pending or queue or active:
            now = self._now(t0)
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            while queue and (self.max_active is None or len(active) < self.max_active):
                j = queue[0]
                if not j.nbytes:
                    j.nint = integrations_of(j.scan)
                    j.nbytes = int(self.ex.job_bytes(j))
                if j.nbytes > self.adm.limit:
                    self.rejected.append(queue.popleft())
                    continue
                if not self.adm.fits(j.nbytes):
                    break
                self.adm.take(j.nbytes)
                self.ex.open(j)
                j.admitted = now
                active.append(j)
                queue.popleft()
            if not active:
                if pending:
                    wait = pending[0].arrival - self._now(t0)
                    if self.virtual:
                        self.vnow = max(self.vnow, pending[0].arrival)
                    elif wait > 0:
                        time.sleep(min(wait, 0.05))
                    continue
                if queue:
                    raise RuntimeError("queued job cannot be admitted with nothing active")
                break
            self.max_batch = max(self.max_batch, len(active))
            dt = self.ex.step(active)
            busy += dt if dt is not None else 0.0
            if self.virtual:
                self.vnow += dt
            self.steps += 1
            now = self._now(t0)
            keep = []
            for j in active:
                j.done += 1
                if j.done >= j.nint:
                    j.finished = now
                    self.ex.close(j)
                    self.adm.give(j.nbytes)
                    done.append(j)
                else:
                    keep.append(j)
            active = keep
        end = self._now(t0)
        lat = [j.finished - j.arrival for j in done]
        samples = sum(j.station_samples for j in done)
        first = min((j.arrival for j in jobs), default=0.0)
        return {
            "jobs": len(done), "rejected": len(self.rejected), "steps": self.steps,
            "max_batch": self.max_batch, "peak_bytes": self.adm.peak, "limit_bytes": self.adm.limit,
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99),
            "makespan_s": end - first, "station_samples": samples,
            "station_samples_per_s": samples / (end - first) if end > first else None,
            "busy_s": busy,
        }


def poisson_arrivals(rate: float, window: float, seed: int) -> List[float]:
    """Arrival times of a Poisson process of the given rate on [0, window)."""
    rng = np.random.Generator(np.random.Philox(key=0x5E7E_0000 + seed))
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= window:
            return out
        out.append(t)


# ----------------------------------------------------------------------------
# GPU executor


class ReplayPool:
    """One device buffer of random packed 2-bit bytes that stations read at
    their own 16-byte-aligned offsets."""

    def __init__(self, nbytes: int, device, seed: int = 0):
        import torch
        self.nbytes = (int(nbytes) // 16) * 16
        gen = torch.Generator(device=device)
        gen.manual_seed(0xB17E + seed)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        chunk = 1 << 28
        for o in range(0, self.nbytes, chunk):
            n = min(chunk, self.nbytes - o)
            self.buf[o:o + n] = torch.randint(0, 256, (n,), generator=gen, device=device, dtype=torch.int32).to(
                torch.uint8)

    def view(self, key: int, nbytes: int):
        if nbytes > self.nbytes:
            raise ValueError("station stream of %d bytes exceeds the sample pool (%d)" % (nbytes, self.nbytes))
        room = (self.nbytes - nbytes) // 16
        off = 16 * ((key * 0x9E3779B97F4A7C15 >> 20) % (room + 1))
        return self.buf[off:off + nbytes]


class Autotuner:
    """Chooses the F/X chunk length (spectra blocks per chunk) and, for the
    FP16 / FP8 modes, the X unit (CUDA cores or tensor cores) per scan shape
    by timing one integration per candidate with CUDA events, within a device
    memory cap per job.  Results are cached per (stations, streams, channels,
    blocks per integration, precision)."""

    CANDIDATES = (64, 256, 1024, 4096)

    def __init__(self, corr_mod, pool: ReplayPool, device, mem_cap: int, timer: Optional[Callable] = None):
        self.corr = corr_mod
        self.pool = pool
        self.dev = device
        self.mem_cap = int(mem_cap)
        self.cache: Dict[tuple, tuple] = {}  # key -> (chunk blocks, X unit)
        self.trials = 0
        # timer(handle, out) -> (return code, ms) of one integration; default: CUDA events
        self.timer = timer or self._time_cuda

    @staticmethod
    def _time_cuda(c, out):
        import torch
        c.correlate_device(out)  # warm: allocation and first launches
        torch.cuda.synchronize()
        c.rewind()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = c.correlate_device(out)
        e1.record()
        torch.cuda.synchronize()
        return rc, e0.elapsed_time(e1)

    def key(self, scan, precision):
        blocks = int(round(scan.fs * scan.tint)) // (2 * scan.nchan)
        return (scan.stations, scan.nsub * scan.npol, scan.nchan, blocks, precision)

    def choose(self, scan, precision) -> int:
        """Chunk length for the scan's shape (tuned on first use)."""
        return self.config(scan, precision)[0]

    def x_unit(self, scan, precision) -> int:
        """X unit for the scan's shape (tuned on first use)."""
        return self.config(scan, precision)[1]

    def config(self, scan, precision) -> tuple:
        import torch
        k = self.key(scan, precision)
        if k in self.cache:
            return self.cache[k]
        blocks = k[3] + 1
        cands = sorted({min(c, blocks) for c in self.CANDIDATES})
        units = (self.corr.CORR_X_AUTO,) if precision == self.corr.CORR_PREC_FP32 else \
            (self.corr.CORR_X_CUDA_CORES, self.corr.CORR_X_TENSOR_CORES)
        best, best_ms = (cands[0], units[0]), None
        out = torch.empty((scan.nbl, scan.nsub * scan.npol, scan.nchan), dtype=torch.complex64, device=self.dev)
        for cb, unit in [(cb, u) for cb in cands for u in units]:
            c = self.corr.from_scan(scan)
            try:
                c.set_precision(precision)
                c.set_x_unit(unit)
                c.set_chunk_blocks(cb)
                if c.device_bytes() + out.numel() * 8 > self.mem_cap and cb != cands[0]:
                    continue
                for s in range(scan.stations):
                    c.attach_device(s, self.pool.view(s + 1, scan.nsamp[s] * scan.G // 4))
                c.flush()
                rc, ms = self.timer(c, out)
                self.trials += 1
                if rc != self.corr.CORR_OK:
                    continue
                if best_ms is None or ms < best_ms:
                    best, best_ms = (cb, unit), ms
            finally:
                c.close()
        self.cache[k] = best
        return best


class GpuExecutor:
    """Runs admitted jobs through the library: one Correlator per job, its
    stations attached to the sample pool, one device output slot per job,
    and per step one corr_batch_run over all active jobs followed by the copy
    of every job's integration to pinned host memory (or a device-side
    callback when keep_on_device is set)."""

    def __init__(self, corr_mod, device, pool: ReplayPool, precision: int,
                 on_result: Optional[Callable] = None, tuner: Optional[Autotuner] = None,
                 chunk_blocks: Optional[int] = None, copy_results: bool = True, plain: bool = False):
        import torch
        self.plain = plain  # one corr_correlate_device per job instead of one graph per step
        self.corr = corr_mod
        self.dev = device
        self.pool = pool
        self.precision = precision
        self.on_result = on_result
        self.tuner = tuner
        self.chunk_blocks = chunk_blocks
        self.copy_results = copy_results
        self.stream = torch.cuda.Stream(device=device)
        self.state: Dict[int, dict] = {}

    def _make(self, job: Job):
        c = self.corr.from_scan(job.scan)
        c.set_precision(job.precision if job.precision is not None else self.precision)
        cb = self.chunk_blocks
        if cb is None and self.tuner is not None:
            cb, unit = self.tuner.config(job.scan, job.precision)
            c.set_x_unit(unit)
        if cb:
            c.set_chunk_blocks(cb)
        return c

    def job_bytes(self, job: Job) -> int:
        sc = job.scan
        c = self._make(job)
        self.state[job.jid] = {"c": c}
        out_bytes = sc.nbl * sc.nsub * sc.npol * sc.nchan * 8 + sc.nbl * 8
        return c.device_bytes() + out_bytes

    def open(self, job: Job) -> None:
        import torch
        sc = job.scan
        st = self.state.setdefault(job.jid, {})
        if "c" not in st:
            st["c"] = self._make(job)
        c = st["c"]
        for s in range(sc.stations):
            c.attach_device(s, self.pool.view(job.jid * 1024 + s + 1, sc.nsamp[s] * sc.G // 4))
        c.flush()
        G = sc.nsub * sc.npol
        st["out"] = torch.empty((sc.nbl, G, sc.nchan), dtype=torch.complex64, device=self.dev)
        st["w"] = torch.empty(sc.nbl, dtype=torch.float64, device=self.dev)
        if self.copy_results:
            st["out_h"] = torch.empty((sc.nbl, G, sc.nchan), dtype=torch.complex64, pin_memory=True)
            st["w_h"] = torch.empty(sc.nbl, dtype=torch.float64, pin_memory=True)

    def step(self, jobs: Sequence[Job]) -> float:
        import torch
        t0 = time.perf_counter()
        sts = [self.state[j.jid] for j in jobs]
        if self.plain:
            for s in sts:
                rc = s["c"].correlate_device(s["out"], s["w"])
                if rc != self.corr.CORR_OK:
                    raise RuntimeError("correlate_device returned %d" % rc)
            torch.cuda.synchronize()
        else:
            self.corr.batch_run([s["c"] for s in sts], [s["out"] for s in sts], [s["w"] for s in sts],
                                stream=self.stream.cuda_stream)
        if self.copy_results:
            with torch.cuda.stream(self.stream):
                for s in sts:
                    s["out_h"].copy_(s["out"], non_blocking=True)
                    s["w_h"].copy_(s["w"], non_blocking=True)
        self.stream.synchronize()
        if self.on_result is not None:
            for j, s in zip(jobs, sts):
                if self.copy_results:
                    self.on_result(j, j.done, s["out_h"], s["w_h"])
                else:
                    self.on_result(j, j.done, s["out"], s["w"])
        return time.perf_counter() - t0

    def close(self, job: Job) -> None:
        st = self.state.pop(job.jid, None)
        if st and "c" in st:
            st["c"].close()


def serial_run(corr_mod, device, pool: ReplayPool, jobs: Sequence[Job], precision: int,
               chunk_blocks: Optional[int] = None, tuner: Optional[Autotuner] = None,
               on_result: Optional[Callable] = None) -> float:
    """The per-scan baseline: each job on its own, one integration per
    corr_correlate_device call, jobs one after another.  Returns seconds."""
    import torch
    ex = GpuExecutor(corr_mod, device, pool, precision, tuner=tuner, chunk_blocks=chunk_blocks,
                     copy_results=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in jobs:
        j.nint = integrations_of(j.scan)
        ex.job_bytes(j)
        ex.open(j)
        st = ex.state[j.jid]
        for i in range(j.nint):
            rc = st["c"].correlate_device(st["out"], st["w"])
            if rc != corr_mod.CORR_OK:
                raise RuntimeError("correlate_device returned %d" % rc)
            if on_result is not None:
                torch.cuda.synchronize()
                on_result(j, i, st["out"], st["w"])
        torch.cuda.synchronize()
        ex.close(j)
    return time.perf_counter() - t0
