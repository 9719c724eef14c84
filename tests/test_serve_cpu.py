"""Host logic of the batch/serve layer, without a GPU: admission by memory
budget, arrival-order admission, continuous batching, retirement, latency
percentiles, the Poisson arrival process and the uneven scan mix."""
import math

import numpy as np
import pytest

import synth
from paper_1502_06894_gb300 import serve


class FakeScan:
    def __init__(self, duration, tint=1.0, stations=2, nsub=1, npol=1, fs=1000.0, nchan=4):
        self.duration, self.tint, self.stations, self.nsub, self.npol, self.fs, self.nchan = (
            duration, tint, stations, nsub, npol, fs, nchan)


class FakeExecutor:
    """Each job needs `mem` bytes; a step costs `cost` seconds of virtual time
    whatever the batch holds.  Records every batch and every open/close."""

    def __init__(self, mem, cost=1.0):
        self.mem = mem
        self.cost = cost
        self.batches = []
        self.open_now = set()
        self.opened = []
        self.max_bytes = 0
        self.bytes = 0

    def job_bytes(self, job):
        return self.mem[job.jid]

    def open(self, job):
        assert job.jid not in self.open_now
        self.open_now.add(job.jid)
        self.opened.append(job.jid)
        self.bytes += self.mem[job.jid]
        self.max_bytes = max(self.max_bytes, self.bytes)

    def step(self, jobs):
        assert all(j.jid in self.open_now for j in jobs)
        self.batches.append([j.jid for j in jobs])
        return self.cost

    def close(self, job):
        self.open_now.remove(job.jid)
        self.bytes -= self.mem[job.jid]


def test_admission_never_exceeds_budget():
    rng = np.random.default_rng(7)
    n = 60
    mem = {i: int(rng.integers(1, 40)) * 10 ** 9 for i in range(n)}
    arr = sorted(rng.uniform(0, 30, n))
    jobs = [serve.Job(i, FakeScan(float(rng.integers(1, 6))), arrival=float(arr[i])) for i in range(n)]
    ex = FakeExecutor(mem, cost=0.5)
    sch = serve.Scheduler(ex, cap=180e9, reserve=30e9, fixed=8e9, virtual=True)
    st = sch.run(jobs)
    assert st["jobs"] == n and st["rejected"] == 0
    assert ex.max_bytes <= 142e9 and st["peak_bytes"] <= st["limit_bytes"] == 142e9
    assert not ex.open_now and ex.bytes == 0
    # every job ran exactly as many steps as it has integrations
    for j in jobs:
        assert sum(j.jid in b for b in ex.batches) == j.nint == int(j.scan.duration)


def test_admission_in_arrival_order_and_oversize_rejected():
    mem = {0: 100, 1: 60, 2: 10, 3: 500}
    jobs = [serve.Job(i, FakeScan(2.0), arrival=0.1 * i) for i in range(4)]
    ex = FakeExecutor(mem)
    sch = serve.Scheduler(ex, cap=200, reserve=50, virtual=True)
    st = sch.run(jobs)
    # job 3 cannot fit even alone; job 2 may not overtake job 1, which waits for job 0
    assert st["rejected"] == 1 and sch.rejected[0].jid == 3
    assert ex.opened == [0, 1, 2]
    assert ex.batches[0] == [0]
    assert 1 not in ex.batches[1] and ex.batches[2] == [1, 2]


def test_continuous_batching_and_latency():
    """A job that arrives while another is running joins the next step; the
    latencies follow from the virtual step clock."""
    mem = {0: 1, 1: 1}
    jobs = [serve.Job(0, FakeScan(4.0), arrival=0.0), serve.Job(1, FakeScan(2.0), arrival=1.5)]
    ex = FakeExecutor(mem, cost=1.0)
    sch = serve.Scheduler(ex, cap=10, reserve=0, virtual=True)
    st = sch.run(jobs)
    # steps end at t = 1, 2, 3, 4; job 1 arrives at 1.5 and is admitted at t = 2
    assert ex.batches == [[0], [0], [0, 1], [0, 1]]
    assert jobs[0].finished == 4.0 and jobs[1].finished == 4.0
    assert jobs[1].admitted == 2.0
    assert st["p50_s"] == 2.5 and st["p99_s"] == 4.0
    assert st["max_batch"] == 2 and st["steps"] == 4


def test_max_active_limits_the_batch():
    mem = {i: 1 for i in range(5)}
    jobs = [serve.Job(i, FakeScan(1.0), arrival=0.0) for i in range(5)]
    ex = FakeExecutor(mem)
    st = serve.Scheduler(ex, cap=100, reserve=0, max_active=2, virtual=True).run(jobs)
    assert [len(b) for b in ex.batches] == [2, 2, 1] and st["jobs"] == 5


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert serve.percentile(xs, 50) == 50 and serve.percentile(xs, 99) == 99
    assert serve.percentile([3.0], 99) == 3.0 and serve.percentile([], 50) is None


def test_poisson_arrivals():
    a = serve.poisson_arrivals(40.0, 120.0, seed=5)
    assert a == serve.poisson_arrivals(40.0, 120.0, seed=5)
    assert all(x < y for x, y in zip(a, a[1:])) and a[-1] < 120.0
    n = len(a)
    assert abs(n - 4800) < 5 * math.sqrt(4800)
    gaps = np.diff([0.0] + a)
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() - 1 / 40) < 0.1 / 40 and abs(gaps.std() / gaps.mean() - 1) < 0.1


def test_scan_mix_shapes():
    mix = synth.scan_mix(seed=4, count=96)
    assert len(mix) == 96
    for sc in mix:
        assert 2 <= sc.stations <= 20 and 1 <= sc.nsub <= 16 and sc.npol in (1, 2)
        assert sc.nchan in [1 << k for k in range(7, 14)]
        spi = sc.fs * sc.tint
        assert abs(spi - round(spi)) < 1e-6 and round(spi) % (2 * sc.nchan) == 0 and sc.tint <= 1.0 + 1e-9
        n = synth.integrations(sc)
        assert abs(n * sc.tint - sc.duration) < 1e-9 and 0.49 < sc.duration < 30.01
        assert len(sc.sample0) == sc.stations
    # reproducible
    b = synth.scan_mix(seed=4, count=96)
    assert [(s.stations, s.nsub, s.npol, s.nchan, s.duration) for s in mix] == \
        [(s.stations, s.nsub, s.npol, s.nchan, s.duration) for s in b]


class FakeCorr:
    """Stands in for the library binding: handles record their settings; the
    memory a handle needs grows with its chunk length."""
    CORR_OK = 0
    CORR_PREC_FP32, CORR_PREC_FP16_TC, CORR_PREC_FP8_TC = 0, 1, 2
    CORR_X_AUTO, CORR_X_CUDA_CORES, CORR_X_TENSOR_CORES = 0, 1, 2

    def __init__(self, bytes_per_block):
        self.bytes_per_block = bytes_per_block
        self.made = []

    def from_scan(self, scan):
        corr = self

        class H:
            def __init__(self):
                self.cfg = {}
                corr.made.append(self)

            def set_precision(self, p): self.cfg["prec"] = p
            def set_x_unit(self, u): self.cfg["unit"] = u
            def set_chunk_blocks(self, cb): self.cfg["cb"] = cb
            def device_bytes(self): return self.cfg["cb"] * corr.bytes_per_block
            def attach_device(self, s, view): pass
            def flush(self): pass
            def close(self): pass
        return H()


class FakePool:
    def view(self, off, n):
        return None


class TuneScan:
    stations, nsub, npol, nchan, fs, tint, G, nbl = 4, 2, 1, 256, 512e3, 1.0, 2, 10
    nsamp = [512000] * 4


def test_autotuner_picks_the_fastest_chunk_and_x_unit_and_caches_it():
    corr = FakeCorr(bytes_per_block=1 << 20)
    # a fake timing table: the CUDA cores are faster at long chunks only
    table = {(64, 1): 5.0, (256, 1): 3.0, (1001, 1): 1.5, (64, 2): 4.0, (256, 2): 2.0, (1001, 2): 2.5}

    def timer(c, out):
        return corr.CORR_OK, table[(c.cfg["cb"], c.cfg["unit"])]

    tuner = serve.Autotuner(corr, FakePool(), "cpu", mem_cap=1 << 40, timer=timer)
    sc = TuneScan()
    # 512e3 / 512 = 1000 blocks per integration, at most 1001 per chunk: candidates 64, 256, 1001
    assert tuner.config(sc, corr.CORR_PREC_FP16_TC) == (1001, corr.CORR_X_CUDA_CORES)
    assert tuner.trials == 6
    assert tuner.choose(sc, corr.CORR_PREC_FP16_TC) == 1001
    assert tuner.x_unit(sc, corr.CORR_PREC_FP16_TC) == corr.CORR_X_CUDA_CORES
    assert tuner.trials == 6  # cached


def test_autotuner_respects_the_memory_cap_and_fp32_has_one_unit():
    corr = FakeCorr(bytes_per_block=1 << 20)
    seen = []

    def timer(c, out):
        seen.append((c.cfg["cb"], c.cfg["unit"]))
        return corr.CORR_OK, 100.0 / c.cfg["cb"]  # longer chunks are faster

    # room for 300 blocks of work buffers (plus the output): the 1001-block candidate is skipped
    tuner = serve.Autotuner(corr, FakePool(), "cpu", mem_cap=300 << 20, timer=timer)
    cb, unit = tuner.config(TuneScan(), corr.CORR_PREC_FP32)
    assert (cb, unit) == (256, corr.CORR_X_AUTO)
    assert {u for _, u in seen} == {corr.CORR_X_AUTO}
    assert max(b for b, _ in seen) == 256
