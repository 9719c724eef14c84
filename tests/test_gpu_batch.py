"""Batched and served correlation on the GPU: one CUDA graph over several
uneven scans gives, per scan, exactly what the scan gives alone; the served
mix gives each job exactly what it gets alone; the batch agrees with the
FP64 oracle; the memory estimate matches what the library allocates."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_FP16 = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr, serve
    dev = torch.device("cuda", 0)
    pool = serve.ReplayPool(64 << 20, dev, seed=3)
    return torch, corr, serve, dev, pool


def small_mix(count=6, seed=11):
    return synth.scan_mix(seed=seed, count=count, stations=(2, 7), nsub=(1, 3), npol=(1, 2),
                          log2_nchan=(6, 10), duration=(0.004, 0.03), tint_max=0.008)


def attach(c, sc, pool, key):
    for s in range(sc.stations):
        c.attach_device(s, pool.view(key * 1024 + s + 1, sc.nsamp[s] * sc.G // 4))
    c.flush()


def alone(env, sc, key, precision):
    torch, corr, serve, dev, pool = env
    c = corr.from_scan(sc)
    c.set_precision(precision)
    attach(c, sc, pool, key)
    outs = []
    for _ in range(synth.integrations(sc)):
        o = torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device=dev)
        w = torch.empty(sc.nbl, dtype=torch.float64, device=dev)
        assert c.correlate_device(o, w) == corr.CORR_OK
        outs.append((o, w))
    torch.cuda.synchronize()
    c.close()
    return [(o.cpu().numpy(), w.cpu().numpy()) for o, w in outs]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone(env, precision):
    """Six scans of 2-7 stations, 1-6 streams, 64-1024 channels and 1-4
    integrations in one graph per step: bit-identical to each scan alone."""
    torch, corr, serve, dev, pool = env
    mix = small_mix()
    ref = [alone(env, sc, q, precision) for q, sc in enumerate(mix)]
    cs = []
    for q, sc in enumerate(mix):
        c = corr.from_scan(sc)
        c.set_precision(precision)
        attach(c, sc, pool, q)
        cs.append(c)
    nint = [synth.integrations(sc) for sc in mix]
    got = [[] for _ in mix]
    for step in range(max(nint)):
        live = [q for q in range(len(mix)) if step < nint[q]]
        outs = [torch.empty((mix[q].nbl, mix[q].G, mix[q].nchan), dtype=torch.complex64, device=dev) for q in live]
        ws = [torch.empty(mix[q].nbl, dtype=torch.float64, device=dev) for q in live]
        corr.batch_run([cs[q] for q in live], outs, ws)
        torch.cuda.synchronize()
        for q, o, w in zip(live, outs, ws):
            got[q].append((o.cpu().numpy(), w.cpu().numpy()))
    for q in range(len(mix)):
        assert cs[q].next_integration() == nint[q]
        cs[q].close()
        for i in range(nint[q]):
            assert np.array_equal(got[q][i][1], ref[q][i][1])
            assert np.array_equal(got[q][i][0].view(np.uint64), ref[q][i][0].view(np.uint64)), (q, i)


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, TOL_FP16)])
def test_batch_against_oracle(env, precision, tol):
    """Two scans of the mix, batched, against the FP64 oracle on the same
    bytes."""
    torch, corr, serve, dev, pool = env
    mix = small_mix(count=2, seed=12)
    cs, refs = [], []
    for q, sc in enumerate(mix):
        c = corr.from_scan(sc)
        c.set_precision(precision)
        attach(c, sc, pool, 50 + q)
        cs.append(c)
        streams = [pool.view((50 + q) * 1024 + s + 1, sc.nsamp[s] * sc.G // 4).cpu().numpy()
                   for s in range(sc.stations)]
        refs.append(oracle.Oracle.from_scan(sc, streams).correlate(0, 1))
    outs = [torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device=dev) for sc in mix]
    ws = [torch.empty(sc.nbl, dtype=torch.float64, device=dev) for sc in mix]
    corr.batch_run(cs, outs, ws)
    torch.cuda.synchronize()
    for sc, o, w, (ref, wref), c in zip(mix, outs, ws, refs, cs):
        c.close()
        assert np.array_equal(w.cpu().numpy(), wref[0])
        v = o.cpu().numpy().reshape(sc.nbl, -1)
        r = ref[0].reshape(sc.nbl, -1)
        err = np.sqrt(np.sum(np.abs(v - r) ** 2, axis=1) / np.sum(np.abs(r) ** 2, axis=1))
        assert np.all(err < tol), err.max()


def test_served_mix_equals_alone(env):
    """Jobs served with staggered arrivals (continuous batching, tensor-core
    precision) return, per integration, exactly what each returns served
    alone."""
    torch, corr, serve, dev, pool = env
    mix = small_mix(count=5, seed=13)

    def run(jobs, rates):
        res = {}

        def keep(job, i, out, w):
            res[(job.jid, i)] = (out.numpy().copy(), w.numpy().copy())

        ex = serve.GpuExecutor(corr, dev, pool, 1, on_result=keep)
        sch = serve.Scheduler(ex, cap=8e9, reserve=1e9)
        st = sch.run(jobs)
        return res, st

    # two jobs at once, the rest arriving while those run
    arrive = [0.0, 0.0] + [0.0005 * q for q in range(1, len(mix) - 1)]
    mixed, st = run([serve.Job(q, sc, arrival=arrive[q], precision=1) for q, sc in enumerate(mix)], None)
    assert st["jobs"] == len(mix) and st["max_batch"] >= 2
    assert st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    for q, sc in enumerate(mix):
        solo, _ = run([serve.Job(q, sc, arrival=0.0, precision=1)], None)
        for i in range(synth.integrations(sc)):
            a, b = mixed[(q, i)], solo[(q, i)]
            assert np.array_equal(a[1], b[1])
            assert np.array_equal(a[0].view(np.uint64), b[0].view(np.uint64)), (q, i)


def test_batch_argument_errors(env):
    torch, corr, serve, dev, pool = env
    sc = small_mix(count=1, seed=14)[0]
    c = corr.from_scan(sc)
    attach(c, sc, pool, 7)
    o = torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device=dev)
    with pytest.raises(corr.CorrError) as ei:
        corr.batch_run([c, c], [o, o])
    assert ei.value.code == corr.CORR_EINVAL
    d = corr.from_scan(sc)  # not flushed
    with pytest.raises(corr.CorrError) as ei:
        corr.batch_run([d], [o])
    assert ei.value.code == corr.CORR_ESTATE
    # a failed call leaves the handle usable
    corr.batch_run([c], [o])
    torch.cuda.synchronize()
    assert c.next_integration() == 1
    c.close()
    d.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_device_bytes_matches_allocation(env, precision):
    """corr_device_bytes, asked before the first correlate, matches the drop
    in free device memory that preparing the handle causes (to allocation
    granularity)."""
    torch, corr, serve, dev, pool = env
    sc = synth.config2(seed=2, duration=0.1, tint=0.05, boundary=0.05)
    c = corr.from_scan(sc)
    c.set_precision(precision)
    attach(c, sc, serve.ReplayPool(max(sc.nsamp) * sc.G // 4 + (1 << 20), dev), 0)
    est = c.device_bytes()
    o = torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    assert c.correlate_device(o) == corr.CORR_OK
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info(dev)[0]
    c.close()
    assert abs(used - est) <= 64 << 20, (used, est)
    c2 = corr.from_scan(sc)
    c2.set_precision(precision)
    c2.set_chunk_blocks(64)
    assert c2.device_bytes() < est
    c2.close()
