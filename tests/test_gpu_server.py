"""The native continuous-batching server (corr_server_*) on the GPU.

Two jobs of different shapes served together give, integration by
integration, exactly (bit for bit) what each gives alone through the
handle path, and match the FP64 oracle within 1e-5; the same holds when the
memory cap admits only one job at a time (the second waits and joins when
the first leaves).  A job that cannot fit even alone gets one callback with
CORR_ENOMEM.  The latency statistics cover every finished job.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr
    torch.cuda.set_device(0)
    scans = [synth.config2(seed=31, duration=0.006, tint=0.002, boundary=0.003, nchan=256, stations=3, nsub=1,
                           npol=2),
             synth.config2(seed=32, duration=0.008, tint=0.004, boundary=0.004, nchan=512, stations=5, nsub=2,
                           npol=2)]
    host = [[synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)] for sc in scans]
    dev = [[torch.from_numpy(b).cuda() for b in h] for h in host]
    alone = []
    for sc, d in zip(scans, dev):
        c = corr.from_scan(sc, device_streams=d)
        c.flush()
        nint = synth.integrations(sc)
        out = torch.empty((nint, sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device="cuda")
        w = torch.empty((nint, sc.nbl), dtype=torch.float64, device="cuda")
        for i in range(nint):
            assert c.correlate_device(out[i], w[i]) == corr.CORR_OK
        torch.cuda.synchronize()
        alone.append((out.cpu().numpy(), w.cpu().numpy()))
        c.close()
    return torch, corr, scans, host, dev, alone


def serve(corr, scans, dev, cap, reserve):
    got = {}
    lock = threading.Lock()

    def on_result(job_id, integration, vis, w, status):
        with lock:
            got.setdefault(job_id, []).append((integration, vis, w, status))

    srv = corr.Server(cap, reserve, on_result)
    statics = [corr.StaticScan(sc, d) for sc, d in zip(scans, dev)]
    ids = [srv.submit(st, synth.integrations(sc)) for st, sc in zip(statics, scans)]
    assert srv.wait(120.0) == corr.CORR_OK
    stats = srv.stats()
    srv.close()
    return ids, got, stats


def check_against_alone(scans, ids, got, alone):
    for sc, jid, (ref, wref) in zip(scans, ids, alone):
        res = sorted(got[jid], key=lambda r: r[0])
        assert [r[0] for r in res] == list(range(synth.integrations(sc)))
        for i, vis, w, status in res:
            assert status == 0
            assert np.array_equal(w, wref[i])
            assert np.array_equal(vis.reshape(sc.nbl, sc.G, sc.nchan), ref[i])


def test_two_jobs_served_together_equal_alone(env):
    torch, corr, scans, host, dev, alone = env
    ids, got, stats = serve(corr, scans, dev, 8 << 30, 1 << 30)
    check_against_alone(scans, ids, got, alone)
    assert stats["jobs_done"] == 2 and stats["p99_s"] >= stats["p50_s"] > 0 and stats["station_samples_per_s"] > 0
    # and the mix against the FP64 oracle
    for sc, h, jid in zip(scans, host, ids):
        ref, wref = oracle.Oracle.from_scan(sc, h).correlate(0, synth.integrations(sc))
        for i, vis, w, _ in got[jid]:
            v = vis.reshape(sc.nbl, sc.G, sc.nchan)
            err = np.sqrt(np.sum(np.abs(v - ref[i]) ** 2, axis=(1, 2)) / np.sum(np.abs(ref[i]) ** 2, axis=(1, 2)))
            assert np.array_equal(w, wref[i]) and np.all(err < 1e-5)


def test_cap_admits_one_job_at_a_time(env):
    torch, corr, scans, host, dev, alone = env
    need = []
    for sc, d in zip(scans, dev):
        c = corr.from_scan(sc, device_streams=d)
        need.append(c.device_bytes() + sc.nbl * sc.G * sc.nchan * 8 + sc.nbl * 8)
        c.close()
    reserve = 1 << 20
    ids, got, stats = serve(corr, scans, dev, max(need) + reserve + 1024, reserve)
    check_against_alone(scans, ids, got, alone)
    assert stats["jobs_done"] == 2


def test_job_larger_than_the_cap_fails_cleanly(env):
    torch, corr, scans, host, dev, alone = env
    ids, got, stats = serve(corr, scans[:1], dev[:1], (1 << 20) + 4096, 1 << 20)
    assert len(got[ids[0]]) == 1
    i, vis, w, status = got[ids[0]][0]
    assert status == corr.CORR_ENOMEM and vis is None and w is None
    assert stats["jobs_done"] == 1
