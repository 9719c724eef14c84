"""Device waits that give up: the X kernels' bounded mbarrier waits.

A process-wide test hook (corr_debug_set_wait_limit) sets the number of polls
before a wait of the X kernels gives up; 0 makes every such wait give up at
once, with nothing broken on the device.  A kernel whose wait gives up stops,
waits (with the default bound) for the bulk copies and tensor-core operations
it has in flight, frees its tensor memory and sets an error flag:
  * a handle reports CORR_ETIMEOUT, and keeps reporting it until corr_reset;
    after the reset it correlates correctly again;
  * corr_correlate_static, which has returned before the device work runs,
    makes every visibility of that call NaN; its next call is correct again.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def corr():
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr as c
    yield c
    c.corr_debug_set_wait_limit(-1)


@pytest.fixture(scope="module")
def scan():
    sc = synth.config2(seed=44, duration=0.004, tint=0.002, boundary=0.002, nchan=256, stations=4, nsub=1, npol=2)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    return sc, streams, ref, wref


def rel_rms_max(v, ref):
    v = v.reshape(ref.shape)
    return float(np.max(np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=(1, 2)) / np.sum(np.abs(ref) ** 2, axis=(1, 2)))))


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-3), (2, 8e-2)])
def test_timeout_reported_until_reset(corr, scan, precision, tol):
    sc, streams, ref, wref = scan
    c = corr.from_scan(sc, streams)
    c.set_precision(precision)
    corr.corr_debug_set_wait_limit(0)
    try:
        with pytest.raises(corr.CorrError) as ei:
            c.correlate()
        assert ei.value.code == corr.CORR_ETIMEOUT
    finally:
        corr.corr_debug_set_wait_limit(-1)
    with pytest.raises(corr.CorrError) as ei:   # still latched: no device work is done
        c.correlate()
    assert ei.value.code == corr.CORR_ETIMEOUT
    c.reset()
    for s, b in enumerate(streams):
        c.push(s, b)
    for i in range(2):
        r = c.correlate()
        assert r is not None
        assert np.array_equal(r[1], wref[i])
        assert rel_rms_max(r[0], ref[i]) < tol
    c.close()


def test_static_timeout_gives_nan_then_recovers(corr, scan):
    import torch
    sc, streams, ref, wref = scan
    dev = [torch.from_numpy(b).cuda() for b in streams]
    st = corr.StaticScan(sc, dev)
    out = torch.zeros((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device="cuda")
    corr.corr_debug_set_wait_limit(0)
    try:
        assert st.correlate(0, out) == corr.CORR_OK
        torch.cuda.synchronize()
    finally:
        corr.corr_debug_set_wait_limit(-1)
    assert torch.isnan(out.real).all() and torch.isnan(out.imag).all()
    w = torch.zeros(sc.nbl, dtype=torch.float64, device="cuda")
    assert st.correlate(0, out, w) == corr.CORR_OK
    torch.cuda.synchronize()
    assert np.array_equal(w.cpu().numpy(), wref[0])
    assert rel_rms_max(out.cpu().numpy(), ref[0]) < 1e-5
