"""The native server's C ABI without a GPU: argument checks happen on the
caller's thread before any device work, an idle server reports empty
statistics, waits return at once and stop joins its worker thread."""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def corr():
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr as c
    return c


def test_server_start_checks_its_budget(corr):
    h = C.c_void_p()
    assert corr.corr_server_start(C.byref(h), 0, 0) == corr.CORR_EINVAL
    assert corr.corr_server_start(C.byref(h), 100, 100) == corr.CORR_EINVAL
    assert corr.corr_server_start(None, 100, 10) == corr.CORR_EINVAL
    assert not h.value


def test_idle_server_and_rejected_jobs(corr):
    h = C.c_void_p()
    assert corr.corr_server_start(C.byref(h), 1 << 30, 1 << 20) == corr.CORR_OK
    try:
        jid = C.c_int64(-5)
        cb = corr.RESULT_FN(lambda *a: None)
        # no job, and jobs whose shape or arrays are wrong: rejected before any device work
        assert corr.corr_server_submit(h, None, cb, None, C.byref(jid)) == corr.CORR_EINVAL
        job = corr.CorrJob()
        job.scan.stations, job.scan.subbands, job.scan.pols, job.scan.nchan = 2, 1, 1, 100
        job.scan.fs_hz, job.scan.tint_s = 32e6, 1e-3
        job.integrations = 1
        assert corr.corr_server_submit(h, C.byref(job), cb, None, C.byref(jid)) == corr.CORR_EINVAL
        job.scan.nchan = 256   # descriptor arrays still NULL
        assert corr.corr_server_submit(h, C.byref(job), cb, None, C.byref(jid)) == corr.CORR_EINVAL
        assert jid.value == -5
        p50, p99, sps, n = C.c_double(-1), C.c_double(-1), C.c_double(-1), C.c_int64(-1)
        assert corr.corr_server_stats(h, C.byref(p50), C.byref(p99), C.byref(sps), C.byref(n)) == corr.CORR_OK
        assert (p50.value, p99.value, sps.value, n.value) == (0.0, 0.0, 0.0, 0)
        assert corr.corr_server_wait(h, 0.0) == corr.CORR_OK
        assert corr.corr_server_stats(None, None, None, None, None) == corr.CORR_EINVAL
    finally:
        corr.corr_server_stop(h)
    corr.corr_server_stop(None)
