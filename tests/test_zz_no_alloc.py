"""corr_correlate_static: the entry point that allocates no device memory.

It is meant for callers that cannot let the library call cudaMalloc (a fixed
device-memory budget owned by the host program, or a real-time loop that must
keep allocation, which can synchronise the whole device, off its hot path).
Its intermediates live in one static 64 MiB device array.  This file is named
so that pytest collects it last.  The test calls the entry point twice in a
row through the C ABI and checks each result against the handle path
(corr_correlate_device) on the same device-resident samples, with the same
tolerance the other parity tests use (1e-5 relative RMS per baseline, weights
exact); then it checks that further calls leave the device's free memory
unchanged.  It must pass alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


def rel_rms_per_baseline(v, ref):
    v = v.reshape(v.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=1) / np.sum(np.abs(ref) ** 2, axis=1))


def test_static_scratch_matches_handle_path_twice():
    import torch
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr

    torch.cuda.set_device(0)
    sc = synth.config2(seed=21, duration=0.05, tint=0.02, boundary=0.03, nchan=512, stations=6, nsub=4, npol=2)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    dev = [torch.from_numpy(b).cuda() for b in streams]
    torch.cuda.synchronize()

    # the handle path (allocates its own work buffers)
    c = corr.from_scan(sc, device_streams=dev)
    c.flush()
    ref = torch.empty((2, sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device="cuda")
    wref = torch.empty((2, sc.nbl), dtype=torch.float64, device="cuda")
    for i in range(2):
        assert c.correlate_device(ref[i], wref[i]) == corr.CORR_OK
    torch.cuda.synchronize()

    # the static-scratch path: two calls in a row, integrations 0 and 1
    st = corr.StaticScan(sc, dev)
    out = torch.full((2, sc.nbl, sc.G, sc.nchan), float("nan"), dtype=torch.complex64, device="cuda")
    w = torch.full((2, sc.nbl), -1.0, dtype=torch.float64, device="cuda")
    for i in range(2):
        assert st.correlate(i, out[i], w[i]) == corr.CORR_OK
    torch.cuda.synchronize()
    c.close()
    torch.cuda.synchronize()

    # the property the entry point exists for: once the first calls have run
    # (module and kernels loaded), further calls take no device memory
    again = torch.empty_like(out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for i in range(2):
            assert st.correlate(i, again[i]) == corr.CORR_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(again, out)  # the same inputs give the same result, call after call

    R, O = ref.cpu().numpy(), out.cpu().numpy()
    assert np.array_equal(w.cpu().numpy(), wref.cpu().numpy())
    for i in range(2):
        assert np.all(np.isfinite(O[i]))
        err = rel_rms_per_baseline(O[i], R[i])
        assert np.all(err < TOL_FP32), (i, err.max())


def test_static_scratch_rejects_oversized_shape():
    import torch
    from paper_1502_06894_gb300 import corr

    # 64 stations x 32 streams x 8192 channels: the partial sums alone are
    # 2080 * 32 * 8192 * 8 bytes, far beyond the 64 MiB static array
    sc = synth.config2(seed=3, duration=0.01, tint=0.01, boundary=0.005, nchan=8192, stations=64, nsub=16,
                       npol=2, plan=False)
    sc.sample0 = [0] * sc.stations
    dev = [torch.zeros(64, dtype=torch.uint8, device="cuda") for _ in range(sc.stations)]
    st = corr.StaticScan(sc, dev)
    out = torch.zeros(16, dtype=torch.complex64, device="cuda")
    assert st.correlate(0, out) == corr.CORR_ETOOBIG
