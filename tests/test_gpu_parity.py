"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: unpacked codes, window starts, delays and validity bit-exact; FP32
visibilities within 1e-5 relative RMS per baseline,
    rel_rms(bl) = sqrt(sum |V - V_ref|^2 / sum |V_ref|^2)  over (stream, channel);
weights exact.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def corr():
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr as c
    return c


def rel_rms_per_baseline(v, ref):
    v = v.reshape(v.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=1) / np.sum(np.abs(ref) ** 2, axis=1))


def run_all(c, nint):
    outs, ws = [], []
    for _ in range(nint):
        r = c.correlate()
        assert r is not None, "correlate returned EAGAIN/EEND"
        outs.append(r[0])
        ws.append(r[1])
    return np.stack(outs), np.stack(ws)


def small_cfg2(seed=2, duration=0.1, tint=0.05, boundary=0.05, nchan=1024, stations=10, nsub=8, npol=2):
    sc = synth.config2(seed=seed, duration=duration, tint=tint, boundary=boundary, nchan=nchan,
                       stations=stations, nsub=nsub, npol=npol)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    return sc, streams


# --------------------------------------------------------------------------
# bit-exact parts


@pytest.mark.parametrize("G", [1, 3, 16, 32])
def test_codes_bit_exact(corr, G):
    nsub, npol = (G, 1) if G in (1, 3) else (G // 2, 2)
    T = 4096
    raw = synth.random_bytes(7, G, T * G // 4)
    c = corr.Correlator(1, nsub, npol, 64, 0.001)
    c.set_delay_poly(0, 0.0, [0.0])
    c.push(0, raw)
    for j in range(G):
        got = c.debug_codes(0, j, 0, T + 8)
        assert np.array_equal(got[:T], oracle.unpack_codes(raw, G, j, 0, T))
        assert np.all(got[T:] == 0xFF)
    c.close()


def test_delays_bit_exact_config1(corr, cfg1):
    sc, streams, o = cfg1
    c = corr.from_scan(sc, streams)
    nb = 62500
    start, eps, tau, valid = c.debug_delays(0, nb)
    n_b, e_o, t_o, v_o = o.delays(0, nb)
    assert np.array_equal(start, np.arange(nb)[None, :] * sc.N + n_b)
    assert np.array_equal(valid, v_o)
    assert np.array_equal(tau, t_o)
    assert np.array_equal(eps, e_o)
    c.close()


def test_delays_bit_exact_across_segment_boundary(corr):
    sc = synth.config2(duration=0.1, tint=0.05, boundary=0.05, plan=True)
    N = sc.N
    c = corr.Correlator(sc.stations, sc.nsub, sc.npol, sc.nchan, sc.tint)
    for s, segs in enumerate(sc.polys):
        for g in segs:
            c.set_delay_poly(s, g.t0, g.coeffs)
    nb = int(0.1 * sc.fs) // N + 8
    start, eps, tau, valid = c.debug_delays(0, nb)
    o = oracle.Oracle(sc.stations, sc.nsub, sc.npol, sc.nchan, sc.fs, sc.tint, sc.nu0, sc.polys,
                      [np.zeros(16, np.uint8)] * sc.stations, [0] * sc.stations, [0] * sc.stations)
    n_b, e_o, t_o, v_o = o.delays(0, nb)
    assert np.array_equal(start, np.arange(nb)[None, :] * N + n_b)
    assert np.array_equal(tau, t_o) and np.array_equal(eps, e_o)
    c.close()


# --------------------------------------------------------------------------
# spectra


def test_spectra_match_oracle(corr, cfg1):
    sc, streams, o = cfg1
    c = corr.from_scan(sc, streams)
    for s in range(sc.stations):
        for b in (0, 1, 777, 31250, 62499):
            got, ok = c.debug_spectrum(s, 0, b)
            ref, ok_o = o.spectrum(s, 0, b)
            assert ok == ok_o
            err = np.sqrt(np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2))
            assert err < 2e-6, (s, b, err)
    c.close()


# --------------------------------------------------------------------------
# visibilities


def test_config1_full_parity(corr, cfg1):
    sc, streams, o = cfg1
    ref, wref = o.correlate(0, 1)
    c = corr.from_scan(sc, streams)
    vis, w = run_all(c, 1)
    assert np.array_equal(w, wref)
    v = vis[0].reshape(sc.nbl, sc.G, sc.nchan)
    err = rel_rms_per_baseline(v, ref[0])
    assert np.all(err < TOL_FP32), err
    # after the flush the streams' tail (the delay margin) still reaches into
    # integration 1 for a few blocks; that partial integration must match too,
    # and the one after it ends the scan (CORR_EEND)
    c.flush()
    tail = c.correlate()
    ref1, wref1 = o.correlate(1, 1)
    assert tail is not None and np.array_equal(tail[1], wref1[0])
    nz = wref1[0] > 0
    if nz.any():
        err = rel_rms_per_baseline(tail[0].reshape(sc.nbl, sc.G, sc.nchan)[nz], ref1[0][nz])
        assert np.all(err < TOL_FP32), err
    assert c.correlate() is None
    c.close()


def test_config2_slice_parity_across_segment_boundary(corr):
    """10 stations, 8 subbands x 2 pols, 1024 channels, 0.1 s cut into two
    0.05 s integrations, a delay-segment boundary at 0.05 s, spacecraft delay
    near one second with its large fringe phase."""
    sc, streams = small_cfg2()
    o = oracle.Oracle.from_scan(sc, streams)
    ref, wref = o.correlate(0, 2)
    c = corr.from_scan(sc, streams)
    vis, w = run_all(c, 2)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL_FP32), (i, err.max())
    c.close()


@pytest.mark.parametrize("nchan,S,nsub,npol", [(4, 2, 1, 1), (16, 3, 3, 1), (64, 5, 1, 2), (128, 13, 2, 1),
                                               (512, 2, 1, 1), (2048, 4, 2, 2), (4096, 3, 1, 2),
                                               (8192, 2, 2, 1)])
def test_shapes_parity(corr, nchan, S, nsub, npol):
    """Every FFT plan, odd stream counts, more stations than one X tile, and
    integrations whose block count is not a multiple of any tile."""
    fs = 32e6
    N = 2 * nchan
    tint = (7 * N + N // 2) / fs if nchan >= 1024 else (37 * N + 3) / fs
    tint = round(tint * fs) / fs
    sc = synth.config2(seed=nchan + S, duration=3 * tint, tint=tint, boundary=1.5 * tint, nchan=nchan,
                       stations=S, nsub=nsub, npol=npol)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    o = oracle.Oracle.from_scan(sc, streams)
    ref, wref = o.correlate(0, 2)
    c = corr.from_scan(sc, streams)
    vis, w = run_all(c, 2)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, nchan), ref[i])
        assert np.all(err < TOL_FP32), (i, err.max())
    c.close()


def test_eagain_then_push_then_flush_partial(corr):
    """Data arriving in pieces: CORR_EAGAIN until a station has pushed what
    the integration needs; after corr_flush the last integration is produced
    with only the blocks that have data (weights below the full count)."""
    sc, streams = small_cfg2(duration=0.1, tint=0.04, nchan=256, stations=3, nsub=1, npol=2)
    o = oracle.Oracle.from_scan(sc, streams)
    c = corr.from_scan(sc)
    half = [(len(b) // 2) // 4 * 4 for b in streams]
    for s in range(sc.stations):
        c.push(s, streams[s][:half[s]])
    # the first 0.04 s need well under half of each stream
    r0 = c.correlate()
    assert r0 is not None
    assert c.correlate() is None  # integration 1 needs more data: EAGAIN
    assert c.next_integration() == 1
    for s in range(sc.stations):
        c.push(s, streams[s][half[s]:])
    r1 = c.correlate()
    assert r1 is not None
    assert c.correlate() is None  # integration 2 reaches past the data: EAGAIN
    c.flush()
    r2 = c.correlate()
    assert r2 is not None
    ref, wref = o.correlate(0, 3)
    for i, r in enumerate((r0, r1, r2)):
        assert np.array_equal(r[1], wref[i])
        err = rel_rms_per_baseline(r[0].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL_FP32)
    assert wref[2].max() < wref[1].max()
    c.close()


def test_station_without_data_has_zero_weight(corr):
    """A station whose recording starts late: blocks before its data are
    invalid; its baselines carry weight 0 and zero visibilities there."""
    sc, streams = small_cfg2(duration=0.06, tint=0.02, nchan=128, stations=3, nsub=1, npol=1)
    late = 2
    skip = int(0.03 * sc.fs) // 16 * 16
    sc.sample0[late] += skip
    streams[late] = streams[late][skip * sc.G // 4:]
    sc.nsamp[late] -= skip
    o = oracle.Oracle.from_scan(sc, streams)
    ref, wref = o.correlate(0, 3)
    c = corr.from_scan(sc, streams)
    c.flush()
    vis, w = run_all(c, 3)
    assert np.array_equal(w, wref)
    assert wref[0][2] == 0 and wref[0][0] > 0
    for i in range(3):
        v = vis[i].reshape(sc.nbl, sc.G, sc.nchan)
        nz = wref[i] > 0
        assert np.all(v[~nz] == 0)
        err = rel_rms_per_baseline(v[nz], ref[i][nz])
        assert np.all(err < TOL_FP32)
    c.close()


def test_bench_workload_sampled_parity(corr):
    """The benchmark's workload and launch path (10 stations, 8 x 2 streams,
    1024 channels, 1 s integrations, spacecraft delay ~1 s; samples attached
    in device memory, visibilities written to device memory): integration 0,
    compared with the oracle on three sampled streams."""
    import torch
    sc = synth.config2(duration=2.0)
    streams = []
    for s in range(sc.stations):
        n = min(sc.nsamp[s], int(1.05 * sc.fs) + 64 * 1024) // 16 * 16
        sc.nsamp[s] = n
        streams.append(synth.random_bytes(100 + s, s, n * sc.G // 4))
    dev = [torch.from_numpy(b).cuda() for b in streams]
    c = corr.from_scan(sc, device_streams=dev)
    out = torch.empty((sc.nbl, sc.G, sc.nchan), dtype=torch.complex64, device="cuda")
    wts = torch.empty(sc.nbl, dtype=torch.float64, device="cuda")
    c.set_stream(torch.cuda.current_stream().cuda_stream)
    assert c.correlate_device(out, wts) == corr.CORR_OK
    torch.cuda.synchronize()
    vis = out.cpu().numpy()
    o = oracle.Oracle.from_scan(sc, streams)
    for j in (0, 7, 15):
        ref, wref = o.correlate(0, 1, j, 1)
        assert np.array_equal(wts.cpu().numpy(), wref[0])
        err = rel_rms_per_baseline(vis[:, j:j + 1, :], ref[0])
        assert np.all(err < TOL_FP32), (j, err.max())
    c.close()


def test_async_pushes_in_pieces_match_oracle(corr):
    """Packed bytes pushed in several pieces with corr_push_samples_async from
    pinned memory, a piece ahead of each integration; results equal the
    oracle's and the library answers CORR_EAGAIN until the bytes exist."""
    import torch
    sc, streams = small_cfg2(duration=0.08, tint=0.02, nchan=256, stations=4, nsub=2, npol=2)
    o = oracle.Oracle.from_scan(sc, streams)
    ref, wref = o.correlate(0, 4)
    c = corr.from_scan(sc)
    for s in range(sc.stations):
        c.reserve(s, len(streams[s]))
    pinned = [torch.from_numpy(b).pin_memory() for b in streams]
    npc = 4
    cuts = [[(len(b) * k // npc) // 4 * 4 for k in range(npc)] + [len(b)] for b in streams]
    pushed = 0

    def push_next():
        nonlocal pushed
        for s in range(sc.stations):
            c.push_async(s, pinned[s][cuts[s][pushed]:cuts[s][pushed + 1]])
        pushed += 1
        if pushed == npc:
            c.flush()

    push_next()
    got = []
    eagain = 0
    while len(got) < 4:
        r = c.correlate()
        if r is None:
            eagain += 1
            assert pushed < npc, "EAGAIN with all data pushed"
            push_next()
            continue
        got.append(r)
    c.wait_pushes()
    assert eagain >= 1
    for i, (v, w) in enumerate(got):
        assert np.array_equal(w, wref[i])
        err = rel_rms_per_baseline(v.reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL_FP32), (i, err.max())
    c.close()


def test_host_attached_streams_match_oracle(corr):
    """Stations' packed bytes left in pinned host memory and attached with
    corr_attach_samples_host (read by the F kernel over the host link)."""
    import torch
    sc, streams = small_cfg2(duration=0.06, tint=0.02, nchan=512, stations=5, nsub=4, npol=2)
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 3)
    pinned = [torch.from_numpy(b).pin_memory() for b in streams]
    c = corr.from_scan(sc)
    for s in range(sc.stations):
        c.attach_host(s, pinned[s])
    c.flush()
    vis, w = run_all(c, 3)
    assert np.array_equal(w, wref)
    for i in range(3):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL_FP32), (i, err.max())
    c.close()
