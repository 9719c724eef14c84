"""GPU parity at the edges of the launch space, through the C ABI.

* The 32-stream F kernel (16 subbands x 2 pols, one sample-time group = two
  words) at 8192-point FFTs, the launch the 64-station dense workload runs,
  over several chunks at all three precisions.
* The tensor-core X step at 64 stations accumulating over several chunks
  (TMEM accumulator -> partial sums, more than once per integration).
* The hot-path 2-bit decode, bit for bit: with integer levels, integer-sample
  delays and no fringe rotation the DC bin of every spectrum is the exact
  integer sum of the window's levels in FP32 and in FP64 alike, so the F
  kernel's staged-window decode (not a debug kernel) must reproduce the
  oracle's DC bin exactly, at window offsets that cross word boundaries.
* Integrations of a fractional number of blocks and stations whose data end
  exactly at a block's window end: weights exact, visibilities within 1e-5.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 8e-2}  # FP32, FP16 tensor cores, FP8 tensor cores


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


def correlate_n(c, n):
    outs, ws = [], []
    for _ in range(n):
        r = c.correlate()
        assert r is not None
        outs.append(r[0])
        ws.append(r[1])
    return np.stack(outs), np.stack(ws)


@pytest.fixture(scope="module")
def g32_scan():
    """3 stations (one in space), 16 subbands x 2 pols at 64 Msample/s, 4096
    channels, two integrations of 70.5 blocks."""
    fs, N = 64e6, 8192
    tint = 70.5 * N / fs
    sc = synth.config2(seed=32, duration=2 * tint, tint=tint, boundary=tint, nchan=4096, stations=3, nsub=16,
                       npol=2, fs=fs, nu0_base=1.6e9)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    return sc, streams, ref, wref


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_g32_8192_point_multichunk(corr, g32_scan, precision):
    sc, streams, ref, wref = g32_scan
    c = corr.from_scan(sc, streams)
    c.set_precision(precision)
    c.set_chunk_blocks(24)  # 3 chunks per integration (24 + 24 + 22.5)
    vis, w = correlate_n(c, 2)
    cb, _ = c.launch_shape()
    c.close()
    assert cb == 24
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL[precision]), (precision, i, err.max())


@pytest.mark.parametrize("precision,chunk", [(1, 64), (2, 128), (1, 40)])
def test_tc_64_stations_multichunk(corr, precision, chunk):
    """64 stations x 1 stream, 512 channels: an integration of 300.5 blocks in
    chunks of 64 / 128 / 40 blocks, so each TMEM accumulator is read out and
    added to the partial sums several times per integration (a 40-block chunk
    also leaves zero-padded K rows in every tile)."""
    fs, nchan = 32e6, 512
    N = 2 * nchan
    tint = 300.5 * N / fs
    sc = synth.config2(seed=640 + chunk, duration=tint, tint=tint, boundary=tint / 2, nchan=nchan, stations=64,
                       nsub=1, npol=1, fs=fs)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 1)
    c = corr.from_scan(sc, streams)
    c.set_precision(precision)
    c.set_chunk_blocks(chunk)
    vis, w = correlate_n(c, 1)
    c.close()
    assert np.array_equal(w, wref)
    err = rel_rms_per_baseline(vis[0].reshape(sc.nbl, sc.G, sc.nchan), ref[0])
    assert np.all(err < TOL[precision]), err.max()


INT_LEVELS = (-512.0, -8.0, 8.0, 512.0)


@pytest.mark.parametrize("G,nchan", [(1, 256), (3, 512), (16, 1024), (32, 4096), (16, 8192), (5, 32)])
def test_hot_path_decode_bit_exact(corr, G, nchan):
    """DC bin of the F kernel's own spectra == the oracle's exact level sum."""
    nsub, npol = (G, 1) if G % 2 else (G // 2, 2)
    fs = 32e6
    N = 2 * nchan
    delays = [0, 3, 7, 13]  # samples: windows start mid-word for every G
    S = len(delays)
    nblk = 20
    T = nblk * N + max(delays) + 64
    streams = [synth.random_bytes(100 + G, s, (T * G + 15) // 16 * 4) for s in range(S)]
    tint = 4 * N / fs
    c = corr.Correlator(S, nsub, npol, nchan, tint, fs=fs, lut=INT_LEVELS)
    polys = []
    for s, d in enumerate(delays):
        c.set_delay_poly(s, 0.0, [d / fs])
        polys.append([synth.Segment(0.0, (d / fs, 0, 0, 0, 0, 0))])
        c.push(s, streams[s])
    o = oracle.Oracle(S, nsub, npol, nchan, fs, tint, [0.0] * nsub, polys, streams, [0] * S, [T] * S,
                      lut=INT_LEVELS)
    n_b, eps, _, _ = o.delays(0, nblk)
    assert np.all(eps == 0.0) and np.array_equal(n_b[:, 0], delays)
    checked = 0
    for s in range(S):
        for j in sorted({0, G // 2, G - 1}):
            for b in (0, 1, 5, nblk - 2):
                got, ok = c.debug_spectrum(s, j, b)
                ref, ok_o = o.spectrum(s, j, b)
                assert ok and ok_o
                # the exact level sum, both sides: integers below 2^24
                assert float(got[0].real) == ref[0].real, (s, j, b, got[0], ref[0])
                assert float(got[0].imag) == 0.0 and ref[0].imag == 0.0
                err = np.sqrt(np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2))
                assert err < 2e-6
                checked += 1
    c.close()
    assert checked >= 4 * 4


def test_ragged_integrations_and_data_edges(corr):
    """fs*tint = 7.5 blocks of 128 samples (integrations of 8, 7, 8, 7, ...
    blocks), three stations with integer and fractional delays, the last
    station's data ending exactly at one block's window end, correlated to
    the end after corr_flush."""
    fs, nchan = 32e6, 64
    N = 2 * nchan
    spi = 960
    tint = spi / fs
    nint = 6
    S, G = 3, 2
    delays = [0.0, 5.0, 2.25]
    polys = [[synth.Segment(0.0, (d / fs, 1e-7 * s, 0, 0, 0, 0))] for s, d in enumerate(delays)]
    # station 2's data end exactly at the window end of block 30, the first
    # block of integration 4 (integrations start at blocks 0, 8, 15, 23, 30, 38)
    o_tmp = oracle.Oracle(S, 1, G, nchan, fs, tint, [1e8], polys, [np.zeros(64, np.uint8)] * S, [0] * S,
                          [1 << 40] * S)
    n_b, _, _, _ = o_tmp.delays(0, 64)
    T = [nint * spi + 4 * N, nint * spi + 4 * N, 30 * N + int(n_b[2, 30]) + N]
    streams = [synth.random_bytes(77, s, (T[s] * G + 15) // 16 * 4) for s in range(S)]
    c = corr.Correlator(S, 1, G, nchan, tint, fs=fs)
    c.set_sky_freq(0, 1e8)
    for s in range(S):
        for g in polys[s]:
            c.set_delay_poly(s, g.t0, g.coeffs)
        c.push(s, streams[s])
    c.flush()
    vis, w = correlate_n(c, nint)
    c.close()
    o = oracle.Oracle(S, 1, G, nchan, fs, tint, [1e8], polys, streams, [0] * S, T)
    ref, wref = o.correlate(0, nint)
    assert np.array_equal(w, wref)
    assert wref[:4, 0].tolist() == [8, 7, 8, 7]
    # baseline (2, 2): all 7 blocks of integration 3, only block 30 of integration 4
    assert wref[3, -1] == 7 and wref[4, -1] == 1 and wref[5, -1] == 0
    for i in range(nint):
        v = vis[i].reshape(S * (S + 1) // 2, G, nchan)
        nz = wref[i] > 0
        err = rel_rms_per_baseline(v[nz], ref[i][nz])
        assert np.all(err < 1e-5), (i, err.max())
        assert np.all(v[~nz] == 0)


@pytest.mark.parametrize("S,nchan,nsub,npol,chunk", [
    (17, 256, 1, 2, 0),    # 3 tile pairs: 32 channels per CTA
    (40, 128, 1, 1, 0),    # 15 tile pairs: 16 channels per CTA
    (50, 64, 2, 1, 24),    # 28 tile pairs: 8 channels per CTA, forced chunks
    (64, 256, 1, 1, 0),    # 36 tile pairs: 4 channels per CTA (the dense FP32 shape)
    (64, 4, 1, 1, 0),      # fewer channels than a CTA takes
])
def test_fp32_x_step_above_12_stations(corr, S, nchan, nsub, npol, chunk):
    """The FP32 X step for more than 12 stations (every station's values of
    a CTA's channels staged once in shared memory, 8 x 8 tile pairs per
    thread): all tile-pair counts and channel widths, ragged integrations of
    about 40 blocks, against the oracle within 1e-5 and with exact weights."""
    fs = 32e6
    N = 2 * nchan
    tint = round((40 * N + 7) / fs * fs) / fs
    sc = synth.config2(seed=S * 7 + nchan, duration=2 * tint, tint=tint, boundary=tint, nchan=nchan, stations=S,
                       nsub=nsub, npol=npol)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    c = corr.from_scan(sc, streams)
    if chunk:
        c.set_chunk_blocks(chunk)
    vis, w = correlate_n(c, 2)
    c.close()
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL[0]), (i, err.max())
