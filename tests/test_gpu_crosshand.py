"""Both hands of two polarisations (corr_set_pol_products(CORR_POL_CROSS)) on
the GPU, against the oracle's cross-hand products: FP32 within 1e-5 relative
RMS per baseline, FP16 / FP8 tensor cores within their stated bounds,
weights exact.  The shapes pick every X kernel the 2S (station, pol) pairs
lead to: the shared-memory ring for 2S <= 12, the tiled kernel with
off-diagonal tiles above, the tensor cores up to 32 stations; pre-F rotation
combined with both hands; the ten-station workload's own shape.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 8e-2}


@pytest.fixture(scope="module")
def corr():
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr as c
    return c


def rel_rms(v, ref):
    # per baseline over (subband, hand product, channel)
    v = v.reshape(v.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=1) / np.sum(np.abs(ref) ** 2, axis=1))


def run(corr, sc, streams, nint, precision=0, rotation=0, chunk=0):
    c = corr.from_scan(sc, streams)
    c.set_pol_products(corr.CORR_POL_CROSS)
    c.set_precision(precision)
    c.set_fringe_rotation(rotation)
    if chunk:
        c.set_chunk_blocks(chunk)
    outs, ws = [], []
    for _ in range(nint):
        r = c.correlate()
        assert r is not None
        assert r[0].shape == (sc.nbl, sc.nsub, 4, sc.nchan)
        outs.append(r[0])
        ws.append(r[1])
    c.close()
    return np.stack(outs), np.stack(ws)


def scan_and_ref(nchan, S, nsub, seed, nblk=60.5, rotation=0):
    fs = 32e6
    N = 2 * nchan
    tint = round(nblk * N / fs * fs) / fs
    sc = synth.config2(seed=seed, duration=2 * tint, tint=tint, boundary=tint, nchan=nchan, stations=S, nsub=nsub,
                       npol=2, fs=fs)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    ref, wref = oracle.Oracle.from_scan(sc, streams, rotation=rotation).correlate_cross(0, 2)
    return sc, streams, ref, wref


@pytest.mark.parametrize("nchan,S,nsub,precision,chunk", [
    (256, 3, 2, 0, 0),     # 2S = 6: TMA ring
    (512, 6, 1, 0, 40),    # 2S = 12, forced chunks
    (128, 7, 3, 0, 0),     # 2S = 14: tiled kernel with off-diagonal tiles
    (256, 3, 2, 1, 0),     # FP16 tensor cores
    (1024, 5, 2, 2, 0),    # FP8 tensor cores
    (64, 32, 1, 1, 0),     # 2S = 64: one channel per 128-row tile
])
def test_cross_hands_match_oracle(corr, nchan, S, nsub, precision, chunk):
    sc, streams, ref, wref = scan_and_ref(nchan, S, nsub, seed=nchan + S + precision)
    vis, w = run(corr, sc, streams, 2, precision, chunk=chunk)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms(vis[i], ref[i])
        assert np.all(err < TOL[precision]), (i, err.max())


def test_cross_hands_with_pre_f_rotation(corr):
    sc, streams, ref, wref = scan_and_ref(256, 4, 2, seed=77, rotation=1)
    vis, w = run(corr, sc, streams, 2, rotation=1)
    assert np.array_equal(w, wref)
    for i in range(2):
        assert np.all(rel_rms(vis[i], ref[i]) < 1e-5)


def test_cross_hands_config2_slice(corr):
    """Ten stations, 8 subbands x 2 pols, 1024 channels, spacecraft delays,
    across a delay segment boundary: 20 (station, pol) pairs per subband."""
    sc = synth.config2(seed=2, duration=0.01, tint=0.005, boundary=0.005)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate_cross(0, 2)
    for precision in (0, 1):
        vis, w = run(corr, sc, streams, 2, precision)
        assert np.array_equal(w, wref)
        for i in range(2):
            assert np.all(rel_rms(vis[i], ref[i]) < TOL[precision]), (precision, i)


def test_cross_hand_argument_errors(corr):
    c = corr.Correlator(3, 2, 1, 64, 0.001)
    with pytest.raises(corr.CorrError) as ei:
        c.set_pol_products(corr.CORR_POL_CROSS)
    assert ei.value.code == corr.CORR_EINVAL
    c.close()
    c = corr.Correlator(33, 1, 2, 64, 0.001)
    c.set_pol_products(corr.CORR_POL_CROSS)
    with pytest.raises(corr.CorrError) as ei:
        c.set_precision(corr.CORR_PREC_FP16_TC)
    assert ei.value.code == corr.CORR_EINVAL
    c.close()
