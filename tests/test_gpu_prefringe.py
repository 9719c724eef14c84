"""Pre-F fringe rotation (corr_set_fringe_rotation(CORR_ROT_PRE_F)) on the GPU.

Parity with the oracle's pre-F path (per-sample fringe phase linear about
the block centre, complex N-point transform, fractional-delay slope) at the
same bars as the post-F path: FP32 within 1e-5 relative RMS per baseline,
FP16 / FP8 tensor cores within their stated bounds, weights exact.  Then the
physics at the ten-station workload's own numbers: a spacecraft baseline at
4.8 GHz and 3e-5 s/s with 1024 channels (64 us blocks) turns its fringe phase
9.2 times per block, so post-F rotation keeps about |sinc(9.2)| of the
2-bit coherence eta * rho and pre-F all of it.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 8e-2}
ETA = 0.8825  # 2-bit efficiency at +-0.98 sigma with levels 1 / 3.336 (pinned on the CPU)


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


def run(corr, sc, streams, nint, precision=0, rotation=1, chunk=0, unit=None):
    c = corr.from_scan(sc, streams)
    c.set_fringe_rotation(rotation)
    c.set_precision(precision)
    if unit is not None:
        c.set_x_unit(unit)
    if chunk:
        c.set_chunk_blocks(chunk)
    outs, ws = [], []
    for _ in range(nint):
        r = c.correlate()
        assert r is not None
        outs.append(r[0])
        ws.append(r[1])
    c.close()
    return np.stack(outs), np.stack(ws)


@pytest.fixture(scope="module")
def cfg2_slice():
    """The ten-station workload's shape (8 subbands x 2 pols, 1024 channels,
    spacecraft at up to 1.2 s and 3e-5 s/s, nu0 = 4.8 GHz + 16 MHz per
    subband), 0.02 s in two integrations of 156.25 blocks, across a delay
    segment boundary."""
    sc = synth.config2(seed=2, duration=0.02, tint=0.01, boundary=0.01)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams, rotation=oracle.ROT_PRE_F).correlate(0, 2)
    return sc, streams, ref, wref


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_pre_f_config2_slice(corr, cfg2_slice, precision):
    sc, streams, ref, wref = cfg2_slice
    vis, w = run(corr, sc, streams, 2, precision)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL[precision]), (precision, i, err.max())


@pytest.mark.parametrize("precision", [1, 2])
def test_pre_f_config2_slice_tensor_cores(corr, cfg2_slice, precision):
    """Pre-F spectra through the corner turn into tensor-core operand tiles
    (the default sends 10 stations' FP16 / E4M3 spectra to the CUDA cores)."""
    sc, streams, ref, wref = cfg2_slice
    vis, w = run(corr, sc, streams, 2, precision, unit=corr.CORR_X_TENSOR_CORES)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < TOL[precision]), (precision, i, err.max())


@pytest.mark.parametrize("nchan,S,nsub,npol,chunk", [(4, 2, 1, 1, 0), (32, 3, 3, 1, 0), (256, 4, 1, 2, 50),
                                                     (512, 5, 2, 1, 0), (2048, 3, 1, 1, 7), (4096, 3, 16, 2, 24)])
def test_pre_f_shapes(corr, nchan, S, nsub, npol, chunk):
    """Every transform plan of the pre-F path (4..8192 points, one thread up
    to 256 threads per transform), runtime and compile-time stream counts
    (G = 1, 2, 3, 32), forced chunks with ragged ends, integrations of a
    fractional number of blocks."""
    fs = 32e6
    N = 2 * nchan
    tint = round((60.5 * N) / fs * fs) / fs
    sc = synth.config2(seed=7 + nchan, duration=2 * tint, tint=tint, boundary=tint, nchan=nchan, stations=S,
                       nsub=nsub, npol=npol, fs=fs)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    ref, wref = oracle.Oracle.from_scan(sc, streams, rotation=oracle.ROT_PRE_F).correlate(0, 2)
    vis, w = run(corr, sc, streams, 2, chunk=chunk)
    assert np.array_equal(w, wref)
    for i in range(2):
        err = rel_rms_per_baseline(vis[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < 1e-5), (i, err.max())


def test_pre_f_spectrum_matches_oracle(corr, cfg2_slice):
    sc, streams, _, _ = cfg2_slice
    c = corr.from_scan(sc, streams)
    c.set_fringe_rotation(corr.CORR_ROT_PRE_F)
    o = oracle.Oracle.from_scan(sc, streams, rotation=oracle.ROT_PRE_F)
    for s in (0, 3):
        for j in (0, 15):
            for b in (0, 100, 311):
                got, ok = c.debug_spectrum(s, j, b)
                ref, ok_o = o.spectrum(s, j, b)
                assert ok == ok_o and ok
                err = np.sqrt(np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2))
                assert err < 2e-6, (s, j, b, err)
    c.close()


def coherence(vis, nblk, k0, k1):
    a0, a1, cr = vis[0].real[k0:k1], vis[2].real[k0:k1], vis[1][k0:k1]
    return np.mean(cr / np.sqrt(a0 * a1)), 1.0 / math.sqrt(nblk * (k1 - k0))


def test_spacecraft_fringe_kept_by_pre_f_lost_by_post_f(corr):
    """Space station 0.9 s and 3e-5 s/s, ground station 10 ms and 2e-7 s/s,
    nu0 = 4.8 GHz, 1024 channels: (3e-5 - 2e-7) * 4.8e9 * 64e-6 = 9.15 turns
    of fringe per block.  0.1 s of generated data at rho = 0.02."""
    fs = 32e6
    polys = [[synth.Segment(0.0, (0.9, 3e-5, 0, 0, 0, 0))], [synth.Segment(0.0, (1e-2, 2e-7, 0, 0, 0, 0))]]
    sc = synth.Scan(2, 1, 1, 1024, fs, 0.1, 0.1, 0.02, 17, [4.8e9], polys)
    synth.plan_windows(sc)
    streams = [synth.station_bytes(sc, s) for s in range(2)]
    nblk = -(-int(round(0.1 * fs)) // sc.N)   # 1562.5 blocks: the integration holds 1563
    k0, k1 = 24, 896   # above the fringe-rate image (2 x 144 kHz = 18 channels), below the roll-off
    pre, w = run(corr, sc, streams, 1, rotation=1)
    post, _ = run(corr, sc, streams, 1, rotation=0)
    assert np.all(w == nblk)
    r_pre, sigma = coherence(pre[0].reshape(3, sc.nchan), nblk, k0, k1)
    r_post, _ = coherence(post[0].reshape(3, sc.nchan), nblk, k0, k1)
    print("coherence: pre-F %.5f%+.5fj, post-F %.5f%+.5fj, eta*rho %.5f, sigma %.5f"
          % (r_pre.real, r_pre.imag, r_post.real, r_post.imag, ETA * sc.rho, sigma))
    assert abs(r_pre.real - ETA * sc.rho) < 4 * sigma and abs(r_pre.imag) < 4 * sigma
    assert abs(r_post) < 0.25 * ETA * sc.rho


def test_pre_f_argument_errors(corr):
    c = corr.Correlator(2, 1, 1, 8192, 0.01)
    with pytest.raises(corr.CorrError) as ei:
        c.set_fringe_rotation(corr.CORR_ROT_PRE_F)
    assert ei.value.code == corr.CORR_EINVAL
    with pytest.raises(corr.CorrError) as ei:
        c.set_fringe_rotation(7)
    assert ei.value.code == corr.CORR_EINVAL
    c.close()
