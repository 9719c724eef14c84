"""Mark5B-style framed input (corr_set_frame_format) on the GPU.

The library deframes the stations' frames on the device and flags blocks
that read from a frame without its sync word.  Against the framed-input
oracle: weights and block validity exact, visibilities within 1e-5; with
every frame valid the visibilities equal those of the same samples pushed
unframed, bit for bit; frames split across pushes (a push ending inside a
frame) give the same result as one push.
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
    return c


def rel_rms_per_baseline(v, ref):
    v = v.reshape(v.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    return np.sqrt(np.sum(np.abs(v - ref) ** 2, axis=1) / np.sum(np.abs(ref) ** 2, axis=1))


def make(corr, sc, payload=0):
    c = corr.Correlator(sc.stations, sc.nsub, sc.npol, sc.nchan, sc.tint, fs=sc.fs)
    if payload:
        c.set_frame_format(payload)
    for sb, nu in enumerate(sc.nu0):
        c.set_sky_freq(sb, nu)
    for s, segs in enumerate(sc.polys):
        for g in segs:
            c.set_delay_poly(s, g.t0, g.coeffs)
        c.set_stream_start(s, sc.sample0[s])
    return c


def run(c, nint):
    outs, ws = [], []
    for _ in range(nint):
        r = c.correlate()
        assert r is not None
        outs.append(r[0])
        ws.append(r[1])
    return np.stack(outs), np.stack(ws)


@pytest.fixture(scope="module")
def scan():
    """Ten stations of the 16-stream workload's shape, 0.01 s in two
    integrations; 10000-byte payloads (625 sample-times of 16 streams)."""
    sc = synth.config2(seed=52, duration=0.01, tint=0.005, boundary=0.005)
    plain = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    return sc, plain


def test_valid_frames_equal_plain_bit_for_bit(corr, scan):
    sc, plain = scan
    c = make(corr, sc)
    for s, b in enumerate(plain):
        c.push(s, b)
    ref, wref = run(c, 2)
    c.close()
    c = make(corr, sc, 10000)
    for s, b in enumerate(plain):
        c.push(s, synth.frame(b))
    got, w = run(c, 2)
    c.close()
    assert np.array_equal(w, wref) and np.array_equal(got, ref)


def test_lost_frames_match_the_oracle(corr, scan):
    sc, plain = scan
    P = 10000
    lost = {1: (3, 4), 4: (0,), 7: (11,)}   # station -> lost frames
    frames = [synth.frame(b, P, invalid=lost.get(s, ())) for s, b in enumerate(plain)]
    nsamp = [len(f) // (16 + P) * P * 4 // sc.G for f in frames]
    o = oracle.Oracle(sc.stations, sc.nsub, sc.npol, sc.nchan, sc.fs, sc.tint, sc.nu0, sc.polys, frames,
                      sc.sample0, nsamp, frame_payload=P)
    ref, wref = o.correlate(0, 2)
    c = make(corr, sc, P)
    for s, f in enumerate(frames):
        # split every station's frames over three pushes that end inside frames
        cuts = [0, len(f) // 3 // 16 * 16 + 4, 2 * len(f) // 3 // 16 * 16 + 8, len(f)]
        for a, b in zip(cuts[:-1], cuts[1:]):
            c.push(s, f[a:b])
    got, w = run(c, 2)
    nb = 2 * int(round(sc.fs * sc.tint)) // sc.N + 1
    _, _, _, v_gpu = c.debug_delays(0, nb)
    c.close()
    assert np.array_equal(v_gpu, o.delays(0, nb)[3])
    assert np.array_equal(w, wref)
    assert np.any(wref < wref.max())          # frames were really lost
    for i in range(2):
        err = rel_rms_per_baseline(got[i].reshape(sc.nbl, sc.G, sc.nchan), ref[i])
        assert np.all(err < 1e-5), err.max()


def test_windows_at_a_frame_boundary(corr):
    """A station 32 samples late with G = 2 and 400-byte payloads: block 30's
    window is the end of frame 4, block 31's the start of frame 5."""
    fs, nchan, m, P = 32e6, 64, 32, 400
    N = 2 * nchan
    T = 60 * N
    plain = synth.random_bytes(9, 0, T * 2 // 4)
    for bad in (4, 5):
        raw = synth.frame(plain, P, invalid=(bad,))
        c = corr.Correlator(1, 1, 2, nchan, 10 * N / fs, fs=fs)
        c.set_frame_format(P)
        c.set_delay_poly(0, 0.0, [m / fs])
        c.push(0, raw)
        _, _, _, v = c.debug_delays(0, 40)
        c.close()
        o = oracle.Oracle(1, 1, 2, nchan, fs, 10 * N / fs, [0.0], [[synth.Segment(0.0, (m / fs, 0, 0, 0, 0, 0))]],
                          [raw], [0], [len(raw) // (16 + P) * P * 2], frame_payload=P)
        assert np.array_equal(v, o.delays(0, 40)[3])
        assert v[0, 30] == (1 if bad == 5 else 0) and v[0, 31] == (0 if bad == 5 else 1)


def test_frame_format_argument_errors(corr):
    c = corr.Correlator(2, 1, 1, 64, 0.001)
    for bad in (-16, 10, 100):
        with pytest.raises(corr.CorrError) as ei:
            c.set_frame_format(bad)
        assert ei.value.code == corr.CORR_EINVAL
    c.set_delay_poly(0, 0.0, [0.0])
    c.push(0, np.zeros(64, np.uint8))
    with pytest.raises(corr.CorrError) as ei:
        c.set_frame_format(10000)
    assert ei.value.code == corr.CORR_ESTATE
    c.close()
