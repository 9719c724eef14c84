"""Pins of the oracle's pre-F fringe rotation.

The paper's point (Sec. 2) is that RadioAstron's large and fast-changing
velocity must be followed by the delay model; the fringe phase nu0 tau(t) of a
spacecraft then changes by several turns within one FFT block (at 4.8 GHz and
3e-5 s/s, 9 turns in 64 us).  Rotating after the transform (one phase per
block) then averages the fringe away; rotating every sample before the
transform, with the phase linear about the block centre, keeps it.  The oracle
implements both; these tests fix the pre-F form by facts it does not compute:

* the delay rate is the exact derivative of the polynomial (rational
  arithmetic on dyadic coefficients) and matches a central difference;
* with zero delay rate the per-sample phase is constant, so pre-F equals
  post-F (a constant factor commutes with the DFT);
* on the generator's signal model at a spacecraft-like rate, pre-F recovers
  the 2-bit coherence eta * rho with phase zero, while post-F loses it to the
  within-block phase drift (|sinc| of the drift in turns); with a fractional
  delay sweeping through the samples, the upper half of the band also needs
  the post-transform fractional-delay slope to keep eta * rho.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def test_rate_is_the_exact_polynomial_derivative():
    fs, nchan = float(1 << 20), 8
    N = 2 * nchan
    rng = np.random.default_rng(31)
    for _ in range(200):
        b = int(rng.integers(0, 20000))
        tc = Fraction(b * N + N // 2) / Fraction(int(fs))
        u = Fraction(int(rng.integers(1, 32)), 8)
        coeffs = [float(Fraction(int(rng.integers(-63, 64)), 1 << int(rng.integers(4, 20)))) for _ in range(6)]
        exact = sum(i * Fraction(c) * u ** (i - 1) for i, c in enumerate(coeffs) if i >= 1)
        assert Fraction(float(exact)) == exact
        o = oracle.Oracle(1, 1, 1, nchan, fs, 64 * N / fs, [0.0], [[synth.Segment(float(tc - u), tuple(coeffs))]],
                          [np.zeros(64, np.uint8)], [-(1 << 50)], [1 << 51])
        rate = o.delays(b, 1, rate=True)[4][0, 0]
        assert Fraction(rate) == exact


def test_rate_matches_central_difference():
    sc = synth.config2(seed=5, duration=1.0, tint=0.5, boundary=0.5, nchan=1024, stations=4, plan=False)
    o = oracle.Oracle(sc.stations, 1, 1, sc.nchan, sc.fs, sc.tint, [0.0], sc.polys,
                      [np.zeros(64, np.uint8)] * sc.stations, [0] * sc.stations, [0] * sc.stations)
    blocks = [0, 5000, 7811, 7812, 15000]
    _, _, tau, _, rate = o.delays(0, 15001, rate=True)
    h = 1e-3
    for s, segs in enumerate(sc.polys):
        for b in blocks:
            tc = (b * sc.N + sc.N / 2) / sc.fs
            fd = (synth.tau_eval(segs, np.array([tc + h]))[0] - synth.tau_eval(segs, np.array([tc - h]))[0]) / (2 * h)
            assert abs(rate[s, b] - fd) <= 1e-12 + 1e-6 * abs(fd), (s, b, rate[s, b], fd)


def test_pre_f_equals_post_f_at_zero_rate():
    fs, nchan = 1024.0, 16
    N = 2 * nchan
    S, nsub, npol = 3, 2, 1
    tint = 8 * N / fs
    # fractional delays 0.3, 0.47, 0.64 samples: the slopes do not cancel in the cross-products
    polys = [[synth.Segment(0.0, ((2.3 + 4.17 * s) / fs, 0, 0, 0, 0, 0))] for s in range(S)]
    T = 3 * 8 * N + 64
    streams = [synth.random_bytes(12, s, T * nsub * npol // 4 + 4) for s in range(S)]
    args = (S, nsub, npol, nchan, fs, tint, [130.0, 377.5], polys, streams, [0] * S, [T] * S)
    post, wpost = oracle.Oracle(*args).correlate(0, 3)
    pre, wpre = oracle.Oracle(*args, rotation=oracle.ROT_PRE_F).correlate(0, 3)
    assert np.array_equal(wpre, wpost)
    assert np.max(np.abs(pre - post)) <= 1e-12 * np.max(np.abs(post))
    # and the phase really is non-trivial: nu0 tau is several turns
    assert np.max(np.abs(np.angle(post[:, 1]))) > 0.1


@pytest.fixture(scope="module")
def spacecraft_scan():
    """A spacecraft (0.7 s delay, 1.3e-5 s/s) and a ground station at
    nu0 = 4.8 GHz, 256 channels (16 us blocks): the differential fringe phase
    drifts by 0.99 turns per block, so post-F keeps |sinc(0.99)| = 1% of the
    fringe, and a phase referenced to the block start instead of its centre
    would be off by half of that, 0.495 turns.  0.1 s at 32 Msample/s,
    correlation 0.02."""
    fs = 32e6
    polys = [[synth.Segment(0.0, (0.7, 1.3e-5, 0, 0, 0, 0))], [synth.Segment(0.0, (3e-3, 1e-7, 0, 0, 0, 0))]]
    sc = synth.Scan(2, 1, 1, 256, fs, 0.1, 0.1, 0.02, 9, [4.8e9], polys)
    synth.plan_windows(sc)
    streams = [synth.station_bytes(sc, s) for s in range(2)]
    return sc, streams


def coherence(vis, k0=8, k1=224):
    """Band-averaged normalised cross-spectrum (channels [k0, k1): the lowest
    ones hold the image of the negative frequencies shifted by the fringe
    rate, the top eighth the generator's interpolator roll-off)."""
    a0, a1, cr = vis[0].real[k0:k1], vis[2].real[k0:k1], vis[1][k0:k1]
    return np.mean(cr / np.sqrt(a0 * a1)), 1.0 / math.sqrt(6250 * (k1 - k0))


def test_pre_f_recovers_coherence_at_spacecraft_rate(spacecraft_scan):
    sc, streams = spacecraft_scan
    eta = 0.8825  # 2-bit efficiency at +-0.98 sigma, levels 1 / 3.336 (pinned in test_oracle_pins)
    vis_pre, w = oracle.Oracle.from_scan(sc, streams, rotation=oracle.ROT_PRE_F).correlate(0, 1)
    vis_post, _ = oracle.Oracle.from_scan(sc, streams).correlate(0, 1)
    assert np.all(w == 6250)
    r_pre, sigma = coherence(vis_pre[0, :, 0])
    r_post, _ = coherence(vis_post[0, :, 0])
    assert abs(r_pre.real - eta * sc.rho) < 4 * sigma, (r_pre, eta * sc.rho, sigma)
    assert abs(r_pre.imag) < 4 * sigma, r_pre
    drift = 4.8e9 * (1.3e-5 - 1e-7) * sc.N / sc.fs     # turns per block
    assert abs(r_post) < 0.25 * eta * sc.rho, (r_post, abs(np.sinc(drift)))
    # the upper half of the band (where a missing fractional-delay slope
    # would cost the most coherence) on its own
    r_hi, sig_hi = coherence(vis_pre[0, :, 0], 128, 224)
    assert abs(r_hi.real - eta * sc.rho) < 4 * sig_hi and abs(r_hi.imag) < 4 * sig_hi, (r_hi, sig_hi)
