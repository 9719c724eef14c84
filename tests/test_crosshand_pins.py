"""Pins of the oracle's cross-hand polarisation products.

With two polarisations per subband the X step can form all four hand
products V_ab^pq = sum over blocks of X_a^p conj(X_b^q) (pq = 00, 01, 10,
11; for circular feeds RR, RL, LR, LL), which the polarisation key science
programmes of the paper's AO-1 correlation need (Sec. 1).  Fixed by:
* the parallel hands (00, 11) are exactly the parallel-hand products;
* an autocorrelation's 10 product is exactly the conjugate of its 01 product;
* data: station 1's second polarisation carries station 0's first, delayed
  by a whole number of samples (no fringe rotation), so V_01^01 equals the
  autocorrelation V_00^00 bit for bit while the other hand pairs hold
  unrelated noise -- this fixes which polarisation of which station each
  hand index takes.
"""
import numpy as np
import pytest

import oracle
import synth


def small_scan(seed=3, S=3, nsub=2, nchan=16, nblk_int=6, nint=2):
    fs = 1024.0
    N = 2 * nchan
    tint = nblk_int * N / fs
    polys = [[synth.Segment(0.0, ((1.3 + 2.2 * s) / fs, 3e-4 * s, 0, 0, 0, 0))] for s in range(S)]
    T = nint * nblk_int * N + 64
    streams = [synth.random_bytes(seed, s, T * nsub * 2 // 4 + 4) for s in range(S)]
    return oracle.Oracle(S, nsub, 2, nchan, fs, tint, [150.0, 37.0][:nsub], polys, streams, [0] * S, [T] * S)


def test_parallel_hands_are_the_parallel_products():
    o = small_scan()
    par, wpar = o.correlate(0, 2)             # [ni, nbl, G, nchan], stream j = 2 sb + p
    cross, w = o.correlate_cross(0, 2)         # [ni, nbl, nsub, 4, nchan]
    assert np.array_equal(w, wpar)
    for sb in range(o.nsub):
        assert np.array_equal(cross[:, :, sb, 0], par[:, :, 2 * sb])
        assert np.array_equal(cross[:, :, sb, 3], par[:, :, 2 * sb + 1])


def test_autocorrelation_cross_hands_are_conjugates():
    o = small_scan(seed=4)
    cross, _ = o.correlate_cross(0, 2)
    S = o.S
    autos = [a * S - a * (a - 1) // 2 for a in range(S)]
    for bl in autos:
        assert np.array_equal(cross[:, bl, :, 2], np.conj(cross[:, bl, :, 1]))
        assert np.all(cross[:, bl, :, 0].imag == 0) and np.all(cross[:, bl, :, 3].imag == 0)
    assert np.max(np.abs(cross[:, 1, :, 1])) > 0  # cross-hands of a cross baseline are not trivial


def test_cross_hand_of_an_exact_copy_is_the_autocorrelation():
    fs, nchan, m = 1024.0, 16, 7
    N = 2 * nchan
    nblk_int, nint = 8, 2
    T = nblk_int * nint * N + 32
    rng = np.random.default_rng(12)
    base = rng.integers(0, 4, (T + m,)).astype(np.uint8)
    c0 = np.stack([base[m:], rng.integers(0, 4, T)], axis=1).astype(np.uint8)            # station 0: (R, L)
    c1 = np.stack([rng.integers(0, 4, T + m), base], axis=1).astype(np.uint8)            # station 1: L = station 0's R, m later
    segs = [[synth.Segment(0.0, (0.0,) * 6)], [synth.Segment(0.0, (m / fs, 0, 0, 0, 0, 0))]]
    o = oracle.Oracle(2, 1, 2, nchan, fs, nblk_int * N / fs, [0.0], segs, [synth.pack(c0), synth.pack(c1)], [0, 0],
                      [T, T + m])
    cross, w = o.correlate_cross(0, nint)
    assert np.all(w == nblk_int)
    v00, v01 = cross[:, 0, 0], cross[:, 1, 0]   # baselines (0,0) and (0,1)
    assert np.array_equal(v01[:, 1], v00[:, 0])  # X_0^R conj(X_1^L) = X_0^R conj(X_0^R)
    for pq in (0, 2, 3):                          # the other hand pairs hold unrelated noise
        assert np.max(np.abs(v01[:, pq] - v00[:, 0])) > 0.1 * np.max(np.abs(v00[:, 0]))
