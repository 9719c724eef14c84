"""Pins of the oracle's delay-rate fringe search (the wide-window fringe
search the paper lists for RadioAstron, Sec. 2): the zero-padded 2-D inverse
DFT of one baseline's visibilities over sub-integration x channel, and its
peak.  Checked against closed forms, brute-force double sums and the shift
theorem, so that a wrong sign, a transposed axis or a missing pad fails."""
import numpy as np
import pytest

import oracle


def brute(V, Nr, Nd):
    T, K = V.shape
    t = np.arange(T)[:, None, None, None]
    k = np.arange(K)[None, :, None, None]
    r = np.arange(Nr)[None, None, :, None]
    l = np.arange(Nd)[None, None, None, :]
    ph = np.exp(2j * np.pi * (k * l / Nd + t * r / Nr))
    return (V[:, :, None, None] * ph).sum(axis=(0, 1))


def test_map_is_the_double_sum():
    rng = np.random.default_rng(5)
    V = rng.normal(size=(3, 5)) + 1j * rng.normal(size=(3, 5))
    M = oracle.fringe_map(V, 4, 8)
    assert M.shape == (4, 8)
    assert np.allclose(M, brute(V, 4, 8), rtol=0, atol=1e-12)


@pytest.mark.parametrize("r0,l0", [(3, 11), (0, 0), (13, 60), (1, 63)])
def test_tone_peaks_at_its_bins_with_amplitude_T_K(r0, l0):
    """V[t][k] = A exp(-2 pi i (k l0/Nd + t r0/Nr)) sums coherently at (r0, l0):
    amplitude A T K there; every other bin is smaller.  l0 = 63 of 64 is a
    lag of -1 (negative lags wrap to the top of the axis)."""
    T, K, Nr, Nd, A = 12, 40, 16, 64, 0.75
    t = np.arange(T)[:, None]
    k = np.arange(K)[None, :]
    V = A * np.exp(-2j * np.pi * (k * l0 / Nd + t * r0 / Nr))
    amp = np.abs(oracle.fringe_map(V, Nr, Nd))
    r, l, a = oracle.fringe_peak(amp)
    assert (r, l) == (r0, l0)
    assert a == pytest.approx(A * T * K, rel=1e-12)
    others = amp.copy()
    others[r0, l0] = 0
    assert others.max() < 0.99 * a


def test_shift_theorem_fixes_the_signs_of_both_axes():
    """Multiplying V by exp(+2 pi i (k d / Nd + t e / Nr)) moves the map to
    M'[r][l] = M[r + e][l + d] (indices mod the pads); the wrong exponent sign
    or swapped axes would move it the other way."""
    rng = np.random.default_rng(9)
    T, K, Nr, Nd, d, e = 6, 10, 8, 16, 5, 3
    V = rng.normal(size=(T, K)) + 1j * rng.normal(size=(T, K))
    t = np.arange(T)[:, None]
    k = np.arange(K)[None, :]
    M = oracle.fringe_map(V, Nr, Nd)
    M2 = oracle.fringe_map(V * np.exp(2j * np.pi * (k * d / Nd + t * e / Nr)), Nr, Nd)
    assert np.allclose(M2, np.roll(np.roll(M, -e, axis=0), -d, axis=1), atol=1e-10)


def test_ties_go_to_the_smaller_flat_index():
    amp = np.zeros((4, 8))
    amp[2, 1] = amp[1, 5] = amp[3, 0] = 7.0
    assert oracle.fringe_peak(amp) == (1, 5, 7.0)


def test_pads_must_cover_the_data():
    with pytest.raises(ValueError):
        oracle.fringe_map(np.ones((5, 4)), 4, 8)
