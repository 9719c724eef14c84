"""The FP8 tolerance's derivation, checked on the CPU with an E4M3 rounding
written out from the format's definition: 4 significant bits (3 stored),
exponents -6..8, subnormals in steps of 2^-9, largest value 448, round to
nearest even, saturating.

The tensor-core FP8 tests state a bound of 8e-2 relative RMS per baseline
from two numbers: E4M3 rounds a Gaussian component with ~2.6% RMS relative
error, and a noise-dominated cross-product sum inherits sqrt(2) times that
(~3.7%).  Both are measured here on synthetic spectra at the F step's FP8
scale (component RMS near 8)."""
import numpy as np


def e4m3(x):
    """Round to the nearest E4M3 value (ties to even), saturating at +-448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -9)))
    e = np.clip(e, -6, 8)                   # below 2^-6: subnormal spacing 2^-9
    step = 2.0 ** (e - 3)                   # 3 stored mantissa bits
    q = np.round(a / step) * step           # numpy rounds halves to even
    q = np.minimum(q, 448.0)
    return np.sign(x) * q


def test_e4m3_grid_points():
    assert e4m3(1.0) == 1.0 and e4m3(1.125) == 1.125 and e4m3(1.0625) == 1.0   # tie to even
    assert e4m3(448.0) == 448.0 and e4m3(1e6) == 448.0 and e4m3(-500.0) == -448.0
    assert e4m3(2.0 ** -9) == 2.0 ** -9 and e4m3(2.0 ** -11) == 0.0
    assert e4m3(17.0) == 16.0 and e4m3(19.0) == 20.0            # spacing 2 in [16, 32)


def test_relative_rounding_of_a_gaussian_component_is_about_2_6_percent():
    rng = np.random.default_rng(1)
    x = rng.normal(scale=8.0, size=2_000_000)
    rel = np.sqrt(np.mean((e4m3(x) - x) ** 2) / np.mean(x ** 2))
    assert 0.022 < rel < 0.030, rel


def test_noise_dominated_cross_products_inherit_sqrt2_times_that():
    """V = sum_b X_a conj(X_b) over 2000 blocks of independent noise spectra
    (64 channels): the rel-RMS of the E4M3 sum against the exact one is
    sqrt(2) x the per-component figure, ~3.7%, below the 8e-2 bound."""
    rng = np.random.default_rng(2)
    M, K = 2000, 64
    Xa = rng.normal(scale=8.0, size=(M, K)) + 1j * rng.normal(scale=8.0, size=(M, K))
    Xb = rng.normal(scale=8.0, size=(M, K)) + 1j * rng.normal(scale=8.0, size=(M, K))
    q = lambda z: e4m3(z.real) + 1j * e4m3(z.imag)
    V = np.sum(Xa * np.conj(Xb), axis=0)
    Vq = np.sum(q(Xa) * np.conj(q(Xb)), axis=0)
    err = np.sqrt(np.sum(np.abs(Vq - V) ** 2) / np.sum(np.abs(V) ** 2))
    assert 0.030 < err < 0.045, err
    assert err < 8e-2
