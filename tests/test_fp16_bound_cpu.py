"""The FP16 tolerance's derivation, checked on the CPU with IEEE binary16
rounding (numpy's float16: 11 significant bits, round to nearest even).

The FP16 tests state a bound of 1e-3 relative RMS per baseline from three
numbers: a Gaussian component rounds with about 2.1e-4 RMS relative error
(half an ulp, 2^-11 of the leading bit, uniform: 2^-11 / sqrt(3), times
sqrt(E[1/m^2]) ~ 0.74 over the mantissa m in [1, 2)); a noise-dominated
cross-product sum inherits sqrt(2) times that, about 3e-4 (the bench
measures 3.0e-4); and the largest of 2080 baselines, each estimated over
only 32 channels, sits well below 1e-3.  The spectra here are at the F
step's FP16 scale for N = 2048 (X * 2^-5, component RMS near 1.5)."""
import numpy as np


def f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def test_binary16_grid_points():
    assert f16(1.0) == 1.0 and f16(1.0 + 2 ** -10) == 1.0 + 2 ** -10
    assert f16(1.0 + 2 ** -11) == 1.0                       # tie to even
    assert f16(1.0 + 3 * 2 ** -11) == 1.0 + 2 ** -9         # tie to even (up)
    assert f16(65504.0) == 65504.0


def test_relative_rounding_of_a_gaussian_component_is_about_2_1e_4():
    rng = np.random.default_rng(3)
    x = rng.normal(scale=1.5, size=2_000_000)
    rel = np.sqrt(np.mean((f16(x) - x) ** 2) / np.mean(x ** 2))
    assert 1.8e-4 < rel < 2.4e-4, rel


def test_noise_dominated_cross_products_and_the_worst_baseline():
    """V = sum_b X_a conj(X_b) over 1000 blocks of independent noise spectra:
    the rel-RMS of the FP16 sum against the exact one is about 3e-4, and the
    worst of 2080 baseline estimates over 32 channels stays far below the
    1e-3 bound."""
    rng = np.random.default_rng(4)
    M, K, NBL = 1000, 32, 2080
    worst = 0.0
    errs = []
    for _ in range(NBL // 40):          # 52 draws x 40 baselines = 2080
        Xa = rng.normal(scale=1.5, size=(40, M, K)) + 1j * rng.normal(scale=1.5, size=(40, M, K))
        Xb = rng.normal(scale=1.5, size=(40, M, K)) + 1j * rng.normal(scale=1.5, size=(40, M, K))
        q = lambda z: f16(z.real) + 1j * f16(z.imag)
        V = np.sum(Xa * np.conj(Xb), axis=1)
        Vq = np.sum(q(Xa) * np.conj(q(Xb)), axis=1)
        e = np.sqrt(np.sum(np.abs(Vq - V) ** 2, axis=1) / np.sum(np.abs(V) ** 2, axis=1))
        errs.extend(e.tolist())
        worst = max(worst, float(e.max()))
    mean = float(np.mean(errs))
    assert 2.5e-4 < mean < 4.5e-4, mean
    assert worst < 1e-3 / 1.5, worst      # the bound keeps at least 1.5x room
