"""The tensor-core X step (tcgen05, FP32 accumulation in TMEM) from FP16 and
from FP8 (E4M3) spectra, against the FP64 oracle.

Stated bounds, relative RMS per baseline:
  FP16 <= 1e-3: FP16 keeps 11 significant bits; rounding a spectrum value
       to it leaves a relative error of about 2.1e-4 RMS per component
       (tests/test_fp16_bound_cpu.py), and for noise-dominated baselines the
       error terms d_a conj(X_b) + X_a conj(d_b) add like the visibility
       itself, about sqrt(2) x 2.1e-4 = 3e-4 (measured 3.0-3.5e-4).  A baseline's estimate
       over only 32 channels scatters by ~1/sqrt(64), and the largest of 2080
       baselines sits ~1.7x above the mean (measured 4.8e-4); 1e-3 leaves 2x
       room above that and still fails a regression of a few ulps.
  FP8  <= 8e-2: E4M3 keeps 4 significant bits, a relative rounding error of
       about 2.6% RMS per component; for noise-dominated baselines
       (X_a conj(X_b) summed over blocks of uncorrelated noise) the error
       terms d_a conj(X_b) + X_a conj(d_b) add like the visibility itself,
       so the expected rel-RMS is sqrt(2) x 2.6% = 3.7% (measured 3.8-3.9%).
       A baseline's estimate over only 32 channels scatters by ~1/sqrt(64),
       and the largest of 2080 such baselines (64 stations) sits ~3.5 sigma
       above the mean, ~1.7 x 3.7% = 6.3%: the bound leaves room for that.
The correlation coefficient between the reduced-precision and the FP64
visibilities (the SNR-equivalent efficiency) is printed with the error.
Weights are exact: validity is integer work shared with the FP32 path.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP16 = 1e-3
TOL_FP8 = 8e-2


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


def run_tc(corr, sc, streams, nint, precision=None, unit=None):
    c = corr.from_scan(sc, streams)
    c.set_precision(corr.CORR_PREC_FP16_TC if precision is None else precision)
    if unit is not None:
        c.set_x_unit(unit)
    outs, ws = [], []
    for _ in range(nint):
        r = c.correlate()
        assert r is not None
        outs.append(r[0])
        ws.append(r[1])
    c.close()
    return np.stack(outs), np.stack(ws)


def efficiency(v, ref):
    """Correlation coefficient of the visibilities with the FP64 ones."""
    v, ref = v.ravel(), ref.ravel()
    return float(np.real(np.vdot(ref, v)) / np.sqrt(np.vdot(v, v).real * np.vdot(ref, ref).real))


def check(sc, vis, w, ref, wref, nint, label, tol=TOL_FP16, name="FP16"):
    assert np.array_equal(w, wref)
    worst, eff = 0.0, 1.0
    for i in range(nint):
        v = vis[i].reshape(sc.nbl, sc.G, sc.nchan)
        assert np.all(np.isfinite(v)), label
        err = rel_rms_per_baseline(v, ref[i])
        worst = max(worst, float(err.max()))
        eff = min(eff, efficiency(v, ref[i]))
        assert np.all(err < tol), (label, i, err.max())
    print("%s: %s X step, max rel-RMS per baseline %.3e, efficiency %.6f" % (label, name, worst, eff))
    return worst


UNITS = pytest.mark.parametrize("unit", ["tensor", "auto"])


def unit_of(corr, name):
    return corr.CORR_X_TENSOR_CORES if name == "tensor" else corr.CORR_X_AUTO


def test_tc_config2_slice(corr, unit):
    """10 stations, 8 subbands x 2 pols, 1024 channels: on the tensor cores
    6 channels of 20 rows per 128-row tile, 12-channel work items, a 0.05 s
    integration of 781.25 blocks (ragged last K tile); by default (10
    stations) the FP16 spectra go to the CUDA-core X step."""
    sc = synth.config2(seed=2, duration=0.1, tint=0.05, boundary=0.05)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2, unit=unit_of(corr, unit))
    check(sc, vis, w, ref, wref, 2, "cfg2 slice (%s)" % unit)


test_tc_config2_slice = UNITS(test_tc_config2_slice)


def test_tc_64_stations(corr):
    """64 stations fill a whole 128-row tile with one channel (config-3
    station count, 4096 channels, 64 Msample/s), two integrations of 130.5
    blocks."""
    fs = 64e6
    N = 8192
    tint = 130.5 * N / fs
    sc = synth.config2(seed=3, duration=2 * tint, tint=tint, boundary=tint, nchan=4096, stations=64, nsub=1, npol=1,
                       fs=fs, nu0_base=1.6e9)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2)
    check(sc, vis, w, ref, wref, 2, "64 stations")


@UNITS
@pytest.mark.parametrize("nchan,S,nsub,npol", [(256, 2, 1, 1), (64, 3, 3, 1), (512, 7, 2, 2), (128, 33, 1, 1),
                                               (2048, 5, 3, 1), (32, 64, 1, 1)])
def test_tc_shapes(corr, nchan, S, nsub, npol, unit):
    """Tiles of 32, 21, 9 and 1 channels, odd stream counts, a slice wider
    than the band, 8-byte copies; 4096-point FFTs whose FP16 spectra are
    corner-turned into tiles (12 channels per tile pair, a ragged last
    corner-turn CTA); 64 stations, one channel per tile.  By default the
    shapes of up to 12 stations and 128+ channels take the CUDA-core X step
    on the same FP16 spectra."""
    fs = 32e6
    N = 2 * nchan
    tint = round((300 * N + 5) / fs * fs) / fs
    sc = synth.config2(seed=nchan + S, duration=2 * tint, tint=tint, boundary=tint, nchan=nchan, stations=S,
                       nsub=nsub, npol=npol)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2, unit=unit_of(corr, unit))
    check(sc, vis, w, ref, wref, 2, "S=%d nchan=%d G=%d (%s)" % (S, nchan, nsub * npol, unit))


def test_tc_rejects_more_than_64_stations(corr):
    c = corr.Correlator(65, 1, 1, 64, 0.001)
    with pytest.raises(corr.CorrError) as ei:
        c.set_precision(corr.CORR_PREC_FP16_TC)
    assert ei.value.code == corr.CORR_EINVAL
    c.close()


def test_tc_two_bit_efficiency_config1(corr, cfg1):
    """End to end through the tensor-core path: the band-averaged normalised
    cross-correlation of config 1 equals eta * rho (Bussgang, 2-bit at
    +-0.98 sigma), as on the FP64 oracle."""
    import math
    sc, streams, o = cfg1
    vis, w = run_tc(corr, sc, streams, 1)
    v = vis[0].reshape(sc.nbl, sc.G, sc.nchan)[:, 0, :]
    k = slice(8, 224)
    r = np.mean(v[1, k] / np.sqrt(v[0, k].real * v[2, k].real))
    p_in = math.erf(0.98 / math.sqrt(2))
    eta = (2 / math.pi) * (1 + 2.336 * math.exp(-0.98 ** 2 / 2)) ** 2 / (p_in + 3.336 ** 2 * (1 - p_in))
    sigma = 1.0 / math.sqrt(62500 * (k.stop - k.start))
    assert abs(r.real - eta * sc.rho) < 4 * sigma, (r, eta * sc.rho)


# ---- FP8 (E4M3) spectra -----------------------------------------------------

@UNITS
def test_fp8_config2_slice(corr, unit):
    """FP8 tiles written by the F step itself (1024 channels, 128-block K
    tiles, a ragged last tile of the 781.25-block integration), or by
    default E4M3 spectra read by the CUDA-core X step."""
    sc = synth.config2(seed=2, duration=0.1, tint=0.05, boundary=0.05)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2, corr.CORR_PREC_FP8_TC, unit=unit_of(corr, unit))
    check(sc, vis, w, ref, wref, 2, "cfg2 slice (%s)" % unit, TOL_FP8, "FP8")


def test_fp8_64_stations(corr):
    """Config-3 station count and FFT length: FP8 spectra of 8192-point FFTs
    corner-turned into tiles (k_tiles8), one channel per 128-row tile."""
    fs = 64e6
    N = 8192
    tint = 130.5 * N / fs
    sc = synth.config2(seed=3, duration=2 * tint, tint=tint, boundary=tint, nchan=4096, stations=64, nsub=1, npol=1,
                       fs=fs, nu0_base=1.6e9)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2, corr.CORR_PREC_FP8_TC)
    check(sc, vis, w, ref, wref, 2, "64 stations", TOL_FP8, "FP8")


@UNITS
@pytest.mark.parametrize("nchan,S,nsub,npol", [(256, 2, 1, 1), (64, 3, 3, 1), (512, 7, 2, 2), (2048, 5, 3, 1),
                                               (32, 64, 1, 1)])
def test_fp8_shapes(corr, nchan, S, nsub, npol, unit):
    """Direct FP8 tiles at several tile fillings and stream counts, and the
    FP8 corner turn for 4096-point FFTs; about 300 blocks per integration,
    so each integration ends in a ragged 128-block K tile."""
    fs = 32e6
    N = 2 * nchan
    tint = round((300 * N + 5) / fs * fs) / fs
    sc = synth.config2(seed=nchan + S, duration=2 * tint, tint=tint, boundary=tint, nchan=nchan, stations=S,
                       nsub=nsub, npol=npol)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(S)]
    ref, wref = oracle.Oracle.from_scan(sc, streams).correlate(0, 2)
    vis, w = run_tc(corr, sc, streams, 2, corr.CORR_PREC_FP8_TC, unit=unit_of(corr, unit))
    check(sc, vis, w, ref, wref, 2, "S=%d nchan=%d G=%d (%s)" % (S, nchan, nsub * npol, unit), TOL_FP8, "FP8")


def test_fp8_two_bit_efficiency_config1(corr, cfg1):
    """The Bussgang 2-bit efficiency survives FP8 spectra: the band-averaged
    normalised cross-correlation of config 1 is eta * rho within the
    statistical error (the FP8 rounding noise averages down over 62,500
    blocks)."""
    import math
    sc, streams, o = cfg1
    vis, w = run_tc(corr, sc, streams, 1, corr.CORR_PREC_FP8_TC)
    v = vis[0].reshape(sc.nbl, sc.G, sc.nchan)[:, 0, :]
    k = slice(8, 224)
    r = np.mean(v[1, k] / np.sqrt(v[0, k].real * v[2, k].real))
    p_in = math.erf(0.98 / math.sqrt(2))
    eta = (2 / math.pi) * (1 + 2.336 * math.exp(-0.98 ** 2 / 2)) ** 2 / (p_in + 3.336 ** 2 * (1 - p_in))
    sigma = 1.0 / math.sqrt(62500 * (k.stop - k.start))
    assert abs(r.real - eta * sc.rho) < 4 * sigma, (r, eta * sc.rho)


def test_fp8_rejects_more_than_64_stations(corr):
    c = corr.Correlator(65, 1, 1, 64, 0.001)
    with pytest.raises(corr.CorrError) as ei:
        c.set_precision(corr.CORR_PREC_FP8_TC)
    assert ei.value.code == corr.CORR_EINVAL
    c.close()


def test_cuda_core_and_tensor_core_x_agree(corr):
    """The two units multiply the same FP16 spectra (the F kernels share
    their arithmetic): exact products, FP32 sums in another order (and the
    tensor cores' own accumulation), so the results agree far inside the
    FP16 bound (5e-5 against 1e-3), and the weights are identical."""
    sc = synth.config2(seed=21, duration=0.02, tint=0.01, boundary=0.01, nchan=512, stations=6, nsub=2, npol=1)
    streams = [synth.station_bytes(sc, s, physics=False) for s in range(sc.stations)]
    vt, wt = run_tc(corr, sc, streams, 2, unit=corr.CORR_X_TENSOR_CORES)
    vc, wc = run_tc(corr, sc, streams, 2, unit=corr.CORR_X_CUDA_CORES)
    assert np.array_equal(wt, wc)
    for i in range(2):
        err = rel_rms_per_baseline(vc[i].reshape(sc.nbl, -1), vt[i].reshape(sc.nbl, -1))
        assert np.all(err < 5e-5), err.max()


def test_x_unit_argument_errors(corr):
    c = corr.Correlator(4, 1, 1, 256, 0.001)
    for unit in (corr.CORR_X_AUTO, corr.CORR_X_CUDA_CORES, corr.CORR_X_TENSOR_CORES):
        c.set_x_unit(unit)
    for bad in (-1, 3):
        with pytest.raises(corr.CorrError) as ei:
            c.set_x_unit(bad)
        assert ei.value.code == corr.CORR_EINVAL
    c.close()
