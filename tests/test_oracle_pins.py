"""Pins of the FP64 oracle against facts it does not compute itself.

Each test fixes one part of the method by something other than the oracle's
own formula: hand-derived bit patterns, exact rational arithmetic, the
brute-force DFT, the lag-domain (XF) form of the cross-spectrum, closed forms
of 2-bit quantisation (Bussgang's theorem), and the position of an injected
fringe.  The paper itself prints no numbers for the correlator path.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
LUT = np.array(oracle.DEFAULT_LUT)


# --------------------------------------------------------------------------
# helpers written independently of the oracle


def my_codes(stream_bytes, G, j, t0, count):
    """Independent numpy unpack: bit 2*(t*G+j) of an LSB-first bit stream."""
    bits = np.unpackbits(np.asarray(stream_bytes, np.uint8), bitorder="little")
    m = (np.arange(t0, t0 + count) * G + j) * 2
    return (bits[m] + 2 * bits[m + 1]).astype(np.uint8)


def tiny_scan(seed=5, nchan=8, S=3, nsub=2, npol=1, fs=1024.0, nblk_int=4, nint=2, nu0=(300.0, 123.4),
              polys=None):
    N = 2 * nchan
    tint = nblk_int * N / fs
    if polys is None:
        polys = [
            [synth.Segment(0.0, ((2 + 0.3) / fs, 1e-3, 0, 0, 0, 0))],
            [synth.Segment(0.0, (0.0,) * 6)],
            [synth.Segment(0.0, (-5.6 / fs, -2e-4, 0, 0, 0, 0))],
        ][:S]
    sc = synth.Scan(S, nsub, npol, nchan, fs, nint * tint, tint, 0.0, seed, list(nu0[:nsub]), polys)
    synth.plan_windows(sc, margin=N)
    streams = [synth.random_bytes(seed, s, sc.nsamp[s] * sc.G // 4 + 4) for s in range(S)]
    return sc, streams


# --------------------------------------------------------------------------
# T1: unpacking


def _golden_patterns():
    out = []
    with open(os.path.join(HERE, "golden", "unpack_patterns.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kv = dict(p.split("=") for p in line.split())
            out.append((int(kv["G"]), bytes.fromhex(kv["bytes"]), int(kv["j"]),
                        [int(c) for c in kv["codes"].split(",")]))
    return out


@pytest.mark.parametrize("G,raw,j,codes", _golden_patterns())
def test_unpack_hand_patterns(G, raw, j, codes):
    got = oracle.unpack_codes(np.frombuffer(raw, np.uint8), G, j, 0, len(codes))
    assert got.tolist() == codes


@pytest.mark.parametrize("G", [1, 2, 3, 4, 5, 8, 16, 32])
def test_unpack_roundtrip_every_position(G):
    # every code value at every bit position of a 32-bit word
    T = 64
    rng = np.random.default_rng(G)
    codes = rng.integers(0, 4, (T, G)).astype(np.uint8)
    codes[:4, :] = np.arange(4)[:, None]
    packed = synth.pack(codes)
    for j in range(G):
        assert np.array_equal(oracle.unpack_codes(packed, G, j, 0, T), codes[:, j])
        assert np.array_equal(my_codes(packed, G, j, 0, T), codes[:, j])


# --------------------------------------------------------------------------
# T1b: integer delay and segment selection


def _const_poly_oracle(c0, fs=32e6, nchan=8, t0=0.0, extra=None):
    segs = [synth.Segment(t0, (c0, 0, 0, 0, 0, 0))] + (extra or [])
    return oracle.Oracle(1, 1, 1, nchan, fs, 16 * nchan * 2 / fs, [0.0], [segs],
                         [np.zeros(64, np.uint8)], [-(1 << 40)], [1 << 41])


def test_integer_delay_near_ties_exact():
    """n_b = floor(fma(tau, fs, 0.5)) must equal the floor of the correctly
    rounded exact value tau*fs + 1/2, including taus one ulp around a tie."""
    fs = 32e6
    taus = []
    for m in (0, 1, 3, 7, 123, 38_400_000, -1, -17):
        t = (m + 0.5) / fs
        taus += [t, np.nextafter(t, 1.0), np.nextafter(t, -1.0), m / fs, np.nextafter(m / fs, -1.0)]
    for tau in taus:
        o = _const_poly_oracle(float(tau), fs)
        n, e, t, v = o.delays(0, 1)
        exact = Fraction(float(tau)) * Fraction(fs) + Fraction(1, 2)
        want = math.floor(float(exact))  # float() of a Fraction rounds to nearest, ties to even
        assert int(n[0, 0]) == want, (tau, int(n[0, 0]), want)
        assert t[0, 0] == tau
        assert e[0, 0] == float(tau) - want / fs


def test_segment_selection_and_ties():
    """Block centre t_c picks the segment with the largest t0 <= t_c."""
    fs, nchan = 1024.0, 8
    N = 2 * nchan
    tb = 5 * N / fs + (N / 2) / fs  # exact centre of block 5
    segs = [synth.Segment(0.0, (0.0,) * 6), synth.Segment(tb, (7.0 / fs, 0, 0, 0, 0, 0))]
    o = oracle.Oracle(1, 1, 1, nchan, fs, 1.0, [0.0], [segs], [np.zeros(64, np.uint8)], [-(1 << 30)], [1 << 31])
    n, e, t, v = o.delays(0, 10)
    assert n[0].tolist() == [0] * 5 + [7] * 5
    # before the first segment the block is not covered, hence not valid
    segs2 = [synth.Segment(tb, (0.0,) * 6)]
    o2 = oracle.Oracle(1, 1, 1, nchan, fs, 1.0, [0.0], [segs2], [np.zeros(64, np.uint8)], [-(1 << 30)], [1 << 31])
    assert o2.delays(0, 10)[3][0].tolist() == [0] * 5 + [1] * 5


def test_integer_shift_is_exact_copy():
    """A station delayed by exactly m samples, holding the same samples
    shifted by m, gives cross = auto exactly (window-selection sign)."""
    fs, nchan, m = 1024.0, 16, 11
    N = 2 * nchan
    T = 40 * N
    rng = np.random.default_rng(3)
    codes = rng.integers(0, 4, (T + m, 1)).astype(np.uint8)
    a = synth.pack(codes[m:])          # station 0: sample t -> codes[t+m], starts at 0
    b = synth.pack(codes)              # station 1: delayed by m, its sample t+m = station 0's t
    segs0 = [synth.Segment(0.0, (0.0,) * 6)]
    segs1 = [synth.Segment(0.0, (m / fs, 0, 0, 0, 0, 0))]
    tint = 8 * N / fs
    o = oracle.Oracle(2, 1, 1, nchan, fs, tint, [0.0], [segs0, segs1], [a, b], [0, 0], [T, T + m])
    vis, w = o.correlate(0, 3)
    assert np.all(w == 8)
    assert np.array_equal(vis[:, 1], vis[:, 0])
    assert np.array_equal(vis[:, 2], vis[:, 0])


# --------------------------------------------------------------------------
# T3: FFT


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024])
def test_fft_vs_bruteforce_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    D = np.exp(-2j * np.pi * np.outer(k, k) / n)
    ref = D @ x
    got = oracle.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    assert np.allclose(got, np.fft.fft(x), rtol=0, atol=1e-11 * max(1, n))
    back = oracle.fft(got, inverse=True) / n
    assert np.max(np.abs(back - x)) < 1e-12


# --------------------------------------------------------------------------
# T2: FX = XF on tiny inputs


def test_fx_equals_xf():
    sc, streams = tiny_scan()
    o = oracle.Oracle.from_scan(sc, streams)
    S, G, N, nch = sc.stations, sc.G, sc.N, sc.nchan
    vis, w = o.correlate(0, 2)
    nper = int(round(sc.tint * sc.fs)) // N
    n_b, eps, tau, valid = o.delays(0, 2 * nper)
    k = np.arange(nch)
    lag = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(k, lag) / N)
    for i in range(2):
        for j in range(G):
            acc = np.zeros((S * (S + 1) // 2, nch), complex)
            wt = np.zeros(S * (S + 1) // 2)
            for b in range(i * nper, (i + 1) * nper):
                xs, rs = [], []
                for s in range(S):
                    t0 = b * N + n_b[s, b] - sc.sample0[s]
                    xs.append(LUT[my_codes(streams[s], G, j, t0, N)] if valid[s, b] else None)
                    phi = (sc.nu0[j // sc.npol] * tau[s, b]) % 1.0
                    rs.append(np.exp(2j * np.pi * (phi + k * sc.fs / N * eps[s, b])))
                bl = 0
                for a in range(S):
                    for c in range(a, S):
                        if xs[a] is not None and xs[c] is not None:
                            cl = np.array([np.dot(np.roll(xs[a], -l), xs[c]) for l in range(N)])
                            acc[bl] += rs[a] * np.conj(rs[c]) * (E @ cl)
                            wt[bl] += 1
                        bl += 1
            ref = acc / np.maximum(wt, 1)[:, None] / N
            assert np.array_equal(w[i], wt)
            assert np.max(np.abs(vis[i, :, j] - ref)) < 1e-12 * np.max(np.abs(ref))


# --------------------------------------------------------------------------
# T4: Hermitian structure


def test_hermitian_and_real_positive_autos():
    sc, streams = tiny_scan(seed=9, nchan=16, S=3, nsub=2, nblk_int=6)
    o = oracle.Oracle.from_scan(sc, streams)
    full, wf = o.correlate(0, 2, full=True)
    S = sc.stations
    V = full.reshape(2, S, S, sc.G, sc.nchan)
    for a in range(S):
        assert np.all(V[:, a, a].imag == 0.0)
        assert np.all(V[:, a, a].real > 0.0)
        for b in range(S):
            assert np.array_equal(V[:, b, a], np.conj(V[:, a, b]))
    tri, _ = o.correlate(0, 2)
    iu = [(a, b) for a in range(S) for b in range(a, S)]
    for bl, (a, b) in enumerate(iu):
        assert np.array_equal(tri[:, bl], V[:, a, b])


# --------------------------------------------------------------------------
# T5 / T7: 2-bit quantisation closed forms on config-1 data


def two_bit_constants(v0=0.98, n=3.336):
    p_in = math.erf(v0 / math.sqrt(2.0))
    power = p_in + n * n * (1.0 - p_in)
    eta = (2.0 / math.pi) * (1.0 + (n - 1.0) * math.exp(-v0 * v0 / 2.0)) ** 2 / power
    return eta, power


def test_two_bit_closed_forms_values():
    eta, power = two_bit_constants()
    assert abs(eta - 0.8825) < 5e-4
    assert abs(power - 4.3130) < 5e-4


@pytest.mark.slow
def test_auto_level_config1(cfg1):
    sc, streams, o = cfg1
    vis, w = cached_cfg1_vis(o)
    _, power = two_bit_constants()
    for bl in (0, 2):
        auto = vis[0, bl, 0].real
        # sigma of a mean of 62500*256 chi-square(2)-like terms ~ power/sqrt(M*nchan)
        assert abs(auto.mean() - power) < 4 * power / math.sqrt(62500 * 256) + 2e-3


_VIS = {}


def cached_cfg1_vis(o):
    if id(o) not in _VIS:
        _VIS[id(o)] = o.correlate(0, 1)
    return _VIS[id(o)]


@pytest.mark.slow
def test_two_bit_efficiency_config1(cfg1):
    """|V_01| / sqrt(V_00 V_11) over the band = eta * rho for the injected
    correlation rho = 0.02 when the delay model is the true one."""
    sc, streams, o = cfg1
    vis, w = cached_cfg1_vis(o)
    assert np.all(w == 62500)
    eta, _ = two_bit_constants()
    k = slice(8, 224)  # the generator's interpolator rolls off in the top eighth
    a0, a1, cr = vis[0, 0, 0].real[k], vis[0, 2, 0].real[k], vis[0, 1, 0][k]
    r = np.mean(cr / np.sqrt(a0 * a1))
    sigma = 1.0 / math.sqrt(62500 * (k.stop - k.start))
    assert abs(r.real - eta * sc.rho) < 4 * sigma, (r, eta * sc.rho, sigma)
    assert abs(r.imag) < 4 * sigma


# --------------------------------------------------------------------------
# T6: fringe at the injected delay and rate


def _lag_peak(V, N, lags):
    k = np.arange(V.size)
    L = np.exp(2j * np.pi * np.outer(lags, k) / N) @ V
    i = int(np.argmax(np.abs(L)))
    return lags[i], L[i]


@pytest.mark.slow
def test_fringe_peak_with_true_model_is_at_zero(cfg1):
    sc, streams, o = cfg1
    vis, _ = cached_cfg1_vis(o)
    lag, val = _lag_peak(vis[0, 1, 0], sc.N, np.arange(-8, 8, 0.02))
    assert abs(lag) < 0.05
    assert abs(np.angle(val)) < 0.05


@pytest.mark.slow
def test_fringe_delay_rate_search_with_zero_model(cfg1):
    """Correlating with tau = 0 leaves the injected delay in the data; a
    delay-rate search over 1/256 s sub-integrations (the kind of wide-window
    fringe search the paper describes for RadioAstron, Sec. 2) must find one
    peak at the injected 3.7 samples and 2e-6 s/s."""
    sc, streams, _ = cfg1
    zero = [[synth.Segment(0.0, (0.0,) * 6)] for _ in range(sc.stations)]
    nsi = 256
    o = oracle.Oracle(sc.stations, sc.nsub, sc.npol, sc.nchan, sc.fs, 1.0 / nsi, sc.nu0, zero,
                      streams, sc.sample0, sc.nsamp)
    vis, w = o.correlate(0, nsi)
    V = vis[:, 1, 0, :]
    up = 8
    pad = np.zeros((nsi, sc.N * up), complex)
    pad[:, :sc.nchan] = V
    A = np.fft.ifft(pad, axis=1) * pad.shape[1]      # A[i, m]: lag transform at lag m/up samples
    t = (np.arange(nsi) + 0.5) / nsi
    taus = np.arange(-8.0, 16.0, 1.0 / up)
    best = (-1.0, None, None)
    rows = np.arange(nsi)[None, None, :]
    for rates in np.array_split(np.arange(-1e-5, 1e-5, 2.5e-8), 8):
        lag = taus[None, :, None] + rates[:, None, None] * sc.fs * t[None, None, :]
        idx = np.rint(lag * up).astype(np.int64) % pad.shape[1]
        rot = np.exp(2j * np.pi * sc.nu0[0] * rates[:, None] * t[None, :])[:, None, :]
        amp = np.abs((A[rows, idx] * rot).sum(axis=2))
        r, k = np.unravel_index(int(np.argmax(amp)), amp.shape)
        if amp[r, k] > best[0]:
            best = (amp[r, k], taus[k], rates[r])
    peak, tau0, rate = best
    assert abs(tau0 - 3.7) <= 0.2, best
    assert abs(rate - 2e-6) <= 5e-8, best


# --------------------------------------------------------------------------
# T1b (continued): every term of the quintic delay polynomial


def _horner_exact(coeffs, u):
    """The polynomial's exact value in rational arithmetic (power form, not Horner)."""
    return sum(Fraction(c) * Fraction(u) ** i for i, c in enumerate(coeffs))


def _one_station_delays(fs, nchan, segs, b):
    o = oracle.Oracle(1, 1, 1, nchan, fs, 64 * 2 * nchan / fs, [0.0], [segs], [np.zeros(64, np.uint8)],
                      [-(1 << 50)], [1 << 51])
    n, e, t, v = o.delays(b, 1)
    return int(n[0, 0]), float(e[0, 0]), float(t[0, 0])


def test_quintic_delay_exact_dyadic():
    """With dyadic coefficients and block centres every step of the FP64
    evaluation is exact, so tau must equal the exact polynomial value bit for
    bit: a dropped or shifted term (c4, c5 included) changes it.  fs = 2^20
    makes tau*fs + 1/2 exact, so n_b and eps are fixed exactly too."""
    fs, nchan = float(1 << 20), 8
    N = 2 * nchan
    rng = np.random.default_rng(20)
    for case in range(300):
        b = int(rng.integers(0, 20000))
        tc = Fraction(b * N + N // 2) / Fraction(int(fs))
        u = Fraction(int(rng.integers(1, 32)), 8)
        t0 = tc - u
        # every term matters; all of them fit one 53-bit significand together
        coeffs = [float(Fraction(int(rng.integers(-63, 64)), 1 << int(rng.integers(4, 20)))) for _ in range(6)]
        coeffs[5] = float(Fraction(int(rng.choice([-1, 1]) * rng.integers(1, 64)), 1 << int(rng.integers(0, 8))))
        exact = _horner_exact(coeffs, u)
        assert Fraction(float(exact)) == exact  # representable: the evaluation has no rounding to hide a slip
        n_b, eps, tau = _one_station_delays(fs, nchan, [synth.Segment(float(t0), tuple(coeffs))], b)
        assert Fraction(tau) == exact, (case, coeffs, float(u))
        want_n = math.floor(exact * int(fs) + Fraction(1, 2))
        assert n_b == want_n
        assert Fraction(eps) == exact - Fraction(want_n, int(fs))
        # dropping c5 (or starting the evaluation at c4) must be visible
        assert _horner_exact(coeffs[:5], u) != exact


def test_quintic_delay_ties_through_all_terms():
    """c0 placed so that tau*fs is exactly m + 1/2 (ties go up, n_b = m+1), and
    2^-13 samples either side of it, with all six coefficients non-zero."""
    fs, nchan = float(1 << 20), 8
    N = 2 * nchan
    rng = np.random.default_rng(21)
    for case in range(60):
        b = int(rng.integers(0, 5000))
        tc = Fraction(b * N + N // 2) / Fraction(int(fs))
        u = Fraction(int(rng.integers(1, 32)), 8)
        hi = [float(Fraction(int(rng.integers(1, 64)), 1 << int(rng.integers(4, 16)))) for _ in range(5)]
        m = int(rng.integers(-(1 << 18), 1 << 18))
        for frac_samples, want in ((Fraction(1, 2), m + 1), (Fraction(1, 2) + Fraction(1, 8192), m + 1),
                                   (Fraction(1, 2) - Fraction(1, 8192), m)):
            target = (m + frac_samples) / Fraction(int(fs))
            c0 = target - sum(Fraction(c) * u ** (i + 1) for i, c in enumerate(hi))
            assert Fraction(float(c0)) == c0
            coeffs = [float(c0)] + hi
            n_b, eps, tau = _one_station_delays(fs, nchan, [synth.Segment(float(tc - u), tuple(coeffs))], b)
            assert Fraction(tau) == target
            assert n_b == want, (case, m, frac_samples, n_b)
            assert Fraction(eps) == target - Fraction(want, int(fs))


def test_quintic_delay_realistic_within_rounding_bound():
    """Spacecraft-like quintic segments (tau ~ 1 s, rate 3e-5, 120 s segments)
    at non-dyadic fs: tau stays within the FP64 rounding bound of the exact
    value (Horner with one rounding per step: 6 * 2^-53 * sum |c_i u^i|), and
    n_b follows the exact value wherever it is not within that bound of a
    tie.  (The exact dyadic cases above fix each term; this one fixes the
    rounding behaviour at the workloads' magnitudes.)"""
    fs, nchan = 32e6, 512
    N = 2 * nchan
    rng = np.random.default_rng(22)
    checked = 0
    for case in range(200):
        coeffs = (float(rng.uniform(0.3, 1.2)), float(rng.uniform(-3e-5, 3e-5)), float(rng.uniform(-1, 1) * 1e-9),
                  float(rng.uniform(-1, 1) * 1e-12), float(rng.uniform(-1, 1) * 1e-15),
                  float(rng.uniform(-1, 1) * 1e-18))
        t0 = -float(rng.uniform(0.0, 120.0))
        b = int(rng.integers(0, 300000))
        tc = Fraction(b * N + N // 2) / Fraction(fs)
        u = Fraction(float(tc)) - Fraction(t0)  # the oracle forms t_c in FP64, then t_c - t0
        u = Fraction(float(u))
        exact = _horner_exact(coeffs, u)
        n_b, eps, tau = _one_station_delays(fs, nchan, [synth.Segment(t0, coeffs)], b)
        terms = [abs(Fraction(c) * u ** i) for i, c in enumerate(coeffs)]
        bound = 6 * Fraction(1, 1 << 53) * sum(terms)
        assert abs(Fraction(tau) - exact) <= bound
        x = exact * Fraction(fs) + Fraction(1, 2)
        if abs(x - round(x)) > 4 * bound * Fraction(fs):
            assert n_b == math.floor(x)
            checked += 1
    assert checked > 150


# --------------------------------------------------------------------------
# D6: integration membership when fs*tint is not a whole number of blocks


def test_ragged_integration_membership():
    """fs*tint = 120 samples = 7.5 blocks of 16: block b belongs to integration
    floor(b*N / (fs*tint)), so integrations hold 8, 7, 8, 7 blocks.  The
    weights must be those brute-force counts and each integration's
    unnormalised sum must be exactly the sum of its own blocks' products."""
    fs, nchan = 1024.0, 8
    N = 2 * nchan
    spi = 120
    tint = spi / fs
    nint = 4
    S = 2
    T = nint * spi + 4 * N
    rng = np.random.default_rng(7)
    streams = [synth.pack(rng.integers(0, 4, (T, 1)).astype(np.uint8)) for _ in range(S)]
    segs = [[synth.Segment(0.0, (0.0,) * 6)], [synth.Segment(0.0, (3.0 / fs, 0, 0, 0, 0, 0))]]
    o = oracle.Oracle(S, 1, 1, nchan, fs, tint, [0.0], segs, streams, [0, 0], [T, T])
    vis, w = o.correlate(0, nint)
    nblocks = -(-nint * spi // N)
    member = [math.floor(Fraction(b * N, spi)) for b in range(nblocks)]
    counts = [member.count(i) for i in range(nint)]
    assert counts == [8, 7, 8, 7]
    for i in range(nint):
        assert w[i].tolist() == [counts[i]] * 3
        acc = np.zeros((3, nchan), complex)
        for b in (b for b in range(nblocks) if member[b] == i):
            X = [o.spectrum(s, 0, b)[0] for s in range(S)]
            acc += np.array([X[0] * np.conj(X[0]), X[0] * np.conj(X[1]), X[1] * np.conj(X[1])])
        got = vis[i, :, 0] * (counts[i] * N)
        assert np.max(np.abs(got - acc)) <= 1e-12 * np.max(np.abs(acc))


# --------------------------------------------------------------------------
# D5: a block is valid exactly when every sample of its window exists


@pytest.mark.parametrize("lead", [0, 1])
@pytest.mark.parametrize("tail", [0, 1])
def test_validity_at_the_data_edges(lead, tail):
    """A station whose data start exactly at block 0's window (lead = 0) or one
    sample later (lead = 1), and end exactly at block 6's window end
    (tail = 0) or one sample earlier (tail = 1).  The first and last blocks
    are valid only when all their samples exist, and a valid edge block's
    spectrum is the DFT of exactly the first (last) N samples present."""
    fs, nchan, m = 1024.0, 8, 5
    N = 2 * nchan
    first = m + lead              # window of block 0 starts at station sample m
    end = 6 * N + m + N - tail    # window of block 6 ends at 6N + m + N
    T = end - first
    rng = np.random.default_rng(8 + 2 * lead + tail)
    codes = rng.integers(0, 4, (T, 1)).astype(np.uint8)
    stream = synth.pack(codes)
    segs = [[synth.Segment(0.0, (m / fs, 0, 0, 0, 0, 0))]]
    o = oracle.Oracle(1, 1, 1, nchan, fs, 8 * N / fs, [0.0], segs, [stream], [first], [T])
    n, e, t, v = o.delays(0, 8)
    assert n[0].tolist() == [m] * 8
    want = [1] * 8
    want[7] = 0                   # block 7 needs samples beyond block 6's window end
    if lead:
        want[0] = 0
    if tail:
        want[6] = 0
    assert v[0].tolist() == want
    k = np.arange(nchan)
    D = np.exp(-2j * np.pi * np.outer(k, np.arange(N)) / N)
    X0, ok0 = o.spectrum(0, 0, 0)
    X6, ok6 = o.spectrum(0, 0, 6)
    assert ok0 == (not lead) and ok6 == (not tail)
    if not lead:
        ref = D @ LUT[my_codes(stream, 1, 0, 0, N)]
        assert np.max(np.abs(X0 - ref)) < 1e-12 * np.max(np.abs(ref))
    if not tail:
        ref = D @ LUT[my_codes(stream, 1, 0, T - N, N)]
        assert np.max(np.abs(X6 - ref)) < 1e-12 * np.max(np.abs(ref))
    else:
        assert np.all(X6 == 0)
