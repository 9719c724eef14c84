"""Seeded synthetic station streams shaped like a RadioAstron + ground VLBI scan.

This module only makes inputs.  It holds none of the correlator's arithmetic:
no window selection, no FFT, no fringe rotation, no cross-multiplication.  Both
the FP64 oracle and the CUDA path consume what it writes, and neither imports
the other.

Signal model (one stream = one subband x polarisation of one station):

    x_s(t_s) = sqrt(rho) * Re{ (c + i H[c])(t_g) * exp(-2 pi i nu0 tau_s(t_g)) }
               + sqrt(1 - rho) * n_s(t_s)

where t_s is the station-clock time of a sample, t_g the geocentric time that
satisfies t_g + tau_s(t_g) = t_s (solved by fixed-point iteration), c a unit
white Gaussian common to all stations, H the Hilbert transform, and n_s an
independent unit white Gaussian.  c is sampled on the geocentric grid and
brought to t_g with a 64-tap Blackman-Harris-windowed sinc interpolator.
The delay tau_s(t) comes from the same per-station polynomial segments that
the correlator is given, so a correct correlator removes it exactly
(the paper: the delay model supplies per-station delays, Sec. 2).

Quantisation: 2-bit codes at +-0.98 sigma (sigma = 1): x < -0.98 -> 0,
-0.98 <= x < 0 -> 1, 0 <= x < 0.98 -> 2, x >= 0.98 -> 3.  Packing: one byte
stream per station; the code of stream j at sample-time t sits at bit offset
2*(t*G + j) of a little-endian bit stream (bytes LSB first), G = nsub*npol
streams interleaved as j = sb*npol + pol.

Random numbers: numpy's Philox4x32-10 counter-based generator (Salmon et al.
2011), keyed by (seed, tag, stream, page) and drawn in fixed pages of 2**16
samples, so that any window of any stream is reproducible on its own.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

PAGE = 1 << 16
QUANT_T = 0.98
TAG_COMMON = 0xC0
TAG_NOISE = 0x10
TAG_POLY = 0x70
TAG_CODES = 0x3C

# 4-term Blackman-Harris coefficients (Harris 1978).
_BH = (0.35875, 0.48829, 0.14128, 0.01168)
_NTAP = 64
_Q = 512  # fractional-delay quantum of the interpolator table (1/512 sample)


@dataclasses.dataclass
class Segment:
    """One delay-polynomial segment: tau(t) = sum_i c_i (t - t0)^i seconds."""
    t0: float
    coeffs: Tuple[float, ...]  # 6 entries, c0..c5


@dataclasses.dataclass
class Scan:
    """A synthetic scan: shapes, delay model and per-station stream windows."""
    stations: int
    nsub: int
    npol: int
    nchan: int
    fs: float
    duration: float
    tint: float
    rho: float
    seed: int
    nu0: List[float]                     # sky (LO) frequency per subband, Hz
    polys: List[List[Segment]]           # per station, sorted by t0
    sample0: List[int] = dataclasses.field(default_factory=list)  # first station sample of each stream
    nsamp: List[int] = dataclasses.field(default_factory=list)    # sample-time groups per station

    @property
    def G(self) -> int:
        return self.nsub * self.npol

    @property
    def N(self) -> int:
        return 2 * self.nchan

    @property
    def nbl(self) -> int:
        return self.stations * (self.stations + 1) // 2


# ----------------------------------------------------------------------------
# random pages


def _key(seed: int, tag: int, a: int, b: int) -> int:
    return ((seed & 0xFFFFFFFF) << 96) | ((tag & 0xFFFF) << 80) | ((a & 0xFFFFFFFF) << 48) | (b & 0xFFFFFFFFFFFF)


def _rng(seed: int, tag: int, a: int, b: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=_key(seed, tag, a, b)))


def normals(seed: int, tag: int, stream: int, start: int, count: int) -> np.ndarray:
    """Unit normals for sample indices [start, start+count) of one keyed stream."""
    if count <= 0:
        return np.zeros(0)
    p0 = start // PAGE
    p1 = (start + count - 1) // PAGE + 1
    buf = np.empty((p1 - p0) * PAGE)
    for p in range(p0, p1):
        # page index may be negative for windows before the scan epoch
        buf[(p - p0) * PAGE:(p - p0 + 1) * PAGE] = _rng(seed, tag, stream, p & 0xFFFFFFFFFFFF).standard_normal(PAGE)
    off = start - p0 * PAGE
    return buf[off:off + count]


# ----------------------------------------------------------------------------
# delay model (the generator's own evaluation, used only to inject delays)


def tau_eval(segs: Sequence[Segment], t: np.ndarray) -> np.ndarray:
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    t0s = np.array([s.t0 for s in segs])
    idx = np.searchsorted(t0s, t, side="right") - 1
    idx = np.clip(idx, 0, len(segs) - 1)
    for i, s in enumerate(segs):
        m = idx == i
        if np.any(m):
            out[m] = np.polynomial.polynomial.polyval(t[m] - s.t0, np.array(s.coeffs))
    return out


def _geo_time_exact(segs: Sequence[Segment], ts: np.ndarray) -> np.ndarray:
    tg = ts - tau_eval(segs, ts)
    for _ in range(3):
        tg = ts - tau_eval(segs, tg)
    return tg


def _geo_time(segs: Sequence[Segment], ts: np.ndarray, step: int = 128) -> Tuple[np.ndarray, np.ndarray]:
    """Solve t_g + tau(t_g) = t_s; returns (t_g, tau(t_g)).  The delay is
    smooth on the scale of microseconds, so the solution is taken exactly on
    a grid every `step` samples and linearly interpolated in between (the
    interpolation error is below 1e-18 s for the delay models used here)."""
    if all(not any(s.coeffs) for s in segs):
        return ts.copy(), np.zeros_like(ts)
    n = ts.size
    idx = np.arange(0, n + step, step)
    idx[-1] = min(idx[-1], n - 1)
    idx = np.unique(np.minimum(idx, n - 1))
    tgc = _geo_time_exact(segs, ts[idx])
    # interpolate the (small) offset ts - tg, not tg itself, to keep precision
    off = np.interp(np.arange(n), idx, ts[idx] - tgc)
    tg = ts - off
    return tg, off


def taylor_segment(t0: float, derivs: Sequence[float]) -> Segment:
    """Segment from the derivatives tau^(i)(t0), i = 0..5."""
    c = [0.0] * 6
    for i, d in enumerate(derivs[:6]):
        c[i] = d / math.factorial(i)
    return Segment(float(t0), tuple(c))


# ----------------------------------------------------------------------------
# interpolator


def _interp_table() -> np.ndarray:
    """H[q, t'] = sinc(f - t) * BH(f - t), f = q/Q, t = t' - 31, t' = 0..63."""
    q = np.arange(_Q)[:, None] / _Q
    t = np.arange(_NTAP)[None, :] - (_NTAP // 2 - 1)
    x = q - t
    z = (x + _NTAP / 2) / _NTAP
    a0, a1, a2, a3 = _BH
    w = a0 - a1 * np.cos(2 * np.pi * z) + a2 * np.cos(4 * np.pi * z) - a3 * np.cos(6 * np.pi * z)
    return np.sinc(x) * w


_HTAB: Optional[np.ndarray] = None


def _htab() -> np.ndarray:
    global _HTAB
    if _HTAB is None:
        _HTAB = _interp_table()
    return _HTAB


def _interpolate(sig: np.ndarray, g0: int, u: np.ndarray) -> np.ndarray:
    """Band-limited value of sig (sampled at integer geocentric indices
    g0, g0+1, ...) at fractional indices u, by runs of constant table row."""
    H = _htab()
    m = np.floor(u).astype(np.int64)
    fi = np.rint((u - m) * _Q).astype(np.int64)
    carry = fi >= _Q
    m[carry] += 1
    fi[carry] = 0
    j = np.arange(u.size, dtype=np.int64)
    d = m - j
    change = np.flatnonzero((np.diff(d) != 0) | (np.diff(fi) != 0)) + 1
    starts = np.concatenate(([0], change))
    ends = np.concatenate((change, [u.size]))
    out = np.empty(u.size)
    half = _NTAP // 2 - 1
    for a, b in zip(starts.tolist(), ends.tolist()):
        dd = int(d[a])
        lo = a + dd - half - g0
        seg = sig[lo: lo + (b - a) + _NTAP - 1]
        out[a:b] = np.correlate(seg, H[int(fi[a])], "valid")
    return out


def _hilbert(x: np.ndarray) -> np.ndarray:
    n = x.size
    X = np.fft.rfft(x)
    X *= -1j
    X[0] = 0
    if n % 2 == 0:
        X[-1] = 0
    return np.fft.irfft(X, n)


# ----------------------------------------------------------------------------
# stream windows


def plan_windows(scan: Scan, margin: int = 64) -> None:
    """Choose, per station, the first station sample and the sample count so
    that every block of [0, duration) can be read after delay tracking."""
    nblk_t = np.linspace(0.0, scan.duration, 257)
    scan.sample0, scan.nsamp = [], []
    span = int(round(scan.duration * scan.fs))
    for segs in scan.polys:
        tau = tau_eval(segs, nblk_t)
        lo = int(math.floor(tau.min() * scan.fs)) - margin
        hi = span + int(math.ceil(tau.max() * scan.fs)) + scan.N + margin
        s0 = (lo // 16) * 16
        n = ((hi - s0 + 15) // 16) * 16
        scan.sample0.append(s0)
        scan.nsamp.append(n)


# ----------------------------------------------------------------------------
# codes and packing


def quantise(x: np.ndarray, t: float = QUANT_T) -> np.ndarray:
    """2-bit offset-binary code of each sample (sigma = 1)."""
    c = np.full(x.shape, 1, dtype=np.uint8)
    c[x < -t] = 0
    c[x >= 0] = 2
    c[x >= t] = 3
    return c


def pack(codes: np.ndarray) -> np.ndarray:
    """Pack codes[T, G] (row-major t*G + j) into bytes, LSB first, padded to
    whole 32-bit words."""
    flat = np.ascontiguousarray(codes, dtype=np.uint8).reshape(-1)
    pad = (-flat.size) % 16
    if pad:
        flat = np.concatenate((flat, np.zeros(pad, np.uint8)))
    q = flat.reshape(-1, 4)
    return (q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)).astype(np.uint8)


def station_codes(scan: Scan, s: int, physics: bool = True) -> np.ndarray:
    """Codes[nsamp, G] of station s over its planned window."""
    if not scan.sample0:
        plan_windows(scan)
    s0, n = scan.sample0[s], scan.nsamp[s]
    G = scan.G
    out = np.empty((n, G), dtype=np.uint8)
    if not physics:
        for j in range(G):
            out[:, j] = quantise(normals(scan.seed, TAG_NOISE, (s << 8) | j, s0, n))
        return out
    ts = (s0 + np.arange(n, dtype=np.float64)) / scan.fs
    tg, tau = _geo_time(scan.polys[s], ts)
    u = tg * scan.fs
    g0 = int(math.floor(u.min())) - _NTAP
    g1 = int(math.ceil(u.max())) + _NTAP
    pad = 4096 if any(v != 0.0 for v in scan.nu0) else 0
    for j in range(G):
        sb = j // scan.npol
        c = normals(scan.seed, TAG_COMMON, j, g0 - pad, g1 - g0 + 2 * pad)
        cd = _interpolate(c[pad:pad + g1 - g0], g0, u)
        nu0 = scan.nu0[sb]
        if nu0 != 0.0:
            hc = _hilbert(c)[pad:pad + g1 - g0]
            hd = _interpolate(hc, g0, u)
            ph = nu0 * tau
            ph = ph - np.floor(ph)
            sig = cd * np.cos(2 * np.pi * ph) + hd * np.sin(2 * np.pi * ph)
        else:
            sig = cd
        x = math.sqrt(scan.rho) * sig + math.sqrt(1.0 - scan.rho) * normals(scan.seed, TAG_NOISE, (s << 8) | j, s0, n)
        out[:, j] = quantise(x)
    return out


MARK5B_SYNC = 0xABADDEED
MARK5B_HEADER = 16
MARK5B_PAYLOAD = 10000


def frame(payload: np.ndarray, P: int = MARK5B_PAYLOAD, invalid=(), seconds0: int = 0) -> np.ndarray:
    """Mark5B-style frames of a packed byte stream: frames of a 16-byte header
    and P payload bytes (the last payload zero-padded).  Header word 0 is the
    sync word (little-endian) except in the frames listed in `invalid`, which
    carry 0 there (a lost or filled frame); word 1 holds the frame number in
    its low 15 bits, word 2 a seconds count; word 3 stays 0."""
    payload = np.asarray(payload, np.uint8)
    nf = -(-payload.size // P)
    out = np.zeros((nf, MARK5B_HEADER + P), np.uint8)
    body = np.zeros(nf * P, np.uint8)
    body[:payload.size] = payload
    out[:, MARK5B_HEADER:] = body.reshape(nf, P)
    words = np.zeros((nf, 4), np.uint32)
    words[:, 0] = MARK5B_SYNC
    words[:, 1] = np.arange(nf, dtype=np.uint32) & 0x7FFF
    words[:, 2] = seconds0
    for f in invalid:
        words[f, 0] = 0
    out[:, :MARK5B_HEADER] = words.view(np.uint8).reshape(nf, MARK5B_HEADER)
    return out.reshape(-1)


def station_bytes(scan: Scan, s: int, physics: bool = True) -> np.ndarray:
    return pack(station_codes(scan, s, physics))


def random_bytes(seed: int, station: int, nbytes: int) -> np.ndarray:
    """Uniformly random packed bytes (every code equally likely)."""
    return _rng(seed, TAG_CODES, station, 0).integers(0, 256, nbytes, dtype=np.uint8)


# ----------------------------------------------------------------------------
# the workloads


def config1(seed: int = 1, nu0: float = 0.0, duration: float = 1.0, rho: float = 0.02) -> Scan:
    """2 stations (space = station 0, ground = station 1), 1 subband, 1 pol,
    32 Msample/s, 256 channels (512-point FFT), one 1 s integration,
    correlation 0.02; the space station carries a cubic delay polynomial with
    a 3.7-sample offset and a 2e-6 s/s rate."""
    fs = 32e6
    r = _rng(seed, TAG_POLY, 0, 0)
    c2 = float(r.uniform(-1, 1)) * 1e-9
    c3 = float(r.uniform(-1, 1)) * 1e-11
    space = [Segment(0.0, (3.7 / fs, 2e-6, c2, c3, 0.0, 0.0))]
    ground = [Segment(0.0, (0.0,) * 6)]
    scan = Scan(2, 1, 1, 256, fs, duration, 1.0, rho, seed, [nu0], [space, ground])
    plan_windows(scan)
    return scan


def config2(seed: int = 2, duration: float = 10.0, tint: float = 1.0, boundary: float = 5.0,
            nu0_base: float = 4.8e9, rho: float = 0.02, nchan: int = 1024, stations: int = 10,
            nsub: int = 8, npol: int = 2, fs: float = 32e6, plan: bool = True) -> Scan:
    """10 stations (station 0 in space), 8 subbands x 2 pols, 1024 channels,
    quintic delay segments 120 s long with a boundary at `boundary` seconds;
    ground delays from tau = A sin(W t + p), |A| <= 20 ms, W = 7.29e-5 rad/s;
    space delay 0.3..1.2 s with rate up to 3e-5 s/s."""
    r = _rng(seed, TAG_POLY, 0, 0)
    polys = []
    t0s = (boundary - 120.0, boundary)
    for s in range(stations):
        segs = []
        if s == 0:
            tau0 = float(r.uniform(0.3, 1.2))
            rate = float(r.uniform(-3e-5, 3e-5))
            acc = float(r.uniform(-1, 1)) * 1e-9
            jerk = float(r.uniform(-1, 1)) * 1e-12
            for t0 in t0s:
                d0 = tau0 + rate * t0 + acc * t0 ** 2 / 2 + jerk * t0 ** 3 / 6
                d1 = rate + acc * t0 + jerk * t0 ** 2 / 2
                d2 = acc + jerk * t0
                segs.append(taylor_segment(t0, (d0, d1, d2, jerk, 0.0, 0.0)))
        else:
            A = float(r.uniform(-20e-3, 20e-3))
            W = 7.29e-5
            p = float(r.uniform(0, 2 * np.pi))
            for t0 in t0s:
                segs.append(taylor_segment(t0, [A * W ** i * math.sin(W * t0 + p + i * math.pi / 2) for i in range(6)]))
        polys.append(segs)
    nu0 = [nu0_base + 16e6 * sb for sb in range(nsub)]
    scan = Scan(stations, nsub, npol, nchan, fs, duration, tint, rho, seed, nu0, polys)
    if plan:
        plan_windows(scan)
    return scan


TAG_MIX = 0x4D


def scan_mix(seed: int = 4, count: int = 96, fs: float = 32e6, tint_max: float = 1.0,
             stations=(2, 20), nsub=(1, 16), npol=(1, 2), log2_nchan=(7, 13),
             duration=(0.5, 30.0)) -> List[Scan]:
    """A seeded mix of uneven scans: per scan, uniform integers for the
    station count, subbands and polarisations, a power-of-two channel count
    drawn uniformly over its exponents, and a duration drawn uniformly in
    seconds.  Station 0 of every scan is in space; delay polynomials follow
    the ten-station generator, keyed by the scan's own seed.

    Integrations: the duration is split into ceil(duration / tint_max)
    integrations of a whole number of FFT blocks each, and the duration is
    rounded to that, so that every integration is full and at most tint_max
    long."""
    r = _rng(seed, TAG_MIX, 0, 0)
    out = []
    for q in range(count):
        S = int(r.integers(stations[0], stations[1] + 1))
        sb = int(r.integers(nsub[0], nsub[1] + 1))
        pol = int(r.integers(npol[0], npol[1] + 1))
        nchan = 1 << int(r.integers(log2_nchan[0], log2_nchan[1] + 1))
        d = float(r.uniform(duration[0], duration[1]))
        N = 2 * nchan
        nint = max(1, math.ceil(d / tint_max - 1e-9))
        blocks = max(1, int(round(d * fs / nint / N)))
        tint = blocks * N / fs
        sc = config2(seed=(seed << 16) + q, duration=nint * tint, tint=tint, boundary=nint * tint / 2,
                     nchan=nchan, stations=S, nsub=sb, npol=pol, fs=fs)
        out.append(sc)
    return out


def integrations(scan: Scan) -> int:
    """Whole integrations in the scan."""
    return int(round(scan.duration / scan.tint))
