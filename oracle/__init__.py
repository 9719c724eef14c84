"""FP64 CPU oracle of the FX correlator hot path (ctypes wrapper of fx_oracle.c).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library; the two meet only at the seeded inputs written by the
``synth`` package.  See fx_oracle.c for the readings it implements.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

DEFAULT_LUT = (-3.336, -1.0, 1.0, 3.336)


def build(force: bool = False) -> str:
    """Compile fx_oracle.c with gcc (no FP contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scan(C.Structure):
    _fields_ = [
        ("S", C.c_int), ("nsub", C.c_int), ("npol", C.c_int), ("nchan", C.c_int),
        ("fs", C.c_double), ("tint", C.c_double), ("lut", C.c_double * 4),
        ("nu0", C.c_void_p), ("nseg", C.c_void_p), ("seg_t0", C.c_void_p), ("seg_c", C.c_void_p),
        ("maxseg", C.c_int),
        ("bytes", C.c_void_p), ("byte_off", C.c_void_p), ("sample0", C.c_void_p), ("nsamp", C.c_void_p),
        ("rotation", C.c_int), ("frame_payload", C.c_int),
    ]

ROT_POST_F = 0   # fringe rotation after the transform, at the block centre (the default)
ROT_PRE_F = 1    # per-sample fringe rotation before a complex transform


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.oracle_delays.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P]
        L.oracle_delays_ex.argtypes = [P, C.c_int64, C.c_int64, P, P, P, P, P]
        L.oracle_correlate_ex.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
        L.oracle_correlate_ex.restype = C.c_int
        L.oracle_correlate_cross.argtypes = [P, C.c_int64, C.c_int, P, P]
        L.oracle_correlate_cross.restype = C.c_int
        L.oracle_spectrum.argtypes = [P, C.c_int, C.c_int, C.c_int64, P]
        L.oracle_spectrum.restype = C.c_int
        L.oracle_fft.argtypes = [P, P, C.c_int, C.c_int]
        L.oracle_unpack_codes.argtypes = [P, C.c_int, C.c_int, C.c_int64, C.c_int64, P]
        L.oracle_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Oracle:
    """One scan held for the oracle.

    ``polys``: per station, a list of (t0, coeffs[6]) with increasing t0.
    ``streams``: per station, packed bytes (uint8) starting at station sample
    ``sample0[s]`` and holding ``nsamp[s]`` sample-time groups.
    """

    def __init__(self, stations: int, nsub: int, npol: int, nchan: int, fs: float, tint: float,
                 nu0: Sequence[float], polys, streams: Sequence[np.ndarray],
                 sample0: Sequence[int], nsamp: Sequence[int], lut=DEFAULT_LUT, rotation: int = ROT_POST_F,
                 frame_payload: int = 0):
        S = stations
        self.S, self.nsub, self.npol, self.nchan = S, nsub, npol, nchan
        self.G = nsub * npol
        self.N = 2 * nchan
        self.fs, self.tint = float(fs), float(tint)
        maxseg = max(len(p) for p in polys)
        self._nu0 = np.ascontiguousarray(nu0, dtype=np.float64)
        self._nseg = np.array([len(p) for p in polys], dtype=np.int32)
        self._t0 = np.zeros(S * maxseg)
        self._c = np.zeros(S * maxseg * 6)
        for s, segs in enumerate(polys):
            for i, seg in enumerate(segs):
                t0, co = (seg.t0, seg.coeffs) if hasattr(seg, "t0") else seg
                self._t0[s * maxseg + i] = t0
                self._c[(s * maxseg + i) * 6:(s * maxseg + i + 1) * 6] = np.asarray(co, dtype=np.float64)
        offs, tot = [], 0
        for b in streams:
            offs.append(tot)
            tot += len(b)
        self._bytes = np.concatenate([np.asarray(b, dtype=np.uint8) for b in streams]) if tot else np.zeros(1, np.uint8)
        self._off = np.array(offs, dtype=np.int64)
        self._s0 = np.asarray(sample0, dtype=np.int64).copy()
        self._ns = np.asarray(nsamp, dtype=np.int64).copy()
        self._lens = [len(b) for b in streams]
        self._sc = _Scan(S, nsub, npol, nchan, self.fs, self.tint, (C.c_double * 4)(*lut),
                         _ptr(self._nu0), _ptr(self._nseg), _ptr(self._t0), _ptr(self._c), maxseg,
                         _ptr(self._bytes), _ptr(self._off), _ptr(self._s0), _ptr(self._ns), int(rotation),
                         int(frame_payload))
        self.frame_payload = int(frame_payload)

    @classmethod
    def from_scan(cls, scan, streams, lut=DEFAULT_LUT, nsamp=None, rotation=ROT_POST_F):
        return cls(scan.stations, scan.nsub, scan.npol, scan.nchan, scan.fs, scan.tint, scan.nu0,
                   scan.polys, streams, scan.sample0, nsamp if nsamp is not None else scan.nsamp, lut,
                   rotation)

    @property
    def nbl(self) -> int:
        return self.S * (self.S + 1) // 2

    def delays(self, b0: int, nb: int, rate: bool = False):
        """(n_b, eps, tau, valid), each [S, nb]; with rate=True also the delay
        rate d tau/dt at each block centre."""
        n = np.zeros((self.S, nb), np.int64)
        e = np.zeros((self.S, nb))
        t = np.zeros((self.S, nb))
        v = np.zeros((self.S, nb), np.uint8)
        r = np.zeros((self.S, nb))
        lib().oracle_delays_ex(C.byref(self._sc), b0, nb, _ptr(n), _ptr(e), _ptr(t), _ptr(v), _ptr(r))
        return (n, e, t, v, r) if rate else (n, e, t, v)

    def _check_bytes(self):
        for s, n in enumerate(self._lens):
            if self.frame_payload > 0:   # payload bytes of the whole frames present
                n = (n // (16 + self.frame_payload)) * self.frame_payload
            if self._ns[s] * self.G * 2 > n * 8:
                raise ValueError("station %d: %d groups need more than %d bytes" % (s, self._ns[s], n))

    def correlate(self, i0: int = 0, ni: int = 1, j0: int = 0, nj: Optional[int] = None, full: bool = False):
        """Visibilities [ni, nbl, nj, nchan] complex128 and weights [ni, nbl]."""
        self._check_bytes()
        nj = self.G - j0 if nj is None else nj
        nbl = self.S * self.S if full else self.nbl
        vis = np.zeros((ni, nbl, nj, self.nchan, 2))
        w = np.zeros((ni, nbl))
        rc = lib().oracle_correlate_ex(C.byref(self._sc), i0, ni, j0, nj, int(full), _ptr(vis), _ptr(w))
        if rc != 0:
            raise ValueError("oracle: fs*tint must be a whole number of samples")
        return vis[..., 0] + 1j * vis[..., 1], w

    def correlate_cross(self, i0: int = 0, ni: int = 1):
        """Both hands of two polarisations: visibilities [ni, nbl, nsub, 4, nchan]
        complex128 (hand products pq = 00, 01, 10, 11: X_a^p conj(X_b^q)) and
        weights [ni, nbl]."""
        self._check_bytes()
        if self.npol != 2:
            raise ValueError("cross-hand products need two polarisations")
        vis = np.zeros((ni, self.nbl, self.nsub, 4, self.nchan, 2))
        w = np.zeros((ni, self.nbl))
        rc = lib().oracle_correlate_cross(C.byref(self._sc), i0, ni, _ptr(vis), _ptr(w))
        if rc != 0:
            raise ValueError("oracle: fs*tint must be a whole number of samples")
        return vis[..., 0] + 1j * vis[..., 1], w

    def spectrum(self, s: int, j: int, b: int):
        self._check_bytes()
        out = np.zeros((self.nchan, 2))
        ok = lib().oracle_spectrum(C.byref(self._sc), s, j, b, _ptr(out))
        return out[:, 0] + 1j * out[:, 1], bool(ok)


def fft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """The oracle's own radix-2 FFT (length a power of two)."""
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    lib().oracle_fft(_ptr(re), _ptr(im), x.size, int(inverse))
    return re + 1j * im


def unpack_codes(stream: np.ndarray, G: int, j: int, t0: int, count: int) -> np.ndarray:
    stream = np.ascontiguousarray(stream, dtype=np.uint8)
    out = np.zeros(count, np.uint8)
    lib().oracle_unpack_codes(_ptr(stream), G, j, t0, count, _ptr(out))
    return out


def threads() -> int:
    return int(lib().oracle_threads())


# ---- delay-rate fringe search (the wide-window fringe search of Sec. 2) ----
#
# The map of one baseline's visibilities V[t][k] (t: sub-integration, k:
# channel) over lag l and rate bin r is the zero-padded two-dimensional
# inverse DFT, unnormalised:
#     M[r][l] = | sum_t sum_k V[t][k] exp(+2 pi i (k l / Nd + t r / Nr)) |,
# l < Nd (lag l ~ l N / Nd samples, l >= Nd/2 read as l - Nd), r < Nr (fringe
# rate r / (Nr T_sub), r >= Nr/2 read as r - Nr).  The peak is the largest
# amplitude, the smaller flat index r * Nd + l on ties.  numpy's inverse FFT
# (times Nr * Nd) is the library step for the double sum.

def fringe_map(V: np.ndarray, pad_rate: int, pad_delay: int) -> np.ndarray:
    """Complex delay-rate map [pad_rate][pad_delay] of V[nsub][nchan] (FP64)."""
    V = np.asarray(V, dtype=np.complex128)
    T, K = V.shape
    if pad_rate < T or pad_delay < K:
        raise ValueError("the padded sizes must cover the sub-integrations and channels")
    pad = np.zeros((pad_rate, pad_delay), np.complex128)
    pad[:T, :K] = V
    return np.fft.ifft2(pad) * (pad_rate * pad_delay)


def fringe_peak(amp: np.ndarray):
    """(rate bin, lag bin, amplitude) of the largest amplitude; ties go to the
    smaller flat index (numpy's argmax returns the first maximum)."""
    i = int(np.argmax(amp))
    r, l = np.unravel_index(i, amp.shape)
    return int(r), int(l), float(amp[r, l])
