"""ctypes binding of libcorr.so (include/corr.h).

Argument marshalling only: every step of the correlator runs in the CUDA
library.  The functions keep the C names; ``Correlator`` wraps a handle.
There is no CPU fallback: importing this module without a built libcorr.so,
or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcorr.so")

CORR_OK = 0
CORR_EINVAL = -1
CORR_ENOMEM = -2
CORR_EAGAIN = -3
CORR_ETIMEOUT = -4
CORR_ECUDA = -5
CORR_ESTATE = -6
CORR_EEND = -7
CORR_ETOOBIG = -8
CORR_PREC_FP32 = 0
CORR_PREC_FP16_TC = 1
CORR_PREC_FP8_TC = 2
CORR_X_AUTO = 0
CORR_X_CUDA_CORES = 1
CORR_X_TENSOR_CORES = 2
CORR_ROT_POST_F = 0
CORR_ROT_PRE_F = 1
CORR_POL_PARALLEL = 0
CORR_POL_CROSS = 1

_ERRNAMES = {0: "CORR_OK", -1: "CORR_EINVAL", -2: "CORR_ENOMEM", -3: "CORR_EAGAIN", -4: "CORR_ETIMEOUT",
             -5: "CORR_ECUDA", -6: "CORR_ESTATE", -7: "CORR_EEND", -8: "CORR_ETOOBIG"}

if not os.path.exists(LIB_PATH):
    raise ImportError("libcorr.so is not built (run __graft_entry__.build() or "
                      "python paper_1502_06894_gb300/_build.py); there is no CPU fallback")

_lib = C.CDLL(LIB_PATH)


class CorrScanDesc(C.Structure):
    """corr_scan_desc of include/corr.h."""
    _fields_ = [("stations", C.c_int), ("subbands", C.c_int), ("pols", C.c_int), ("nchan", C.c_int),
                ("fs_hz", C.c_double), ("tint_s", C.c_double), ("lut", C.c_float * 4),
                ("nu0_hz", C.c_void_p), ("nseg", C.c_void_p), ("seg_t0", C.c_void_p),
                ("seg_coeffs", C.c_void_p), ("dev_bytes", C.c_void_p), ("nbytes", C.c_void_p),
                ("first_sample", C.c_void_p)]

class CorrJob(C.Structure):
    """corr_job of include/corr.h."""
    _fields_ = [("scan", CorrScanDesc), ("precision", C.c_int), ("rotation", C.c_int), ("integrations", C.c_int64)]


RESULT_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_double),
                        C.c_int)

_P = C.c_void_p
_H = C.c_void_p
_SIGS = {
    "corr_create": ([C.POINTER(_H), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double], C.c_int),
    "corr_set_format": ([_H, C.c_double, _P], C.c_int),
    "corr_set_sky_freq": ([_H, C.c_int, C.c_double], C.c_int),
    "corr_set_precision": ([_H, C.c_int], C.c_int),
    "corr_set_x_unit": ([_H, C.c_int], C.c_int),
    "corr_set_stream": ([_H, _P], C.c_int),
    "corr_set_chunk_blocks": ([_H, C.c_int], C.c_int),
    "corr_set_pipeline": ([_H, C.c_int], C.c_int),
    "corr_set_fringe_rotation": ([_H, C.c_int], C.c_int),
    "corr_set_pol_products": ([_H, C.c_int], C.c_int),
    "corr_set_frame_format": ([_H, C.c_int], C.c_int),
    "corr_set_delay_poly": ([_H, C.c_int, C.c_double, _P], C.c_int),
    "corr_set_stream_start": ([_H, C.c_int, C.c_int64], C.c_int),
    "corr_reserve": ([_H, C.c_int, C.c_size_t], C.c_int),
    "corr_push_samples": ([_H, C.c_int, _P, C.c_size_t], C.c_int),
    "corr_push_samples_async": ([_H, C.c_int, _P, C.c_size_t], C.c_int),
    "corr_wait_pushes": ([_H], C.c_int),
    "corr_attach_samples_device": ([_H, C.c_int, _P, C.c_size_t], C.c_int),
    "corr_attach_samples_host": ([_H, C.c_int, _P, C.c_size_t], C.c_int),
    "corr_flush": ([_H], C.c_int),
    "corr_correlate": ([_H, _P, _P], C.c_int),
    "corr_correlate_device": ([_H, _P, _P], C.c_int),
    "corr_next_integration": ([_H, C.POINTER(C.c_int64)], C.c_int),
    "corr_rewind": ([_H], C.c_int),
    "corr_reset": ([_H], C.c_int),
    "corr_last_error": ([_H], C.c_char_p),
    "corr_destroy": ([_H], None),
    "corr_debug_delays": ([_H, C.c_int64, C.c_int64, _P, _P, _P, _P], C.c_int),
    "corr_debug_codes": ([_H, C.c_int, C.c_int, C.c_int64, C.c_int64, _P], C.c_int),
    "corr_debug_spectrum": ([_H, C.c_int, C.c_int, C.c_int64, _P, C.POINTER(C.c_int)], C.c_int),
    "corr_debug_set_wait_limit": ([C.c_longlong], C.c_int),
    "corr_set_profiling": ([_H, C.c_int], C.c_int),
    "corr_read_profile": ([_H, _P, _P], C.c_int),
    "corr_launch_shape": ([_H, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "corr_correlate_static": ([C.POINTER(CorrScanDesc), C.c_int64, _P, _P, _P], C.c_int),
    "corr_batch_run": ([_P, C.c_int, _P, _P, _P], C.c_int),
    "corr_device_bytes": ([_H, C.POINTER(C.c_size_t)], C.c_int),
    "corr_server_start": ([C.POINTER(_H), C.c_size_t, C.c_size_t], C.c_int),
    "corr_server_submit": ([_H, C.POINTER(CorrJob), RESULT_FN, _P, C.POINTER(C.c_int64)], C.c_int),
    "corr_server_stats": ([_H, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(C.c_int64)], C.c_int),
    "corr_server_wait": ([_H, C.c_double], C.c_int),
    "corr_server_stop": ([_H], None),
    "corr_fringe_search": ([_P, C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_float), _P, _P], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
    globals()[_name] = _f

EXPORTED = tuple(_SIGS)


class CorrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, str(code)), msg))
        self.code = code


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return int(a)


class Correlator:
    """One scan: S stations, nsub subbands x npol pols, nchan channels."""

    def __init__(self, stations: int, subbands: int, pols: int, nchan: int, tint: float,
                 fs: float = 32e6, lut: Optional[Sequence[float]] = None):
        h = _H()
        rc = corr_create(C.byref(h), stations, subbands, pols, nchan, float(tint))
        if rc != CORR_OK:
            raise CorrError(rc, corr_last_error(None).decode())
        self.h = h
        self.S, self.nsub, self.npol, self.nchan = stations, subbands, pols, nchan
        self.G = subbands * pols
        self.nbl = stations * (stations + 1) // 2
        self._keep = []
        if fs != 32e6 or lut is not None:
            lt = None if lut is None else np.asarray(lut, np.float32)
            self._check(corr_set_format(self.h, float(fs), _ptr(lt)))

    # ---------------------------------------------------------------- utils
    def _check(self, rc: int) -> int:
        if rc != CORR_OK:
            raise CorrError(rc, corr_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            corr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- setup
    def set_sky_freq(self, subband: int, nu0: float):
        self._check(corr_set_sky_freq(self.h, subband, float(nu0)))

    def set_precision(self, mode: int):
        self._check(corr_set_precision(self.h, int(mode)))

    def set_x_unit(self, unit: int):
        self._check(corr_set_x_unit(self.h, int(unit)))

    def set_fringe_rotation(self, mode: int):
        self._check(corr_set_fringe_rotation(self.h, int(mode)))

    def set_frame_format(self, payload_bytes: int):
        self._check(corr_set_frame_format(self.h, int(payload_bytes)))

    def set_pol_products(self, mode: int):
        self._check(corr_set_pol_products(self.h, int(mode)))
        self.cross = mode == CORR_POL_CROSS

    def set_pipeline(self, overlap: int):
        self._check(corr_set_pipeline(self.h, int(overlap)))

    def set_chunk_blocks(self, blocks: int):
        self._check(corr_set_chunk_blocks(self.h, int(blocks)))

    def set_stream(self, stream_handle: int):
        self._check(corr_set_stream(self.h, stream_handle))

    def set_delay_poly(self, station: int, t0: float, coeffs: Sequence[float]):
        c = np.zeros(6, np.float64)
        c[:len(coeffs)] = coeffs
        self._check(corr_set_delay_poly(self.h, station, float(t0), _ptr(c)))

    def set_stream_start(self, station: int, first_sample: int):
        self._check(corr_set_stream_start(self.h, station, int(first_sample)))

    def reserve(self, station: int, nbytes: int):
        self._check(corr_reserve(self.h, station, int(nbytes)))

    def push(self, station: int, data):
        """Append packed bytes (numpy uint8 array or a pinned host torch tensor)."""
        if isinstance(data, np.ndarray):
            data = np.ascontiguousarray(data, dtype=np.uint8)
            n = data.nbytes
        else:
            n = data.numel() * data.element_size()
        self._check(corr_push_samples(self.h, station, _ptr(data), n))

    def push_async(self, station: int, data):
        """Append pinned host bytes without waiting; keep `data` unchanged (and
        alive) until wait_pushes()."""
        if isinstance(data, np.ndarray):
            n = data.nbytes
        else:
            n = data.numel() * data.element_size()
        self._keep.append(data)
        self._check(corr_push_samples_async(self.h, station, _ptr(data), n))

    def wait_pushes(self):
        self._check(corr_wait_pushes(self.h))
        self._keep = [k for k in self._keep if hasattr(k, "is_cuda") and k.is_cuda]

    def attach_device(self, station: int, dev_tensor):
        """Use a CUDA tensor's bytes as the station's whole stream (kept alive here)."""
        self._keep.append(dev_tensor)
        n = dev_tensor.numel() * dev_tensor.element_size()
        self._check(corr_attach_samples_device(self.h, station, dev_tensor.data_ptr(), n))

    def attach_host(self, station: int, pinned):
        """Use a pinned host tensor (or array) as the station's whole stream,
        read by the kernels over the host link without a copy (kept alive here)."""
        self._keep.append(pinned)
        n = pinned.nbytes if isinstance(pinned, np.ndarray) else pinned.numel() * pinned.element_size()
        self._check(corr_attach_samples_host(self.h, station, _ptr(pinned), n))

    def flush(self):
        self._check(corr_flush(self.h))

    def rewind(self):
        self._check(corr_rewind(self.h))

    def reset(self):
        self._check(corr_reset(self.h))
        self._keep = []

    # ---------------------------------------------------------------- run
    def correlate(self, weights: bool = True):
        """Next integration -> (vis [nbl, nsub, npol, nchan] complex64, weights [nbl])
        or None when the library answers CORR_EAGAIN / CORR_EEND.  With both
        hands (set_pol_products(CORR_POL_CROSS)) vis is [nbl, nsub, 4, nchan]."""
        out = np.empty((self.nbl, self.nsub, 4 if getattr(self, "cross", False) else self.npol, self.nchan),
                       np.complex64)
        w = np.empty(self.nbl, np.float64) if weights else None
        rc = corr_correlate(self.h, _ptr(out), _ptr(w))
        if rc in (CORR_EAGAIN, CORR_EEND):
            return None
        self._check(rc)
        return out, w

    def correlate_into(self, out, weights=None) -> int:
        """Host-buffer variant that returns the code (no allocation)."""
        return corr_correlate(self.h, _ptr(out), _ptr(weights))

    def correlate_device(self, dev_out, dev_weights=None) -> int:
        rc = corr_correlate_device(self.h, _ptr(dev_out), _ptr(dev_weights))
        if rc not in (CORR_OK, CORR_EAGAIN, CORR_EEND):
            self._check(rc)
        return rc

    def device_bytes(self) -> int:
        v = C.c_size_t()
        self._check(corr_device_bytes(self.h, C.byref(v)))
        return v.value

    def next_integration(self) -> int:
        v = C.c_int64()
        self._check(corr_next_integration(self.h, C.byref(v)))
        return v.value

    # ---------------------------------------------------------------- inspection
    STAGES = ("delay", "fstage", "xstage", "finalize")

    def set_profiling(self, on: bool = True):
        self._check(corr_set_profiling(self.h, int(on)))

    def read_profile(self):
        """{stage: (total ms, launches)} since the last read."""
        ms = np.zeros(4, np.float64)
        n = np.zeros(4, np.int64)
        self._check(corr_read_profile(self.h, _ptr(ms), _ptr(n)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.STAGES)}

    def launch_shape(self):
        cb, kz = C.c_int(), C.c_int()
        self._check(corr_launch_shape(self.h, C.byref(cb), C.byref(kz)))
        return cb.value, kz.value

    def debug_delays(self, b0: int, nb: int):
        start = np.zeros((self.S, nb), np.int64)
        eps = np.zeros((self.S, nb))
        tau = np.zeros((self.S, nb))
        valid = np.zeros((self.S, nb), np.uint8)
        self._check(corr_debug_delays(self.h, b0, nb, _ptr(start), _ptr(eps), _ptr(tau), _ptr(valid)))
        return start, eps, tau, valid

    def debug_codes(self, station: int, stream: int, t0: int, count: int):
        out = np.zeros(count, np.uint8)
        self._check(corr_debug_codes(self.h, station, stream, t0, count, _ptr(out)))
        return out

    def debug_spectrum(self, station: int, stream: int, block: int):
        out = np.zeros(self.nchan, np.complex64)
        v = C.c_int()
        self._check(corr_debug_spectrum(self.h, station, stream, block, _ptr(out), C.byref(v)))
        return out, bool(v.value)


def from_scan(scan, streams=None, device_streams=None, nchan=None) -> Correlator:
    """Configure a Correlator from a synthetic scan description (stations,
    shapes, sky frequencies, delay segments, stream starts) and optionally
    push host streams or attach device streams."""
    c = Correlator(scan.stations, scan.nsub, scan.npol, nchan or scan.nchan, scan.tint, fs=scan.fs)
    for sb, nu in enumerate(scan.nu0):
        if nu:
            c.set_sky_freq(sb, nu)
    for s, segs in enumerate(scan.polys):
        for seg in segs:
            c.set_delay_poly(s, seg.t0, seg.coeffs)
        c.set_stream_start(s, scan.sample0[s])
    if streams is not None:
        for s, b in enumerate(streams):
            c.push(s, b)
    if device_streams is not None:
        for s, t in enumerate(device_streams):
            c.attach_device(s, t)
    return c


class StaticScan:
    """Descriptor for corr_correlate_static: a scan whose packed samples are
    already in device memory (one CUDA tensor per station).  Holds the host
    arrays the descriptor points to."""

    MAXSEG = 64

    def __init__(self, scan, dev_tensors, lut=(-3.336, -1.0, 1.0, 3.336)):
        S = scan.stations
        self._nu0 = np.ascontiguousarray(scan.nu0, dtype=np.float64)
        self._nseg = np.array([len(p) for p in scan.polys], dtype=np.int32)
        self._t0 = np.zeros((S, self.MAXSEG))
        self._c = np.zeros((S, self.MAXSEG, 6))
        for s, segs in enumerate(scan.polys):
            for i, g in enumerate(segs):
                self._t0[s, i] = g.t0
                self._c[s, i, :] = g.coeffs
        self._tensors = list(dev_tensors)
        self._ptrs = (C.c_void_p * S)(*[t.data_ptr() for t in dev_tensors])
        self._nb = np.array([t.numel() * t.element_size() for t in dev_tensors], dtype=np.uint64)
        self._s0 = np.asarray(scan.sample0, dtype=np.int64).copy()
        self.desc = CorrScanDesc(S, scan.nsub, scan.npol, scan.nchan, float(scan.fs), float(scan.tint),
                                 (C.c_float * 4)(*lut), _ptr(self._nu0), _ptr(self._nseg), _ptr(self._t0),
                                 _ptr(self._c), C.cast(self._ptrs, C.c_void_p), _ptr(self._nb), _ptr(self._s0))

    def correlate(self, integration: int, dev_out, dev_weights=None, stream: Optional[int] = None) -> int:
        return corr_correlate_static(C.byref(self.desc), int(integration), _ptr(dev_out), _ptr(dev_weights),
                                     stream)


def batch_run(correlators, dev_outs, dev_weights=None, stream=None) -> int:
    """Next integration of every Correlator as one CUDA graph (corr_batch_run)."""
    n = len(correlators)
    hs = (C.c_void_p * n)(*[c.h.value for c in correlators])
    outs = (C.c_void_p * n)(*[_ptr(o) for o in dev_outs])
    ws = (C.c_void_p * n)(*[_ptr(w) for w in dev_weights]) if dev_weights is not None else None
    rc = corr_batch_run(C.cast(hs, C.c_void_p), n, C.cast(outs, C.c_void_p),
                        C.cast(ws, C.c_void_p) if ws is not None else None, stream)
    if rc != CORR_OK:
        raise CorrError(rc, "corr_batch_run failed: " + corr_last_error(correlators[0].h).decode())
    return rc



def fringe_search(vis, pad_rate: int, pad_delay: int, stream: Optional[int] = None):
    """Delay-rate fringe search (corr_fringe_search) of one baseline's
    visibilities vis (a CUDA complex64 tensor [nsub][nchan]).  Returns the
    complex map (a new CUDA complex64 tensor [pad_rate][pad_delay]) and the
    peak as (rate bin, lag, amplitude, complex value)."""
    import torch
    if vis.dtype != torch.complex64 or not vis.is_cuda or vis.dim() != 2:
        raise ValueError("vis must be a CUDA complex64 tensor [nsub][nchan]")
    vis = vis.contiguous()
    nsub, nchan = vis.shape
    out = torch.empty((pad_rate, pad_delay), dtype=torch.complex64, device=vis.device)
    r, l, a = C.c_int(), C.c_int(), C.c_float()
    val = (C.c_float * 2)()
    if stream is None:
        stream = torch.cuda.current_stream(vis.device).cuda_stream
    rc = corr_fringe_search(vis.data_ptr(), int(nsub), int(nchan), int(pad_rate), int(pad_delay), out.data_ptr(),
                            C.byref(r), C.byref(l), C.byref(a), C.cast(val, C.c_void_p), stream)
    if rc != CORR_OK:
        raise CorrError(rc, "corr_fringe_search")
    return out, (r.value, l.value, a.value, complex(val[0], val[1]))


class Server:
    """The continuous-batching server of libcorr (corr_server_*): a worker
    thread admits submitted jobs by device memory and advances all admitted
    jobs one integration per CUDA graph.  ``on_result(job_id, integration,
    vis, weights, status)`` runs on that worker thread; vis (complex64
    [nbl, nsub, npol, nchan]) and weights are copies."""

    def __init__(self, hbm_cap: int, reserve: int, on_result=None):
        h = _H()
        rc = corr_server_start(C.byref(h), int(hbm_cap), int(reserve))
        if rc != CORR_OK:
            raise CorrError(rc, "corr_server_start")
        self.h = h
        self.on_result = on_result
        self._jobs = {}   # key (the callback's user pointer) -> job metadata
        self._next_key = 1

        def trampoline(user, job_id, integration, vis, weights, status):
            meta = self._jobs.get(user or 0)
            v = w = None
            if status == CORR_OK and meta is not None:
                nbl, nsub, npol, nchan = meta["shape"]
                v = np.ctypeslib.as_array(vis, shape=(nbl * nsub * npol * nchan * 2,)).view(np.complex64).reshape(
                    nbl, nsub, npol, nchan).copy()
                w = np.ctypeslib.as_array(weights, shape=(nbl,)).copy()
            if meta is not None and (status != CORR_OK or integration + 1 >= meta["nint"]):
                self._jobs.pop(user, None)
            if self.on_result is not None:
                self.on_result(job_id, integration, v, w, status)

        self._cb = RESULT_FN(trampoline)

    def submit(self, static_scan: "StaticScan", integrations: int, precision: int = CORR_PREC_FP32,
               rotation: int = CORR_ROT_POST_F) -> int:
        """Queue a job: the scan held by a StaticScan (samples in device
        memory, which must stay alive until the job's last result)."""
        job = CorrJob(static_scan.desc, int(precision), int(rotation), int(integrations))
        jid = C.c_int64()
        d = static_scan.desc
        nbl = d.stations * (d.stations + 1) // 2
        key = self._next_key
        self._next_key += 1
        # registered before the worker can report on it
        self._jobs[key] = {"shape": (nbl, d.subbands, d.pols, d.nchan), "nint": int(integrations),
                           "keep": static_scan}
        # no Python callback at all when nobody listens (results still reach
        # the server's pinned host buffers every integration)
        fn = self._cb if self.on_result is not None else RESULT_FN()  # RESULT_FN(): a NULL pointer
        rc = corr_server_submit(self.h, C.byref(job), fn, C.c_void_p(key), C.byref(jid))
        if rc != CORR_OK:
            self._jobs.pop(key, None)
            raise CorrError(rc, "corr_server_submit")
        return jid.value

    def stats(self):
        p50, p99, sps, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        corr_server_stats(self.h, C.byref(p50), C.byref(p99), C.byref(sps), C.byref(n))
        return {"p50_s": p50.value, "p99_s": p99.value, "station_samples_per_s": sps.value, "jobs_done": n.value}

    def wait(self, timeout: float = -1.0) -> int:
        return corr_server_wait(self.h, float(timeout))

    def close(self):
        if getattr(self, "h", None):
            corr_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
