"""GB300 FX correlator for space-VLBI (DiFX dra path): a C-ABI CUDA library
(libcorr.so, include/corr.h) and its thin ctypes binding.

    from paper_1502_06894_gb300 import corr
    c = corr.Correlator(stations, subbands, pols, nchan, tint)
"""
import os as _os

LIB_PATH = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "libcorr.so")
INCLUDE_DIR = _os.path.join(_os.path.dirname(_os.path.dirname(_os.path.abspath(__file__))), "include")


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
