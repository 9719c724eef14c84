"""The C-ABI library builds, loads and exports every entry point that
include/corr.h declares (no device work: these run without a GPU)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "corr.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|void|const char \*)\s*\*?(corr_\w+)\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_06894_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("corr_create", "corr_set_delay_poly", "corr_push_samples", "corr_correlate",
              "corr_set_format", "corr_set_sky_freq", "corr_flush", "corr_last_error", "corr_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(corr_\w+)$", out, re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_1502_06894_gb300 import corr
    assert sorted(corr.EXPORTED) == declared()


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "corr.h"\nint main(void){corr_t *h = 0; (void)h; return CORR_OK;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                    "-o", str(tmp_path / "t.o")], check=True)


def test_null_handle_calls_fail_cleanly(lib):
    L = C.CDLL(lib)
    L.corr_flush.argtypes = [C.c_void_p]
    L.corr_rewind.argtypes = [C.c_void_p]
    L.corr_last_error.argtypes = [C.c_void_p]
    L.corr_last_error.restype = C.c_char_p
    L.corr_destroy.argtypes = [C.c_void_p]
    assert L.corr_flush(None) == -1
    assert L.corr_rewind(None) == -1
    L.corr_destroy(None)
    L.corr_create.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
    h = C.c_void_p()
    # argument checks come before any device work
    assert L.corr_create(C.byref(h), 0, 1, 1, 256, 1.0) == -1
    assert b"stations" in L.corr_last_error(None)
    assert L.corr_create(C.byref(h), 2, 1, 1, 100, 1.0) == -1
    assert L.corr_create(C.byref(h), 2, 20, 2, 256, 1.0) == -1
    assert L.corr_create(C.byref(h), 2, 1, 3, 256, 1.0) == -1
    assert L.corr_create(C.byref(h), 2, 1, 1, 256, -1.0) == -1
    assert not h.value


def test_fringe_search_checks_arguments_before_any_device_work(lib):
    """corr_fringe_search rejects missing buffers and pads that are not powers
    of two, below the data, above 16384 or too large together with
    CORR_EINVAL, before it touches the device (so this runs without a GPU)."""
    L = C.CDLL(lib)
    L.corr_fringe_search.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    dummy = C.c_void_p(16)  # never dereferenced: the checks fail first
    assert L.corr_fringe_search(None, 4, 8, 4, 8, dummy, None, None, None, None, None) == -1
    assert L.corr_fringe_search(dummy, 4, 8, 4, 8, None, None, None, None, None, None) == -1
    assert L.corr_fringe_search(dummy, 0, 8, 4, 8, dummy, None, None, None, None, None) == -1
    for nr, nd in ((3, 8), (4, 12), (2, 8), (4, 4), (32768, 8), (8192, 16384)):
        assert L.corr_fringe_search(dummy, 4, 8, nr, nd, dummy, None, None, None, None, None) == -1, (nr, nd)

