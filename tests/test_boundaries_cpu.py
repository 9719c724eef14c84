"""The oracle is test infrastructure and independent of the CUDA path.

- The product package never imports, loads or names the oracle; only tests,
  __graft_entry__.smoke() and bench.py's CPU legs may.
- The two sides share no code: the oracle's C file includes only system
  headers, and the library's sources include only their own headers.
- The seeded input module holds no correlator arithmetic (no FFT, no
  cross-multiplication): it imports neither side.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1502_06894_gb300")


def sources(top, exts):
    for d, _, files in os.walk(top):
        if "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_uses_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b)|liboracle|fx_oracle", re.M)
    for p in sources(PKG, (".py", ".cu", ".cuh", ".h")):
        assert not pat.search(open(p).read()), p
    for p in sources(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in open(p).read().lower(), p


def test_oracle_includes_only_system_headers():
    src = open(os.path.join(ROOT, "oracle", "fx_oracle.c")).read()
    for inc in re.findall(r'#include\s+([<"][^>"]+[>"])', src):
        assert inc.startswith("<"), inc


def test_library_includes_only_its_own_headers():
    allowed = {'"corr_internal.cuh"', '"k_fstage_impl.cuh"', '"../../include/corr.h"'}
    for p in sources(os.path.join(PKG, "csrc"), (".cu", ".cuh")):
        for inc in re.findall(r'#include\s+("[^"]+")', open(p).read()):
            assert inc in allowed, (p, inc)


def test_input_generator_imports_neither_side():
    src = open(os.path.join(ROOT, "synth", "__init__.py")).read()
    assert not re.search(r"^\s*(import|from)\s+(oracle|paper_1502_06894_gb300)\b", src, re.M)
