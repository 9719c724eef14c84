"""Host-side arithmetic of bench.py's roofline report (no GPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_issue_fraction():
    import bench
    # 4 issue slots x 152 SMs x 2070 MHz = 1.2586e12 warp instructions/s
    assert bench.issue_frac(1.2586e9, 1e-3, 2070.0) == pytest.approx(1.0, rel=1e-4)
    assert bench.issue_frac(329837046, 0.367e-3, 2070.0) == pytest.approx(0.714, abs=1e-3)
    assert bench.issue_frac(None, 1e-3, 2070.0) is None
    assert bench.issue_frac(1e9, 0.0, 2070.0) is None


def test_committed_profile_tables_cover_the_dominant_kernel():
    import bench
    t = bench.traffic_per_launch("k_fstage<1024,16>")
    i = bench.profile_value("instructions.txt", "k_fstage<1024,16>")
    assert t and 1.0e9 < t < 1.2e9          # ~ 0.25 B packed + 4 B FP32 spectra per station-sample
    assert i and 1e8 < i < 1e9
    assert bench.profile_value("instructions.txt", "no_such_kernel") is None
