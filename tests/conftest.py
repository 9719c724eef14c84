import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


_cache = {}


def cached(key, fn):
    if key not in _cache:
        _cache[key] = fn()
    return _cache[key]


@pytest.fixture(scope="session")
def cfg1():
    """Config-1 scan (2 stations, 1 s, 256 channels, rho 0.02, sky frequency
    10 MHz so that fringe rotation is exercised), its packed
    station streams and the oracle holding them."""
    import synth
    import oracle

    def make():
        sc = synth.config1(nu0=1e7)
        streams = [synth.station_bytes(sc, s) for s in range(sc.stations)]
        return sc, streams, oracle.Oracle.from_scan(sc, streams)

    return cached("cfg1", make)
