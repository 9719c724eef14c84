"""The delay-rate fringe search on the GPU (corr_fringe_search, the paper's
wide-window fringe search, Sec. 2) against the FP64 oracle.

The map is FP32 arithmetic throughout (FFTs of up to 2^13 x 2^7 points with
twiddles from sincospif): relative RMS over the map <= 1e-5, the bar of the
FP32 path.  The peak index is an argmax taken in FP32 on the GPU and in FP64
in the oracle: the GPU's peak must be a maximum of the oracle's map to
within that tolerance, and equal to the oracle's peak wherever the runner-up
is further than 1e-4 below it."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def corr():
    from paper_1502_06894_gb300 import _build
    _build.build()
    from paper_1502_06894_gb300 import corr as c
    return c


def to_gpu(V):
    import torch
    return torch.from_numpy(np.ascontiguousarray(V.astype(np.complex64))).cuda()


def check_peak(amp_ref, peak):
    r, l, a, _ = peak
    top = amp_ref.max()
    assert amp_ref[r, l] >= top * (1 - TOL), (r, l, amp_ref[r, l], top)
    assert a == pytest.approx(top, rel=TOL)
    second = np.partition(amp_ref.ravel(), -2)[-2]
    if second < top * (1 - 1e-4):
        assert (r, l) == oracle.fringe_peak(amp_ref)[:2]


@pytest.mark.parametrize("nsub,nchan,Nr,Nd", [(16, 256, 64, 4096), (5, 37, 8, 64), (64, 1024, 128, 8192),
                                               (1, 4, 2, 4), (33, 129, 64, 256)])
def test_map_matches_oracle(corr, nsub, nchan, Nr, Nd):
    rng = np.random.default_rng(nsub * 1000 + nchan)
    V = rng.normal(size=(nsub, nchan)) + 1j * rng.normal(size=(nsub, nchan))
    M, peak = corr.fringe_search(to_gpu(V), Nr, Nd)
    ref = oracle.fringe_map(V.astype(np.complex64).astype(np.complex128), Nr, Nd)
    got = M.cpu().numpy().astype(np.complex128)
    err = np.sqrt(np.sum(np.abs(got - ref) ** 2) / np.sum(np.abs(ref) ** 2))
    assert err < TOL, err
    check_peak(np.abs(ref), peak)
    r, l, _, val = peak
    assert abs(val - ref[r, l]) <= TOL * abs(ref).max() * 4


def test_tone_peaks_at_its_bins(corr):
    """A tone at rate bin 7 and lag -5 sums coherently to A T K."""
    T, K, Nr, Nd, A, r0, l0 = 24, 300, 32, 1024, 0.5, 7, 1024 - 5
    t = np.arange(T)[:, None]
    k = np.arange(K)[None, :]
    V = A * np.exp(-2j * np.pi * (k * l0 / Nd + t * r0 / Nr))
    _, (r, l, a, val) = corr.fringe_search(to_gpu(V), Nr, Nd)
    assert (r, l) == (r0, l0)
    assert a == pytest.approx(A * T * K, rel=TOL)
    assert abs(np.angle(val)) < 1e-4


def test_residual_delay_of_config1_on_the_gpu(corr, cfg1):
    """End to end on the GPU: config 1 correlated (FP32) with a delay model
    3.7 samples short of the injected one and the right rate, 16
    sub-integrations of 1/256 s; the fringe search of the space-ground
    baseline peaks at a lag of 3.7 samples (0.25-sample bins) and rate 0."""
    import torch
    sc, streams, _ = cfg1
    shift = 3.7 / sc.fs
    polys = []
    for s, segs in enumerate(sc.polys):
        if s == 0:  # the space station carries the injected delay
            segs = [synth.Segment(g.t0, (g.coeffs[0] - shift,) + tuple(g.coeffs[1:])) for g in segs]
        polys.append(segs)
    nsi = 16
    sc2 = dataclasses.replace(sc, polys=polys, tint=1.0 / 256, duration=nsi / 256)
    c = corr.from_scan(sc2, streams)
    V = torch.empty((nsi, sc.nchan), dtype=torch.complex64, device="cuda")
    for i in range(nsi):
        r = c.correlate()
        assert r is not None
        vis, w = r
        V[i] = torch.from_numpy(np.ascontiguousarray(vis.reshape(sc.nbl, sc.G, sc.nchan)[1, 0]))
    c.close()
    Nr, Nd = 64, 8 * sc.nchan
    M, (rb, l, a, val) = corr.fringe_search(V, Nr, Nd)
    lag = (l if l < Nd // 2 else l - Nd) * sc.N / Nd
    rate = rb if rb < Nr // 2 else rb - Nr
    assert abs(abs(lag) - 3.7) <= 0.25, lag
    assert rate == 0, rate
    ref = oracle.fringe_map(V.cpu().numpy().astype(np.complex128), Nr, Nd)
    check_peak(np.abs(ref), (rb, l, a, val))


def test_rejects_bad_sizes(corr):
    V = to_gpu(np.ones((8, 16)))
    for Nr, Nd in ((4, 16), (8, 12), (8, 8), (32768, 16)):
        with pytest.raises(corr.CorrError) as ei:
            corr.fringe_search(V, Nr, Nd)
        assert ei.value.code == corr.CORR_EINVAL
