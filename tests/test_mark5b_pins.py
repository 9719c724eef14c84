"""Pins of the oracle's Mark5B-style framed input (NEXT-4 reading).

The paper's data path converts RadioAstron's RDF recordings to Mark5B
(Sec. 2).  Read here: a station's bytes are frames of a 16-byte header and
P payload bytes, the payloads in order form the packed sample stream, and a
frame whose first header word is not the sync word 0xABADDEED (a lost or
filled frame) invalidates every block that reads a sample from it.  Fixed by
the data themselves:
* framing with valid headers is transparent: the same samples framed or
  plain give identical visibilities and weights;
* an invalid frame's payload never matters: garbage or the true samples
  there give identical results;
* the weights drop by exactly the blocks whose windows touch that frame,
  counted from the windows' byte ranges.
"""
import numpy as np
import pytest

import oracle
import synth

P = 400   # payload bytes per frame in these tests (10000 in Mark5B proper)


def scan(seed=6, S=3, nsub=2, npol=1, nchan=64, nblk_int=20, nint=3):
    fs = 32e6
    N = 2 * nchan
    tint = nblk_int * N / fs
    polys = [[synth.Segment(0.0, ((3.3 + 17.6 * s) / fs, 1e-6 * s, 0, 0, 0, 0))] for s in range(S)]
    T = nint * nblk_int * N + 160
    G = nsub * npol
    plain = [synth.random_bytes(seed, s, T * G // 4) for s in range(S)]
    args = (S, nsub, npol, nchan, fs, tint, [1e9, 2e9][:nsub], polys)
    return args, plain, T, nint


def test_valid_frames_are_transparent():
    args, plain, T, nint = scan()
    S = args[0]
    ref, wref = oracle.Oracle(*args, plain, [0] * S, [T] * S).correlate(0, nint)
    framed = [synth.frame(b, P) for b in plain]
    got, w = oracle.Oracle(*args, framed, [0] * S, [T] * S, frame_payload=P).correlate(0, nint)
    assert np.array_equal(w, wref) and np.array_equal(got, ref)


def test_invalid_frame_payload_never_matters_and_drops_exactly_its_blocks():
    args, plain, T, nint = scan(seed=7)
    S, nsub, npol, nchan = args[0], args[1], args[2], args[3]
    G, N = nsub * npol, 2 * nchan
    bad_station, bad = 1, 5          # frame 5 of station 1 is lost
    framed = [synth.frame(b, P, invalid=(bad,) if s == bad_station else ()) for s, b in enumerate(plain)]
    garbage = [f.copy() for f in framed]
    off = bad * (16 + P) + 16
    garbage[bad_station][off:off + P] = np.random.default_rng(1).integers(0, 256, P, dtype=np.uint8)
    o1 = oracle.Oracle(*args, framed, [0] * S, [T] * S, frame_payload=P)
    o2 = oracle.Oracle(*args, garbage, [0] * S, [T] * S, frame_payload=P)
    v1, w1 = o1.correlate(0, nint)
    v2, w2 = o2.correlate(0, nint)
    assert np.array_equal(w1, w2) and np.array_equal(v1, v2)
    # weights: the plain scan's minus the blocks whose windows read frame `bad`
    vref, wref = oracle.Oracle(*args, plain, [0] * S, [T] * S).correlate(0, nint)
    nb = int(round(args[5] * args[4])) // N * nint
    n_b = o1.delays(0, nb)[0]
    lo, hi = bad * P, (bad + 1) * P          # payload bytes of the lost frame
    touched = [b for b in range(nb)
               if (2 * (b * N + n_b[bad_station, b]) * G) // 8 < hi
               and (2 * ((b * N + n_b[bad_station, b] + N) * G) - 1) // 8 >= lo]
    assert len(touched) >= 1
    nblk_int = nb // nint
    bls = [(a, c) for a in range(S) for c in range(a, S)]
    for i in range(nint):
        lost = sum(1 for b in touched if b // nblk_int == i)
        for k, (a, c) in enumerate(bls):
            expect = wref[i, k] - (lost if bad_station in (a, c) else 0)
            assert w1[i, k] == expect, (i, a, c, w1[i, k], expect)
            if bad_station not in (a, c):
                assert np.array_equal(v1[i, k], vref[i, k])


def test_window_ending_at_a_frame_boundary():
    """A station 32 samples late, G = 2 (two sample-times per byte), 128-sample
    windows and 400-byte payloads: block 30 reads payload bytes 1936..1999,
    the last 64 of frame 4, and block 31 bytes 2000..2063, the first of frame
    5.  With frame 5 lost, block 30 stays valid and block 31 does not; with
    frame 4 lost, the reverse holds for blocks 30 and 31."""
    fs, nchan, m = 32e6, 64, 32
    N = 2 * nchan
    T = 60 * N
    plain = synth.random_bytes(9, 0, T * 2 // 4)
    polys = [[synth.Segment(0.0, (m / fs, 0, 0, 0, 0, 0))]]
    for bad, want30, want31 in ((5, 1, 0), (4, 0, 1)):
        raw = synth.frame(plain, P, invalid=(bad,))
        o = oracle.Oracle(1, 1, 2, nchan, fs, 10 * N / fs, [0.0], polys, [raw], [0], [T], frame_payload=P)
        n_b, _, _, v = o.delays(0, 40)
        assert n_b[0, 30] == m
        assert (v[0, 30], v[0, 31]) == (want30, want31), bad
        assert v[0, 29] == (1 if bad == 5 else 0) and v[0, 32] == (0 if bad == 5 else 1)
