"""The oracle's piecewise chunking (a stream handed over in pieces) against
the whole stream chunked at once (CPU only).

Each chunk is one step s -> next(s) of the sequential loop (Section 3.3) and
depends only on the bytes before s + H (H = max for RAM / AE, max + w for
MAXP, Section 2.1). So emitting a chunk once s + H bytes have arrived must
give, over all pieces, exactly the boundaries of the whole stream. Planted
horizons that are too short must break that on inputs built for it.
"""
import numpy as np
import pytest

import oracle
import synth

CASES = [
    ("ram", 64, 32, 512),
    ("ae", 64, 32, 512),
    ("ae_min", 64, 32, 512),
    ("maxp", 40, 200, 1500),   # min - 1 >= w
    ("maxp", 200, 64, 1500),   # min - 1 < w: the first targets of a chunk look left of its start
    ("maxp", 7, 3, 90),
]


def _splits(rng, n, k, with_empty=True):
    cuts = np.sort(rng.integers(0, n + 1, size=k))
    if with_empty:
        cuts = np.concatenate([cuts, cuts[: k // 4]])  # repeated cuts give empty pieces
        cuts.sort()
    return [0] + cuts.tolist() + [n]


def _pieces(data, cuts):
    return [data[cuts[i]:cuts[i + 1]] for i in range(len(cuts) - 1)]


def _mixed(seed, n):
    return synth.mixed_range(seed, 4 << 20, 0, n)


@pytest.mark.parametrize("alg,w,mn,mx", CASES)
def test_pieces_concatenate_to_whole_stream(alg, w, mn, mx):
    rng = np.random.default_rng(7)
    for trial in range(6):
        data = _mixed(trial + 1, 40_000) if trial % 2 else synth.uniform(trial + 11, 40_000)
        whole = oracle.chunk(alg, data, w, mn, mx)
        for k in (1, 3, 17, 120):
            cuts = _splits(rng, data.size, k)
            got = oracle.chunk_pieces(alg, _pieces(data, cuts), w, mn, mx)
            assert np.array_equal(np.concatenate(got), whole), (alg, trial, k)
            H = oracle.get().horizon(alg, w, mx)
            start = 0
            for i, ends in enumerate(got[:-1]):
                received = cuts[i + 1]
                for e in ends.tolist():
                    assert start + H <= received and e <= received
                    start = e
                # nothing settled was held back
                assert start + H > received


def test_empty_stream_and_final_empty_piece():
    data = synth.uniform(3, 5000)
    assert [a.size for a in oracle.chunk_pieces("ram", [np.zeros(0, np.uint8)], 64, 32, 512)] == [0]
    got = oracle.chunk_pieces("ram", [data, np.zeros(0, np.uint8)], 64, 32, 512)
    assert np.array_equal(np.concatenate(got), oracle.chunk("ram", data, 64, 32, 512))
    assert got[-1].size >= 1 and int(got[-1][-1]) == data.size


def test_one_byte_pieces():
    data = _mixed(5, 3000)
    for alg, w, mn, mx in CASES:
        got = oracle.chunk_pieces(alg, [data[i:i + 1] for i in range(data.size)], w, mn, mx)
        assert np.array_equal(np.concatenate(got), oracle.chunk(alg, data, w, mn, mx)), alg


def test_short_horizon_is_caught_ram():
    # bytes falling by one per position: the window maximum is its first byte
    # and nothing reaches it again within max (unless the window holds the
    # wrap from 0 to 255), so most chunks are forced cuts at s + max, which a
    # piece ending one byte short would truncate
    w, mn, mx = 8, 8, 100
    data = (255 - (np.arange(5000) % 256)).astype(np.uint8)
    whole = oracle.chunk("ram", data, w, mn, mx)
    assert (np.diff(whole[:-1].astype(np.int64)) == mx).sum() > 20
    rng = np.random.default_rng(1)
    caught = False
    for _ in range(20):
        cuts = _splits(rng, data.size, 40)
        bad = oracle.chunk_pieces("ram", _pieces(data, cuts), w, mn, mx, horizon=mx - 1)
        caught |= not np.array_equal(np.concatenate(bad), whole)
    assert caught


def test_short_horizon_is_caught_maxp():
    # the MAXP horizon without the right window: a target within w of the
    # bytes received is not yet a target (w large against max, so that many
    # chunks find their first target late)
    w, mn, mx = 200, 64, 600
    data = synth.uniform(9, 60_000)
    whole = oracle.chunk("maxp", data, w, mn, mx)
    rng = np.random.default_rng(2)
    caught = False
    for _ in range(20):
        cuts = _splits(rng, data.size, 200)
        bad = oracle.chunk_pieces("maxp", _pieces(data, cuts), w, mn, mx, horizon=mx)
        caught |= not np.array_equal(np.concatenate(bad), whole)
    assert caught
