"""The oracle's byte shares of the two processing patterns (Section 3.3's
composition of RAM and AE from Extreme Byte Searches and Range Scans), pinned
by identities, an independent restatement and a closed form (CPU only)."""
import numpy as np
import pytest

import oracle
import synth


def _chunks(alg, data, w, mn, mx):
    b = oracle.chunk(alg, data, w, mn, mx).astype(np.int64)
    return np.concatenate([[0], b[:-1]]), b


def test_ram_reads_every_byte_once():
    # with min <= w + 1 the window search covers [s, s + w) and the scan
    # [s + w, e): together every byte of the chunk, once
    for data in (synth.uniform(1, 300_000), synth.mixed_range(2, 8 << 20, 0, 300_000)):
        for w, mn, mx in ((700, 256, 8192), (64, 65, 1000), (3000, 1024, 16384)):
            ebs, rs = oracle.byte_shares("ram", data, w, mn, mx)
            assert ebs + rs == data.size
            s, e = _chunks("ram", data, w, mn, mx)
            tail = (data.size - s) <= w
            assert ebs == w * int((~tail).sum()) + int((e - s)[tail].sum())


def test_ram_skipping_below_min():
    # min - 1 > w: bytes [s + w, s + min - 1) are read by neither pattern
    data = synth.uniform(3, 200_000)
    w, mn, mx = 100, 2000, 16384
    ebs, rs = oracle.byte_shares("ram", data, w, mn, mx)
    s, e = _chunks("ram", data, w, mn, mx)
    full = (data.size - s) > w
    skipped = np.minimum(e - s, mn - 1) - w
    assert ebs + rs == data.size - int(skipped[full].clip(min=0).sum())


def test_ram_scan_share_closed_form():
    # uniform bytes, w = 7936: the window maximum is 255 (probability
    # 1 - (255/256)^7936), so each scan reads a geometric number of bytes with
    # p = 1/256: mean 256, standard deviation sqrt(255) * 16
    data = synth.uniform(0, 64 << 20)
    w, mn, mx = 7936, 2048, 65536
    ebs, rs = oracle.byte_shares("ram", data, w, mn, mx)
    n = oracle.count("ram", data, w, mn, mx) - 1  # the last chunk may be short
    mean = rs / n
    assert abs(mean - 256.0) < 4 * np.sqrt(255.0) * 16 / np.sqrt(n), mean
    assert abs(ebs / (ebs + rs) - w / (w + 256.0)) < 2e-3


def _ae_by_targets(data, w, mn, mx, dir_):
    """AE shares restated from the targets of each chunk (the bytes beyond
    every earlier byte of the chunk), not from the search / scan loop."""
    s_all, e_all = _chunks("ae" if dir_ > 0 else "ae_min", data, w, mn, mx)
    x = data.astype(np.int64) if dir_ > 0 else 255 - data.astype(np.int64)
    ebs = rs = 0
    for s, e in zip(s_all.tolist(), e_all.tolist()):
        seg = x[s:e]
        before = np.concatenate([[-1], np.maximum.accumulate(seg)[:-1]])
        tp = np.nonzero(seg > before)[0] + s
        ebs += int(np.minimum(w, e - 1 - tp).sum())
        rs += int(tp[-1] - s)
    return ebs, rs


@pytest.mark.parametrize("w,mn,mx", [(64, 32, 512), (300, 200, 4000), (7, 8, 90), (1000, 1001, 30000)])
def test_ae_matches_target_restatement(w, mn, mx):
    for data in (synth.uniform(5, 60_000), synth.mixed_range(6, 8 << 20, 1 << 20, 60_000),
                 np.arange(5000, dtype=np.uint8), (255 - np.arange(5000) % 256).astype(np.uint8)):
        assert oracle.byte_shares("ae", data, w, mn, mx) == _ae_by_targets(data, w, mn, mx, +1)
        assert oracle.byte_shares("ae_min", data, w, mn, mx) == _ae_by_targets(data, w, mn, mx, -1)


def test_ae_min_is_ae_max_of_complement():
    data = synth.mixed_range(7, 8 << 20, 0, 200_000)
    assert oracle.byte_shares("ae_min", data, 500, 300, 8000) == oracle.byte_shares("ae", 255 - data, 500, 300, 8000)


def _left_max(x, w):
    """m[c] = max x[c - w .. c - 1] for c >= w (numpy sliding windows)."""
    win = np.lib.stride_tricks.sliding_window_view(x, w)
    m = np.full(x.size, -1, dtype=np.int64)
    m[w:] = win.max(axis=1)[:x.size - w]
    return m


def _maxp_scan_and_stops(data, w, mn, mx):
    """From the oracle's chunks alone: the bytes the MAXP Range Scans must read
    (every position that may end the chunk, from p0 = max(s + min - 1, w) up to
    its cut, never past len - w where the right window leaves the data) and the
    bytes that beat their whole left window there (each stops a scan and costs
    one right-window search)."""
    n = data.size
    x = data.astype(np.int64)
    rec = x > _left_max(x, w)
    s_all, e_all = _chunks("maxp", data, w, mn, mx)
    rs = stops = searched = 0
    for s, e in zip(s_all.tolist(), e_all.tolist()):
        p0 = max(s + mn - 1, w)
        hi = min(e, n - w) if n > w else 0
        if p0 < hi:
            rs += hi - p0
            stops += int(rec[p0:hi].sum())
            searched += 1
    return rs, stops, searched


@pytest.mark.parametrize("w,mn,mx", [(63, 1, 2000), (150, 512, 8192), (291, 2048, 65536), (7, 40, 300),
                                     (1000, 1, 5000)])
def test_maxp_scan_bytes_and_stops(w, mn, mx):
    # Section 3.3: MAXP runs GT Range Scans, each followed by the Extreme Byte
    # Searches of the two windows. Independent of how the procedure walks, its
    # scans read each position in [p0, cut) once, and exactly the positions
    # that beat their left window stop a scan and cost a right-window search;
    # the rest of EBS is whole left-window searches, at least one per chunk
    # that has a position to test
    rng = np.random.default_rng(w)
    for data in (synth.uniform(9, 150_000), synth.mixed_range(10, 8 << 20, 2 << 20, 150_000),
                 synth.mixed_range(1, 4 << 30, 6 << 20, 150_000), rng.integers(0, 3, 150_000).astype(np.uint8)):
        ebs, rs = oracle.byte_shares("maxp", data, w, mn, mx)
        rs_exp, stops, searched = _maxp_scan_and_stops(data, w, mn, mx)
        assert rs == rs_exp
        left = ebs - w * stops
        assert left % w == 0 and left // w >= searched, (ebs, stops, searched)
        # a left search is followed by a scan of at least one byte
        assert left // w <= rs


def test_maxp_constant_bytes_closed_form():
    # no byte beats an equal neighbour: every chunk is forced; from p0 each left
    # search ends at the last byte before p, so a scan reads w positions
    n, w, mn, mx = 50_000, 100, 300, 4000
    data = np.full(n, 7, dtype=np.uint8)
    ebs = rs = 0
    for s in range(0, n, mx):
        p0, hi = max(s + mn - 1, w), min(s + mx, n - w)
        if p0 < hi:
            rs += hi - p0
            ebs += w * -(-(hi - p0) // w)
    assert oracle.byte_shares("maxp", data, w, mn, mx) == (ebs, rs)


def test_maxp_ramp_closed_form():
    # a strictly increasing ramp: each position beats its left window (the scan
    # stops at once) and loses to its right one, so it costs one byte of scan
    # and two w-byte searches
    w = 10
    data = np.arange(200, dtype=np.uint8)
    p0, hi = w, 200 - w
    assert oracle.byte_shares("maxp", data, w, 1, 10_000) == (2 * w * (hi - p0), hi - p0)


@pytest.mark.parametrize("t", [35, 40, 57, 1000])
def test_maxp_single_spike_closed_form(t):
    # zeros with one non-zero byte at t: the first chunk's left searches step w
    # bytes at a time from w until the scan containing t stops there, t is the
    # only target; the second chunk starts at t + 1 with t in its first left
    # window, then steps w bytes at a time again up to len - w
    n, w = 3000, 10
    data = np.zeros(n, dtype=np.uint8)
    data[t] = 200
    cend = n - w
    ebs = w * ((t - w) // w + 1) + w + w * -(-(cend - t - 1) // w)
    rs = (t - w + 1) + (cend - t - 1)
    assert oracle.chunk("maxp", data, w, 1, 100_000).tolist() == [t + 1, n]
    assert oracle.byte_shares("maxp", data, w, 1, 100_000) == (ebs, rs)


def test_undefined_cases():
    data = synth.uniform(8, 10_000)
    assert oracle.byte_shares("ae", data, 100, 200, 4000) is None  # min > w + 1
    assert oracle.byte_shares("ram", np.zeros(0, np.uint8), 100, 200, 4000) == (0, 0)
