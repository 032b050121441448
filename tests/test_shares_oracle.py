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


def test_undefined_cases():
    data = synth.uniform(8, 10_000)
    assert oracle.byte_shares("maxp", data, 100, 200, 4000) is None
    assert oracle.byte_shares("ae", data, 100, 200, 4000) is None  # min > w + 1
    assert oracle.byte_shares("ram", np.zeros(0, np.uint8), 100, 200, 4000) == (0, 0)
