"""Resumable chunking (cdc_feed_*): a stream handed over in device pieces.

Every push must emit exactly what the oracle's piecewise chunker emits for
the same pieces (the chunks whose start s has s + H <= bytes received,
H = max, plus w for MAXP; Section 3.3), and the pushes together must give the
boundaries of the whole stream."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import params, to_device

pytestmark = pytest.mark.gpu

CASES = [
    ("ram",) + params("mixed_4g_seed1", "ram", 4096),
    ("ae",) + params("mixed_4g_seed1", "ae", 4096),
    ("ae_min",) + params("mixed_4g_seed1", "ae", 4096),
    ("maxp",) + params("mixed_4g_seed1", "maxp", 4096),
    ("maxp", 291, 64, 4096),   # min - 1 < w: targets near a start look into the kept context
    ("maxp", 20, 16, 1024),    # byte-level MAXP (w below the summary path)
    ("ram", 100, 50, 2000),
]


def _run_feed(ck, alg, w, mn, mx, data, cuts, offsets):
    import paper_2508_05797_gb300 as pkg
    f = pkg.Feed(ck, alg, w, mn, mx)
    got = []
    for i in range(len(cuts) - 1):
        piece = data[cuts[i]:cuts[i + 1]]
        d = to_device(piece, offsets[i % len(offsets)]) if piece.size else None
        got.append(f.push(d, final=(i == len(cuts) - 2)).cpu().numpy().astype(np.uint64))
    received, start = f.position()
    assert received == data.size and start == data.size
    f.close()
    return got


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-w%d-min%d-max%d" % c)
def test_feed_matches_oracle_per_push(case):
    import paper_2508_05797_gb300 as pkg
    alg, w, mn, mx = case
    ck = pkg.Chunker(0)
    rng = np.random.default_rng(100 + CASES.index(case))
    n = 6 << 20
    data = synth.mixed_range(3, 64 << 20, 0, n)
    for trial in range(3):
        k = (3, 12, 40)[trial]
        cuts = np.sort(rng.integers(0, n + 1, size=k))
        cuts = np.concatenate([cuts, cuts[:2], [cuts[0] + 1]])  # empty pieces, a one-byte piece
        cuts = [0] + sorted(min(int(c), n) for c in cuts) + [n]
        got = _run_feed(ck, alg, w, mn, mx, data, cuts, (0, 1, 7, 13))
        exp = oracle.chunk_pieces(alg, [data[cuts[i]:cuts[i + 1]] for i in range(len(cuts) - 1)], w, mn, mx)
        assert len(got) == len(exp)
        for i, (g, e) in enumerate(zip(got, exp)):
            assert np.array_equal(g, e), (alg, trial, i, g.size, e.size)
    ck.close()


def test_feed_capacity_retry_and_misuse():
    import torch
    import paper_2508_05797_gb300 as pkg
    from paper_2508_05797_gb300.cdc import CdcError, ERR_CAPACITY, ERR_INVALID
    alg, w, mn, mx = CASES[0]
    ck = pkg.Chunker(0)
    data = synth.mixed_range(4, 8 << 20, 0, 2 << 20)
    f = pkg.Feed(ck, alg, w, mn, mx)
    small = torch.empty(3, dtype=torch.int64, device="cuda")
    with pytest.raises(CdcError) as ei:
        f.push(to_device(data[: 1 << 20]), out=small)
    assert ei.value.status == ERR_CAPACITY
    assert f.position() == (1 << 20, 0)  # the piece stays staged, nothing consumed
    a = f.push(None).cpu().numpy().astype(np.uint64)
    b = f.push(to_device(data[1 << 20:], 5), final=True).cpu().numpy().astype(np.uint64)
    assert np.array_equal(np.concatenate([a, b]), oracle.chunk(alg, data, w, mn, mx))
    with pytest.raises(CdcError) as ei:
        f.push(to_device(data[:10]))
    assert ei.value.status == ERR_INVALID
    # reset: a new stream on the same feed, with pushes on two streams
    f.reset()
    assert f.position() == (0, 0)
    s2 = torch.cuda.Stream()
    a = f.push(to_device(data[: 3 << 19], 3), stream=s2).cpu().numpy().astype(np.uint64)
    b = f.push(to_device(data[3 << 19:]), final=True).cpu().numpy().astype(np.uint64)
    assert np.array_equal(np.concatenate([a, b]), oracle.chunk(alg, data, w, mn, mx))
    f.close()
    # an empty stream: one final empty push, no boundaries
    f = pkg.Feed(ck, alg, w, mn, mx)
    assert f.push(None, final=True).numel() == 0
    f.close()
    ck.close()


def test_feed_full_size_equals_one_call():
    """1 GiB of the mixed data in ragged pieces of about 64 MiB: the pushes
    concatenate to the one-call boundaries; sampled boundaries checked
    against the oracle's next() on the whole stream."""
    import torch
    import paper_2508_05797_gb300 as pkg
    n = 1 << 30
    host = synth.mixed_range(1, 4 << 30, 0, n)
    d = torch.from_numpy(host).cuda()
    ck = pkg.Chunker(0)
    rng = np.random.default_rng(11)
    for alg in ("ram", "maxp"):
        w, mn, mx = params("mixed_4g_seed1", alg, 8192)
        whole = ck.chunk(d, alg, w, mn, mx).cpu().numpy().astype(np.uint64)
        f = pkg.Feed(ck, alg, w, mn, mx)
        parts, pos = [], 0
        while pos < n:
            ln = int(min(n - pos, rng.integers(32 << 20, 96 << 20)))
            parts.append(f.push(d[pos:pos + ln], final=(pos + ln == n)).cpu().numpy().astype(np.uint64))
            pos += ln
        got = np.concatenate(parts)
        assert np.array_equal(got, whole), alg
        idx = rng.choice(got.size - 1, size=200, replace=False)
        for i in idx.tolist():
            s = int(got[i - 1]) if i else 0
            assert oracle.next_cut(alg, host, s, w, mn, mx) == int(got[i])
        f.close()
    ck.close()
