"""Batched chunking (many files, one launch) against the oracle per file."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_05797_gb300 import Chunker
    c = Chunker(0)
    yield c
    c.close()


def _files(seed, n_files, median, sigma, hi, empty_every=0):
    sizes = synth.lognormal_sizes(seed, n_files, median, sigma, 1, hi).astype(np.int64)
    if empty_every:
        sizes[::empty_every] = 0
        sizes[:3] = 0
        sizes[-2:] = 0
    off = np.zeros(n_files + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    arena = synth.mixed_range(seed, max(int(off[-1]), 1), 0, int(off[-1]))
    return arena, off


def _run(ck, arena, off, alg, w, mn, mx, base_offset=0):
    import torch
    t = torch.empty(arena.size + base_offset + 64, dtype=torch.uint8, device="cuda")
    a = t[base_offset:base_offset + arena.size]
    if arena.size:
        a.copy_(torch.from_numpy(arena))
    d_off = torch.from_numpy(off).cuda()
    b, idx = ck.chunk_batch(a, d_off, alg, w, mn, mx)
    return b.cpu().numpy().astype(np.uint64), idx.cpu().numpy()


@pytest.mark.parametrize("alg", ["ram", "ae", "maxp", "ae_min"])
def test_batch_matches_per_file_oracle(ck, alg):
    arena, off = _files(3, 3000, 16 * 1024, 1.5, 4 << 20, empty_every=97)
    w, mn, mx = params("mixed_4g_seed1", "ae" if alg == "ae_min" else alg, 4096)
    b, idx = _run(ck, arena, off, alg, w, mn, mx, base_offset=13)
    assert idx[0] == 0 and idx[-1] == b.size
    for f in range(off.size - 1):
        exp = oracle.chunk(alg, arena[off[f]:off[f + 1]], w, mn, mx)
        got = b[idx[f]:idx[f + 1]]
        assert np.array_equal(got, exp), (alg, f, off[f], off[f + 1])


def test_batch_small_segments_and_windows(ck):
    from paper_2508_05797_gb300.cdc import OPT_SEGMENT
    arena, off = _files(8, 400, 3000, 1.2, 1 << 20, empty_every=11)
    try:
        for seg in (64, 512, 0):
            ck.set_option(OPT_SEGMENT, seg)
            for alg, w, mn, mx in (("ram", 300, 64, 4000), ("ae", 5, 2, 300), ("maxp", 90, 64, 4000),
                                   ("maxp", 3, 1, 100)):
                b, idx = _run(ck, arena, off, alg, w, mn, mx)
                for f in range(off.size - 1):
                    exp = oracle.chunk(alg, arena[off[f]:off[f + 1]], w, mn, mx)
                    assert np.array_equal(b[idx[f]:idx[f + 1]], exp), (seg, alg, f)
    finally:
        ck.set_option(OPT_SEGMENT, 0)


def test_batch_equals_per_file_calls(ck):
    import torch
    arena, off = _files(5, 300, 30_000, 1.5, 8 << 20)
    w, mn, mx = params("mixed_4g_seed1", "ram", 8192)
    b, idx = _run(ck, arena, off, "ram", w, mn, mx)
    t = torch.from_numpy(arena).cuda()
    for f in range(off.size - 1):
        if off[f + 1] == off[f]:
            continue
        one = ck.chunk(t[off[f]:off[f + 1]], "ram", w, mn, mx).cpu().numpy().astype(np.uint64)
        assert np.array_equal(one, b[idx[f]:idx[f + 1]])


def test_batch_all_empty_files(ck):
    import torch
    off = np.zeros(6, dtype=np.int64)
    a = torch.zeros(16, dtype=torch.uint8, device="cuda")
    b, idx = ck.chunk_batch(a, torch.from_numpy(off).cuda(), "ram", 10, 1, 100)
    assert b.numel() == 0 and idx.cpu().numpy().tolist() == [0] * 6


def test_autotune_keeps_results(ck):
    """The autotuner only picks segment size and warp-chain threshold: the
    boundaries after tuning equal those before (stream and batch forms)."""
    import torch
    from paper_2508_05797_gb300 import Chunker
    from paper_2508_05797_gb300.cdc import OPT_SEGMENT, OPT_WARP_CHAINS
    c = Chunker(0)
    try:
        data = torch.from_numpy(synth.mixed_range(1, 4 << 30, 7 << 20, 24 << 20)).cuda()
        for alg in ("ram", "ae", "maxp"):
            w, mn, mx = params("mixed_4g_seed1", alg, 8192)
            before = c.chunk(data, alg, w, mn, mx).clone()
            seg, wc, ms = c.autotune(data, alg, w, mn, mx)
            assert ms > 0 and c.get_option(OPT_SEGMENT) == seg and c.get_option(OPT_WARP_CHAINS) == wc
            assert torch.equal(c.chunk(data, alg, w, mn, mx), before)
        arena, off = _files(9, 500, 40_000, 1.5, 4 << 20)
        w, mn, mx = params("mixed_4g_seed1", "maxp", 8192)
        b0, i0 = _run(c, arena, off, "maxp", w, mn, mx)
        a = torch.from_numpy(arena).cuda()
        d_off = torch.from_numpy(off).cuda()
        c.autotune(a, "maxp", w, mn, mx, file_off=d_off)
        b1, i1 = _run(c, arena, off, "maxp", w, mn, mx)
        assert np.array_equal(b0, b1) and np.array_equal(i0, i1)
    finally:
        c.close()


def test_batch_graph_replay_matches(ck):
    """The batched call captured in a CUDA graph (workspace reserved first)
    and replayed gives the direct call's boundaries."""
    import torch
    from paper_2508_05797_gb300 import Chunker
    arena, off = _files(11, 2000, 20_000, 1.5, 2 << 20)
    w, mn, mx = params("mixed_4g_seed1", "ram", 8192)
    expect, eidx = _run(ck, arena, off, "ram", w, mn, mx)
    c = Chunker(0)
    try:
        a = torch.from_numpy(arena).cuda()
        d_off = torch.from_numpy(off).cuda()
        n_files = off.size - 1
        c.reserve("ram", w, mn, mx, arena.size, n_files)
        out = torch.full((arena.size // mn + n_files + 1,), -1, dtype=torch.int64, device="cuda")
        idx = torch.empty(n_files + 1, dtype=torch.int64, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            c.chunk_batch(a, d_off, "ram", w, mn, mx, out=out, index=idx, stream=s, sync=False)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            c.chunk_batch(a, d_off, "ram", w, mn, mx, out=out, index=idx, stream=s, sync=False)
        for _ in range(2):
            out.fill_(-1)
            g.replay()
            torch.cuda.synchronize()
            c.sync_status()
            i = idx.cpu().numpy()
            assert np.array_equal(i, eidx)
            assert np.array_equal(out[:int(i[-1])].cpu().numpy().astype(np.uint64), expect)
    finally:
        c.close()
