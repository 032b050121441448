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
