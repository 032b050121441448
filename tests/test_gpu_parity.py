"""GPU boundaries against the CPU oracle, bit for bit (integer work: exact).

Every test calls the CUDA library through its C ABI (Python ctypes binding)
on seeded synthetic inputs and compares with oracle/ on the same bytes.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_chunk, params, to_device

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture(scope="module")
def ck():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2508_05797_gb300 import Chunker
    c = Chunker(0)
    yield c
    c.close()


def expect_equal(ck, data, alg, w, mn, mx, offset=0, tag=""):
    exp = oracle.chunk(alg, data, w, mn, mx)
    got = gpu_chunk(ck, data, alg, w, mn, mx, offset)
    if not np.array_equal(got, exp):
        n = min(got.size, exp.size)
        bad = int(np.argmax(got[:n] != exp[:n])) if np.any(got[:n] != exp[:n]) else n
        raise AssertionError("%s %s w=%d min=%d max=%d off=%d len=%d: gpu %d bounds, oracle %d; first diff at %d "
                             "(gpu %s, oracle %s)" % (tag, alg, w, mn, mx, offset, data.size, got.size, exp.size,
                                                      bad, got[bad:bad + 3], exp[bad:bad + 3]))


def test_uniform_16mib_ram(ck):
    """16 MiB of uniform bytes (seed 0), RAM with the calibrated window."""
    data = synth.uniform(0, 16 * MIB)
    w, mn, mx = params("uniform_16m_seed0", "ram", 8192)
    expect_equal(ck, data, "ram", w, mn, mx)


@pytest.mark.parametrize("alg", ["ram", "ae", "maxp"])
def test_uniform_16mib_other_algorithms(ck, alg):
    data = synth.uniform(0, 16 * MIB)
    w, mn, mx = params("uniform_16m_seed0", alg, 8192)
    expect_equal(ck, data, alg, w, mn, mx)


@pytest.mark.parametrize("alg", ["ram", "ae", "maxp", "ae_min"])
@pytest.mark.parametrize("mean", [4096, 8192, 16384])
def test_mixed_stream_prefix(ck, alg, mean):
    """64 MiB prefix of the 4 GiB mixed stream (random / text / zero runs)."""
    data = synth.mixed_range(1, 4 << 30, 0, 64 * MIB)
    w, mn, mx = params("mixed_4g_seed1", "ae" if alg == "ae_min" else alg, mean)
    expect_equal(ck, data, alg, w, mn, mx)


EDGE_LENS = [1, 2, 3, 31, 63, 64, 65, 127, 128, 129, 1000, 4095, 4096, 4097, 65537, 300_001]


@pytest.mark.parametrize("offset", [0, 1, 15, 16, 33, 63])
def test_ragged_lengths_and_misaligned_pointers(ck, offset):
    rng = np.random.default_rng(offset)
    for n in EDGE_LENS:
        data = rng.integers(0, 256, size=n).astype(np.uint8)
        for alg, w, mn, mx in (("ram", 100, 16, 2000), ("ram", 3, 1, 50), ("ae", 64, 1, 900),
                               ("ae", 5, 2, 40), ("ae_min", 70, 8, 1000), ("maxp", 63, 4, 3000),
                               ("maxp", 2, 1, 30), ("maxp", 200, 100, 5000)):
            expect_equal(ck, data, alg, w, mn, mx, offset, tag="ragged")


def test_empty_input(ck):
    import torch
    t = torch.empty(0, dtype=torch.uint8, device="cuda")
    for alg in ("ram", "ae", "maxp", "ae_min"):
        assert ck.chunk(t, alg, 100, 10, 1000).numel() == 0


@pytest.mark.parametrize("kind", ["zeros", "ff", "ramp", "period", "runs", "ternary"])
def test_pathological_content(ck, kind):
    n = 3 * MIB + 17
    rng = np.random.default_rng(7)
    if kind == "zeros":
        data = np.zeros(n, dtype=np.uint8)
    elif kind == "ff":
        data = np.full(n, 255, dtype=np.uint8)
    elif kind == "ramp":
        data = (np.arange(n) % 256).astype(np.uint8)
    elif kind == "period":
        data = (np.arange(n) % 701 == 0).astype(np.uint8) * 200
    elif kind == "runs":
        data = np.repeat(rng.integers(0, 256, size=n // 5000 + 1).astype(np.uint8), 5000)[:n].copy()
    else:
        data = rng.integers(0, 3, size=n).astype(np.uint8)
    for alg, w, mn, mx in (("ram", 700, 256, 8192), ("ae", 700, 256, 8192), ("ae_min", 700, 256, 8192),
                           ("maxp", 150, 256, 8192), ("ram", 7000, 2048, 65536), ("maxp", 64, 1, 100000)):
        expect_equal(ck, data, alg, w, mn, mx, offset=5, tag=kind)


@pytest.mark.parametrize("seg", [64, 192, 1024, 4096, 65536])
def test_tiny_segments_stress_lookback(ck, seg):
    """Many segments per chunk (and the reverse): stitching, look-back and
    the walks that settle entries the tables do not cover."""
    from paper_2508_05797_gb300.cdc import OPT_PIPELINE, OPT_SEGMENT, OPT_SPAN, PIPE_SPECULATE
    data = synth.mixed_range(9, 64 * MIB, 3 * MIB, 2 * MIB + 333)
    try:
        ck.set_option(OPT_PIPELINE, PIPE_SPECULATE)
        for span in (0, 64, 10_000):
            ck.set_option(OPT_SEGMENT, seg)
            ck.set_option(OPT_SPAN, span)
            for alg, w, mn, mx in (("ram", 3000, 1024, 16384), ("ae", 3000, 1024, 16384), ("maxp", 120, 1024, 16384),
                                   ("ram", 40, 8, 300)):
                expect_equal(ck, data, alg, w, mn, mx, offset=3, tag="seg%d/span%d" % (seg, span))
    finally:
        ck.set_option(OPT_SEGMENT, 0)
        ck.set_option(OPT_SPAN, 0)
        ck.set_option(OPT_PIPELINE, 0)


@pytest.mark.parametrize("starts", [1, 3, 16, 128])
def test_speculative_start_counts(ck, starts):
    """Any number of distinct speculative starts per segment gives the
    oracle's boundaries (few starts leave most entries to the stitch and the
    resolution walks)."""
    from paper_2508_05797_gb300.cdc import OPT_PIPELINE, OPT_SEGMENT, OPT_STARTS, PIPE_SPECULATE
    data = synth.mixed_range(9, 64 * MIB, 5 * MIB, 2 * MIB + 77)
    try:
        ck.set_option(OPT_PIPELINE, PIPE_SPECULATE)
        ck.set_option(OPT_STARTS, starts)
        for seg in (0, 4096):
            ck.set_option(OPT_SEGMENT, seg)
            for alg, w, mn, mx in (("ram", 3000, 1024, 16384), ("ae", 3000, 1024, 16384), ("maxp", 120, 1024, 16384)):
                expect_equal(ck, data, alg, w, mn, mx, offset=1, tag="starts%d/seg%d" % (starts, seg))
    finally:
        ck.set_option(OPT_STARTS, 0)
        ck.set_option(OPT_SEGMENT, 0)
        ck.set_option(OPT_PIPELINE, 0)


def test_byte_rules_equal_summary_rules(ck):
    from paper_2508_05797_gb300.cdc import OPT_FORCE_BYTES
    data = synth.mixed_range(4, 64 * MIB, 5 * MIB, 1 * MIB + 77)
    cases = (("ram", 900, 256, 8192), ("ae", 900, 256, 8192), ("ae_min", 900, 256, 8192), ("maxp", 100, 256, 8192))
    ref = [gpu_chunk(ck, data, *c) for c in cases]
    try:
        ck.set_option(OPT_FORCE_BYTES, 1)
        for c, r in zip(cases, ref):
            got = gpu_chunk(ck, data, *c)
            assert np.array_equal(got, r), c
            assert np.array_equal(got, oracle.chunk(c[0], data, *c[1:])), c
    finally:
        ck.set_option(OPT_FORCE_BYTES, 0)


def test_small_windows(ck):
    rng = np.random.default_rng(11)
    data = rng.integers(0, 256, size=200_003).astype(np.uint8)
    for alg in ("ram", "ae", "ae_min", "maxp"):
        for w in (1, 2, 7, 31, 62):
            expect_equal(ck, data, alg, w, 1 + w // 2, 64 * w + 64, offset=9, tag="smallw")


def test_capacity_error_reports_needed_count(ck):
    import torch
    from paper_2508_05797_gb300.cdc import ERR_CAPACITY, CdcError, Params
    data = synth.uniform(3, 1 * MIB)
    exp = oracle.chunk("ram", data, 700, 128, 8192)
    t = to_device(data)
    out = torch.empty(10, dtype=torch.int64, device="cuda")
    cap = ctypes.c_size_t(10)
    st = ck.lib.cdc_chunk(ck.h, 0, Params(700, 128, 8192), t.data_ptr(), t.numel(), out.data_ptr(),
                          ctypes.byref(cap), torch.cuda.current_stream().cuda_stream)
    assert st == ERR_CAPACITY and cap.value == exp.size
    # the handle stays usable
    assert np.array_equal(ck.chunk(t, "ram", 700, 128, 8192).cpu().numpy().astype(np.uint64), exp)


def test_invalid_arguments(ck):
    import torch
    from paper_2508_05797_gb300.cdc import ERR_INVALID, Params
    t = to_device(np.zeros(100, dtype=np.uint8))
    out = torch.empty(200, dtype=torch.int64, device="cuda")
    bad = [(0, Params(0, 1, 10)), (0, Params(5, 0, 10)), (0, Params(5, 11, 10)), (0, Params(10, 1, 10)),
           (1, Params(10, 1, 10)), (7, Params(5, 1, 10))]
    for alg, p in bad:
        cap = ctypes.c_size_t(200)
        st = ck.lib.cdc_chunk(ck.h, alg, p, t.data_ptr(), 100, out.data_ptr(), ctypes.byref(cap), None)
        assert st == ERR_INVALID, (alg, p.w, p.min, p.max)
    cap = ctypes.c_size_t(200)
    assert ck.lib.cdc_chunk(ck.h, 0, Params(5, 1, 10), None, 100, out.data_ptr(), ctypes.byref(cap), None) == ERR_INVALID
    # MAXP allows w >= max
    assert ck.lib.cdc_chunk(ck.h, 2, Params(20, 1, 10), t.data_ptr(), 100, out.data_ptr(), ctypes.byref(cap), None) == 0


def test_timeout_is_reported_and_handle_recovers(ck):
    """A segment that never publishes (test switch) makes its successors'
    bounded waits run out; the call returns CDC_ERR_TIMEOUT instead of
    hanging, and the next call on the same handle is correct."""
    from paper_2508_05797_gb300.cdc import (ERR_TIMEOUT, OPT_DEBUG_HOLD_ITEM, OPT_PIPELINE, OPT_SEGMENT,
                                            OPT_TIMEOUT_MS, PIPE_SPECULATE, CdcError)
    data = synth.uniform(5, 1 * MIB)
    t = to_device(data)
    try:
        ck.set_option(OPT_PIPELINE, PIPE_SPECULATE)  # the speculative pipeline has the bounded waits
        ck.set_option(OPT_SEGMENT, 4096)
        ck.set_option(OPT_TIMEOUT_MS, 200)
        ck.set_option(OPT_DEBUG_HOLD_ITEM, 3)
        with pytest.raises(CdcError) as ei:
            ck.chunk(t, "ram", 700, 128, 8192)
        assert ei.value.status == ERR_TIMEOUT
    finally:
        ck.set_option(OPT_DEBUG_HOLD_ITEM, -1)
        ck.set_option(OPT_TIMEOUT_MS, 2000)
        ck.set_option(OPT_SEGMENT, 0)
        ck.set_option(OPT_PIPELINE, 0)
    exp = oracle.chunk("ram", data, 700, 128, 8192)
    assert np.array_equal(ck.chunk(t, "ram", 700, 128, 8192).cpu().numpy().astype(np.uint64), exp)


def test_async_call_and_graph_replay(ck):
    import torch
    data = synth.mixed_range(1, 4 << 30, 0, 8 * MIB)
    w, mn, mx = params("mixed_4g_seed1", "ram", 8192)
    exp = oracle.chunk("ram", data, w, mn, mx)
    t = to_device(data)
    out = torch.full((data.size // mn + 1,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ck.reserve("ram", w, mn, mx, data.size)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ck.chunk_async(t, "ram", w, mn, mx, out, cnt, stream=s)
    s.synchronize()
    ck.sync_status(s)
    assert int(cnt.item()) == exp.size
    assert np.array_equal(out[:exp.size].cpu().numpy().astype(np.uint64), exp)
    g = torch.cuda.CUDAGraph()
    out.fill_(-1)
    cnt.zero_()
    with torch.cuda.graph(g, stream=s):
        ck.chunk_async(t, "ram", w, mn, mx, out, cnt, stream=s)
    for _ in range(3):
        out.fill_(-1)
        cnt.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(cnt.item()) == exp.size
        assert np.array_equal(out[:exp.size].cpu().numpy().astype(np.uint64), exp)
    ck.sync_status(s)


def test_host_entry_point(ck):
    data = synth.mixed_range(2, 64 * MIB, 7 * MIB, 3 * MIB + 5)
    for alg in ("ram", "ae", "maxp"):
        w, mn, mx = params("mixed_4g_seed1", alg, 4096)
        got = ck.chunk_host(data, alg, w, mn, mx)
        assert np.array_equal(got, oracle.chunk(alg, data, w, mn, mx)), alg


@pytest.mark.parametrize("w", [63, 64, 127, 128, 1000, 2111, 4095, 16384])
def test_maxp_window_sizes(ck, w):
    """MAXP over the window sizes its block-summary kernel takes (63 to 16384 bytes):
    halos of 2 to 258 blocks each side, one or two rounds of the block-key pass."""
    rng = np.random.default_rng(w)
    n = 8 * MIB
    data = (synth.uniform(5, n) >> 1).astype(np.uint8)  # background below 128
    spikes = rng.integers(0, n, size=max(4, n // max(w // 2, 1)))  # about two per window
    data[spikes] = rng.integers(128, 256, size=spikes.size).astype(np.uint8)
    expect_equal(ck, data, "maxp", w, 64, max(8 * w, 65536), tag="window")


def test_maxp_maxima_at_block_edges(ck):
    """Isolated maxima on the first or the last byte of 64-byte blocks, where with
    w = 63 a window ends inside the maximum's own block, and spikes that tie with
    their neighbour (no target on either side)."""
    rng = np.random.default_rng(11)
    n = 2 * MIB
    data = np.zeros(n, dtype=np.uint8)
    pos = np.cumsum(rng.integers(60, 400, size=n // 60))
    pos = pos[pos < n - 64]
    pos = (pos & ~63) + np.where(rng.random(pos.size) < 0.5, 0, 63)
    pos = np.unique(pos)
    val = rng.integers(1, 256, size=pos.size).astype(np.uint8)
    tie = rng.random(pos.size) < 0.2
    val[1:][tie[1:]] = val[:-1][tie[1:]]
    data[pos] = val
    for w in (63, 64, 100, 191):
        expect_equal(ck, data, "maxp", w, 1, 1 << 16, tag="block-edges")
