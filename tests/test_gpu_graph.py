"""The candidate-graph chain stage (graph.cu) against the CPU oracle, bit for bit.

cdc_chunk takes the candidate graph by default for RAM, AE-Max and MAXP; these
tests force each chain stage in turn (CDC_OPT_PIPELINE) and push the graph
through its less common paths: segments as small as max (many units, exits
that jump several segments through zero runs), candidate slots far too small
for the data (every overflow path steps the chain instead), dense candidates
(low-alphabet bytes), lengths around segment multiples, misaligned pointers,
and AE-Min on the graph.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_chunk, params
from test_gpu_parity import MIB, expect_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2508_05797_gb300 import Chunker
    c = Chunker(0)
    yield c
    c.close()


def _with(ck, **opts):
    from paper_2508_05797_gb300 import cdc
    names = {"pipeline": cdc.OPT_PIPELINE, "seg": cdc.OPT_GRAPH_SEGMENT, "slots": cdc.OPT_GRAPH_SLOTS}

    class _Ctx:
        def __enter__(self):
            for k, v in opts.items():
                ck.set_option(names[k], v)

        def __exit__(self, *a):
            for k in opts:
                ck.set_option(names[k], 0)
    return _Ctx()


@pytest.mark.parametrize("pipe", [1, 2])
@pytest.mark.parametrize("alg", ["ram", "ae", "maxp"])
def test_both_pipelines_mixed_and_uniform(ck, pipe, alg):
    mixed = synth.mixed_range(1, 4 << 30, 0, 32 * MIB)
    uni = synth.uniform(0, 16 * MIB)
    with _with(ck, pipeline=pipe):
        for mean in (4096, 8192, 16384):
            w, mn, mx = params("mixed_4g_seed1", alg, mean)
            expect_equal(ck, mixed, alg, w, mn, mx, tag="pipe%d" % pipe)
        w, mn, mx = params("uniform_16m_seed0", alg, 8192)
        expect_equal(ck, uni, alg, w, mn, mx, offset=7, tag="pipe%d" % pipe)


@pytest.mark.parametrize("seg_kib", [0, 64, 128, 1024])
@pytest.mark.parametrize("slots", [0, 1, 9, 100])
def test_graph_segments_and_slots(ck, seg_kib, slots):
    """Small slots overflow on every segment: the chase and the output then
    step the chain between the candidates that have a slot."""
    data = synth.mixed_range(9, 64 * MIB, 3 * MIB, 3 * MIB + 333)
    with _with(ck, pipeline=2, seg=seg_kib << 10, slots=slots):
        for alg, w, mn, mx in (("ram", 3000, 1024, 16384), ("ae", 3000, 1024, 16384),
                               ("maxp", 120, 1024, 16384), ("ram", 7101, 2048, 65536)):
            expect_equal(ck, data, alg, w, mn, mx, offset=3, tag="seg%dk/slots%d" % (seg_kib, slots))


@pytest.mark.parametrize("kind", ["ternary", "zero_runs", "ff_runs", "ramp", "text"])
def test_graph_dense_and_quiet_content(ck, kind):
    rng = np.random.default_rng(5)
    n = 3 * MIB + 17
    if kind == "ternary":
        data = rng.integers(0, 3, size=n).astype(np.uint8)
    elif kind == "zero_runs":
        data = np.zeros(n, dtype=np.uint8)
        k = 40
        data[rng.integers(0, n, size=k)] = rng.integers(1, 256, size=k)
    elif kind == "ff_runs":
        data = np.full(n, 255, dtype=np.uint8)
        k = 40
        data[rng.integers(0, n, size=k)] = rng.integers(0, 255, size=k)
    elif kind == "ramp":
        data = (np.arange(n) % 251).astype(np.uint8)
    else:
        data = synth.mixed_range(1, 4 << 30, 6 * MIB, n)  # a text-like block
    with _with(ck, pipeline=2, seg=128 << 10):
        for alg, w, mn, mx in (("ram", 700, 256, 8192), ("ae", 700, 256, 8192), ("ae_min", 700, 256, 8192),
                               ("maxp", 150, 256, 8192), ("ram", 7000, 2048, 65536), ("maxp", 64, 1, 100000)):
            expect_equal(ck, data, alg, w, mn, mx, offset=5, tag="graph/" + kind)


def test_graph_many_units_and_long_jumps(ck):
    """1024 segments in 32 units; zero runs of up to 4 MiB make exits that
    skip whole segments and units."""
    rng = np.random.default_rng(8)
    parts = []
    for i in range(24):
        parts.append(synth.uniform(100 + i, int(rng.integers(1, 3 * MIB))))
        z = np.zeros(int(rng.integers(64 << 10, 4 * MIB)), dtype=np.uint8)
        z[rng.integers(0, z.size, size=3)] = rng.integers(1, 256, size=3)
        parts.append(z)
    data = np.concatenate(parts)[:64 * MIB]
    with _with(ck, pipeline=2, seg=64 << 10):
        for alg in ("ram", "ae", "maxp"):
            w, mn, mx = params("mixed_4g_seed1", alg, 8192)
            expect_equal(ck, data, alg, w, mn, mx, offset=1, tag="units")


def test_graph_ragged_lengths(ck):
    rng = np.random.default_rng(12)
    S = 64 << 10
    base = synth.mixed_range(3, 64 * MIB, 1 * MIB, 5 * S + 4096)
    lens = [1, 2, 63, 64, 65, 700, 7102, 8193, S - 1, S, S + 1, 2 * S - 7, 3 * S + 1, 5 * S + 4095]
    with _with(ck, pipeline=2, seg=S):
        for n in lens:
            d = np.ascontiguousarray(base[:n])
            for alg, w, mn, mx in (("ram", 7101, 2048, 65536), ("ae", 700, 128, 8192), ("maxp", 291, 2048, 65536)):
                expect_equal(ck, d, alg, w, mn, mx, offset=int(rng.integers(0, 64)), tag="len%d" % n)


def test_graph_equals_speculation_on_random_params(ck):
    """Random (w, min, max) within the graph's range, both stages, same bytes."""
    rng = np.random.default_rng(21)
    data = synth.mixed_range(4, 64 * MIB, 7 * MIB, 2 * MIB + 999)
    for t in range(24):
        alg = ("ram", "ae", "maxp")[t % 3]
        w = int(rng.integers(64, 5000)) if alg != "maxp" else int(rng.integers(63, 600))
        mn = int(rng.integers(1, w + 2)) if alg != "maxp" else int(rng.integers(1, 4000))
        mx = int(rng.integers(max(w + 1, mn) + 1, 80_000))
        exp = oracle.chunk(alg, data, w, mn, mx)
        for pipe in (1, 2):
            with _with(ck, pipeline=pipe):
                got = gpu_chunk(ck, data, alg, w, mn, mx, offset=t % 64)
            assert np.array_equal(got, exp), (alg, w, mn, mx, pipe)


def test_last_stage_reports_the_chain_stage(ck):
    """cdc_last_stage names the chain stage a call took: forced either way,
    and the automatic choice (the graph for a 4 MiB RAM call; speculation for
    AE-Min, which takes the graph only when forced)."""
    data = synth.uniform(1, 4 * MIB)
    for pipe, stage in ((1, 1), (2, 2), (0, 2)):
        with _with(ck, pipeline=pipe):
            gpu_chunk(ck, data, "ram", 700, 128, 8192)
            assert ck.last_stage() == stage, (pipe, ck.last_stage())
    gpu_chunk(ck, data, "ae_min", 700, 128, 8192)
    assert ck.last_stage() == 1


@pytest.mark.parametrize("alg", ["ram", "ae", "maxp"])
def test_capture_after_reserve_without_a_warm_up_call(alg):
    """cdc_reserve sizes the candidate graph's workspace too, so a fresh
    handle's first cdc_chunk_async can be captured into a CUDA graph; the
    replays equal the oracle."""
    import torch
    from paper_2508_05797_gb300 import Chunker
    data = synth.mixed_range(2, 64 * MIB, 3 * MIB, 6 * MIB + 77)
    w, mn, mx = params("mixed_4g_seed1", alg, 8192)
    exp = oracle.chunk(alg, data, w, mn, mx)
    ck = Chunker(0)
    try:
        d = torch.from_numpy(data).cuda()
        ck.reserve(alg, w, mn, mx, d.numel())
        out = torch.full((d.numel() // mn + 2,), -1, dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ck.chunk_async(d, alg, w, mn, mx, out, cnt, stream=s)
        for _ in range(2):
            out.fill_(-1)
            with torch.cuda.stream(s):
                g.replay()
            s.synchronize()
            ck.sync_status(s)
            n = int(cnt.item())
            assert n == exp.size and np.array_equal(out[:n].cpu().numpy().astype(np.uint64), exp), alg
        assert ck.last_stage() == 2
    finally:
        ck.close()
