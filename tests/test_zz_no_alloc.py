"""cdc_chunk_static: the chunk path on the library's fixed scratch array.

Called through the C ABI (ctypes) and compared with cdc_chunk, the handle
entry point, on the same device buffers: twice in a row for every algorithm,
so the second call runs on scratch the first one left behind. The file is
named to be collected last, so that in a full run it follows every other GPU
test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_util import params, to_device

pytestmark = pytest.mark.gpu

ALG_IDS = {"ram": 0, "ae": 1, "maxp": 2, "ae_min": 3}
INVALID, CAPACITY = 1, 2


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_2508_05797_gb300 as pkg
    lib = pkg.load_library()
    ck = pkg.Chunker(0)
    yield torch, pkg, lib, ck
    ck.close()


def call_static(torch, pkg, lib, data, alg, w, mn, mx, out, cap=None):
    n = ctypes.c_size_t(out.numel() if cap is None else cap)
    st = lib.cdc_chunk_static(ALG_IDS[alg], pkg.Params(w, mn, mx), data.data_ptr(), data.numel(), out.data_ptr(),
                              ctypes.byref(n), torch.cuda.current_stream().cuda_stream)
    return st, n.value


CASES = [("ram", 8192), ("ae", 8192), ("maxp", 8192), ("ae_min", 8192), ("ram", 4096), ("maxp", 16384)]


@pytest.mark.parametrize("alg,mean", CASES)
def test_two_calls_in_a_row_match_cdc_chunk(env, alg, mean):
    torch, pkg, lib, ck = env
    w, mn, mx = params("mixed_4g_seed1", "ae" if alg == "ae_min" else alg, mean)
    n = pkg.STATIC_MAX_LEN - 12345
    host = synth.mixed_range(1, 4 << 30, 5 << 20, n)  # random, text and zero-run blocks
    data = to_device(host, offset=7)
    expect = ck.chunk(data, alg, w, mn, mx).clone()
    out = torch.full((pkg.max_boundaries(n, mn),), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):
        out.fill_(-1)
        st, cnt = call_static(torch, pkg, lib, data, alg, w, mn, mx, out)
        assert st == 0, pkg.cdc.STATUS[st]
        assert cnt == expect.numel()
        assert torch.equal(out[:cnt], expect)
        assert int(out[cnt:].max()) == -1  # nothing written past the count


def test_largest_input_and_the_limit(env):
    torch, pkg, lib, ck = env
    w, mn, mx = params("mixed_4g_seed1", "ram", 8192)
    n = pkg.STATIC_MAX_LEN
    data = to_device(synth.uniform(0, n))
    expect = ck.chunk(data, "ram", w, mn, mx)
    got = pkg.chunk_static(data, "ram", w, mn, mx)
    assert torch.equal(got, expect)
    # one byte more is refused before anything is enqueued
    big = torch.zeros(n + 1, dtype=torch.uint8, device="cuda")
    out = torch.empty(pkg.max_boundaries(n + 1, mn), dtype=torch.int64, device="cuda")
    st, _ = call_static(torch, pkg, lib, big, "ram", w, mn, mx, out)
    assert st == INVALID


def test_capacity_error_then_a_good_call(env):
    torch, pkg, lib, ck = env
    w, mn, mx = 1000, 256, 8000
    data = to_device(synth.uniform(3, 1 << 20), offset=3)
    expect = ck.chunk(data, "ae", w, mn, mx)
    out = torch.empty(pkg.max_boundaries(data.numel(), mn), dtype=torch.int64, device="cuda")
    st, cnt = call_static(torch, pkg, lib, data, "ae", w, mn, mx, out, cap=5)
    assert st == CAPACITY and cnt == expect.numel()
    st, cnt = call_static(torch, pkg, lib, data, "ae", w, mn, mx, out)
    assert st == 0 and torch.equal(out[:cnt], expect)


def test_small_and_empty_inputs(env):
    torch, pkg, lib, ck = env
    for n in (1, 63, 64, 65, 4097, 100_003):
        host = synth.mixed_range(2, 64 << 20, 3 << 20, n)
        data = to_device(host, offset=n % 13)
        for alg in ("ram", "ae", "maxp"):
            w, mn, mx = (300, 64, 4096) if alg != "maxp" else (100, 64, 4096)
            assert torch.equal(pkg.chunk_static(data, alg, w, mn, mx), ck.chunk(data, alg, w, mn, mx)), (n, alg)
    empty = torch.empty(0, dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    n = ctypes.c_size_t(1)
    assert lib.cdc_chunk_static(0, pkg.Params(8, 4, 64), None, 0, out.data_ptr(), ctypes.byref(n), None) == 0
    assert n.value == 0


def test_no_device_memory_is_taken(env):
    torch, pkg, lib, ck = env
    w, mn, mx = params("mixed_4g_seed1", "maxp", 8192)
    data = to_device(synth.mixed_range(1, 4 << 30, 0, 8 << 20))
    out = torch.empty(pkg.max_boundaries(data.numel(), mn), dtype=torch.int64, device="cuda")
    st, _ = call_static(torch, pkg, lib, data, "maxp", w, mn, mx, out)  # warm (first-call set-up done)
    assert st == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for alg in ("ram", "ae", "maxp"):
        st, _ = call_static(torch, pkg, lib, data, alg, w, mn, mx, out)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_host_memory_is_refused(env):
    """Pointers that are not the current device's memory return INVALID
    before anything is enqueued (the output keeps its contents)."""
    torch, pkg, lib, ck = env
    w, mn, mx = 300, 64, 4096
    host_np = synth.uniform(4, 1 << 16)
    pinned = torch.from_numpy(host_np).pin_memory()
    data = to_device(host_np)
    out = torch.full((pkg.max_boundaries(data.numel(), mn),), -1, dtype=torch.int64, device="cuda")
    out_pinned = torch.full(out.shape, -1, dtype=torch.int64).pin_memory()
    out_np = np.full(out.numel(), -1, dtype=np.int64)
    stream = torch.cuda.current_stream().cuda_stream
    for src, dst in ((pinned.data_ptr(), out.data_ptr()), (host_np.ctypes.data, out.data_ptr()),
                     (data.data_ptr(), out_pinned.data_ptr()), (data.data_ptr(), out_np.ctypes.data)):
        n = ctypes.c_size_t(out.numel())
        st = lib.cdc_chunk_static(0, pkg.Params(w, mn, mx), src, host_np.size, dst, ctypes.byref(n), stream)
        assert st == INVALID
    torch.cuda.synchronize()
    assert int(out.max()) == -1 and int(out_pinned.max()) == -1 and int(out_np.max()) == -1
    # the Python wrapper refuses an output on another device than the data
    with pytest.raises(AssertionError):
        pkg.chunk_static(data, "ram", w, mn, mx, out=torch.empty(out.numel(), dtype=torch.int64))
    assert torch.equal(pkg.chunk_static(data, "ram", w, mn, mx), ck.chunk(data, "ram", w, mn, mx))
