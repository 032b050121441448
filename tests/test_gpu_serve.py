"""Serving engine (cdc_server_*): continuous batching of requests from host
memory under a device-memory budget. Every result equals the request chunked
alone (cdc_chunk on a device copy of its bytes) and the oracle's boundaries,
with request bytes in pageable memory (one copy per request) and in
page-locked memory at odd offsets (the gather kernel)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import params

pytestmark = pytest.mark.gpu

ALGS = ("ram", "ae", "maxp")


def _requests(n, seed, pinned=False):
    sizes = synth.lognormal_sizes(seed, n, 64 * 1024, 1.5, 4096, 8 << 20).astype(np.int64)
    algs = synth.choice(seed + 1, n, 3)
    total = int(sizes.sum())
    pool = synth.mixed_range(seed, 4 << 30, 9 << 20, total + n)
    if pinned:
        import torch
        t = torch.empty(pool.size, dtype=torch.uint8, pin_memory=True)
        t.numpy()[:] = pool
        pool = t.numpy()  # page-locked; requests start at odd offsets below
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(sizes + 1, out=off[1:])  # a one-byte gap: sources at every alignment
    return [(ALGS[int(algs[i])], pool[off[i]:off[i] + sizes[i]]) for i in range(n)]


def _serve(reqs, gap_ms, slots=3, budget=2 << 30, seed=7):
    from paper_2508_05797_gb300 import Server
    srv = Server(0, budget, slots)
    try:
        rng = np.random.default_rng(seed)
        t0 = srv.clock() + 5.0
        arrive = t0 + np.cumsum(rng.exponential(gap_ms, size=len(reqs))) if gap_ms > 0 else np.full(len(reqs), -1.0)
        outs = []
        for i, (alg, data) in enumerate(reqs):
            w, mn, mx = params("mixed_4g_seed1", alg, 8192)
            out = np.zeros(data.size // mn + 2, dtype=np.uint64)
            outs.append(out)
            srv.submit(data, alg, w, mn, mx, out, tag=i, arrive_ms=float(arrive[i]))
        res = {}
        while len(res) < len(reqs):
            for r in srv.poll(1024, wait_ms=200):
                res[r["tag"]] = r
        return res, outs
    finally:
        srv.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_each_request_equals_it_alone(pinned):
    import torch
    from paper_2508_05797_gb300 import Chunker
    reqs = _requests(400, 21, pinned)
    res, outs = _serve(reqs, gap_ms=0.05)
    ck = Chunker(0)
    batched = 0
    for i, (alg, data) in enumerate(reqs):
        r = res[i]
        assert r["status"] == 0, r
        assert r["t_arrive_ms"] <= r["t_start_ms"] <= r["t_done_ms"]
        batched += r["batch_size"] > 1
        w, mn, mx = params("mixed_4g_seed1", alg, 8192)
        alone = ck.chunk(torch.from_numpy(data).cuda(), alg, w, mn, mx).cpu().numpy().astype(np.uint64)
        got = outs[i][:r["n_bounds"]]
        assert np.array_equal(got, alone), (i, alg, data.size)
        assert np.array_equal(got, oracle.chunk(alg, np.ascontiguousarray(data), w, mn, mx)), (i, alg)
    ck.close()
    assert batched > 0  # requests that arrived together shared batches


def test_burst_and_capacity_errors():
    reqs = _requests(200, 33)
    res, outs = _serve(reqs, gap_ms=0.0, slots=2)
    assert all(r["status"] == 0 for r in res.values())
    assert max(r["batch_size"] for r in res.values()) > 1
    # a boundary buffer that is too small is reported per request, with the count needed
    from paper_2508_05797_gb300 import Server
    srv = Server(0, 1 << 30, 1)
    try:
        alg, data = reqs[0]
        w, mn, mx = params("mixed_4g_seed1", alg, 8192)
        small = np.zeros(1, dtype=np.uint64)
        srv.submit(data, alg, w, mn, mx, small, tag=99)
        r = []
        while not r:
            r = srv.poll(4, wait_ms=200)
        assert r[0]["status"] == 2 and r[0]["n_bounds"] > 1
    finally:
        srv.close()
