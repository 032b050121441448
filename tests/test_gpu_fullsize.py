"""Full-size workloads in the benchmark's launch configuration.

* The 4 GiB mixed stream (seed 1) with RAM, AE and MAXP at the calibrated
  windows: the 8 KiB-mean runs are compared with the oracle over the whole
  stream (oracle runs in spawned processes that regenerate the bytes); the
  4 and 16 KiB runs are checked boundary by boundary on a random sample
  (b[i+1] == next(b[i]) by the oracle, first and last boundary exact).
* Dedup-shaped versions: a uniform base plus 15 versions with 0.1% of the
  bytes edited; AE and RAM boundaries equal the oracle's on every version,
  so the unique-chunk ratio and space savings (Section 2.2, Eq. 1) do too.
"""
import hashlib

import numpy as np
import pytest

import oracle
import synth
from gpu_util import oracle_pool_map, params, to_device

pytestmark = pytest.mark.gpu

MIB = 1 << 20
GIB = 1 << 30


@pytest.fixture(scope="module")
def ck():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_05797_gb300 import Chunker
    c = Chunker(0)
    yield c
    c.close()


def test_mixed_4gib_all_algorithms(ck):
    import torch
    n = 4 * GIB
    jobs = []
    for alg in ("ram", "ae", "maxp"):
        w, mn, mx = params("mixed_4g_seed1", alg, 8192)
        jobs.append(("mixed", 1, n, n, alg, w, mn, mx))
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(len(jobs))
    async_res = pool.map_async(__import__("gpu_util")._oracle_job, jobs)
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    data = synth.mixed_range(1, n, 0, n, out=host.numpy())
    dev = host.cuda()
    got = {}
    for alg in ("ram", "ae", "maxp"):
        for mean in (4096, 8192, 16384):
            w, mn, mx = params("mixed_4g_seed1", alg, mean)
            got[(alg, mean)] = ck.chunk(dev, alg, w, mn, mx).cpu().numpy().astype(np.uint64)
    del dev
    rng = np.random.default_rng(0)
    for alg in ("ram", "ae", "maxp"):
        for mean in (4096, 16384):
            w, mn, mx = params("mixed_4g_seed1", alg, mean)
            b = got[(alg, mean)]
            assert b[-1] == n and np.all(np.diff(b.astype(np.int64)) > 0)
            assert b[0] == oracle.next_cut(alg, data, 0, w, mn, mx)
            for i in rng.integers(0, b.size - 1, size=1500).tolist():
                assert b[i + 1] == oracle.next_cut(alg, data, int(b[i]), w, mn, mx), (alg, mean, i)
    exp = async_res.get(timeout=1200)
    pool.close()
    pool.join()
    for (alg, *_), e in zip([(j[4],) for j in jobs], exp):
        assert np.array_equal(got[(alg, 8192)], e), alg


def test_versions_dedup_equal_oracle(ck):
    base_n = 128 * MIB
    vs = synth.versions(2, base_n, 15)
    total = sum(v.size for v in vs)
    for alg in ("ae", "ram"):
        w, mn, mx = params("uniform_16m_seed0", alg, 8192)
        seen = set()
        uniq_bytes = 0
        for v in vs:
            g = ck.chunk(to_device(v), alg, w, mn, mx).cpu().numpy().astype(np.uint64)
            o = oracle.chunk(alg, v, w, mn, mx)
            assert np.array_equal(g, o), (alg, v.size)
            s = 0
            mv = memoryview(v)
            for e in g.tolist():
                key = (e - s, hashlib.blake2b(mv[s:e], digest_size=16).digest())
                if key not in seen:
                    seen.add(key)
                    uniq_bytes += e - s
                s = e
        # equal boundaries give equal unique chunks and savings (Eq. 1); the
        # versions share most of their bytes, so most chunks repeat
        savings = (total - uniq_bytes) / total * 100.0
        assert savings > 50.0, (alg, savings)
