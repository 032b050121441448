"""Full-size workloads, at the benchmark's sizes, against the oracle.

* The 4 GiB mixed stream (seed 1): all nine (algorithm, mean) pairs, the
  whole boundary list, with the automatic chain stage and with the candidate
  graph forced.
* Dedup-shaped versions: the 1 GiB uniform base (seed 2) and 15 versions,
  AE and RAM at 8 KiB mean, every version's boundaries equal the oracle's;
  the GPU dedup report (unique chunks, unique bytes, Eq. 1 savings) equals an
  exact host dedup (length + BLAKE2b-128) of the oracle's chunks.
* The 100,000-file arena (log-normal sizes, seed 3, about 20 GB), MAXP and
  RAM in one batched call, every file's boundaries equal the oracle's.
* The serving workload: 20,000 requests cut from the pinned 4 GiB stream,
  every served result equals the oracle's boundaries for its bytes.

The oracle runs on host threads (its C loops release the GIL), over the same
host arrays the GPU inputs were copied from.
"""
import hashlib
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth
from gpu_util import params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

MIB = 1 << 20
GIB = 1 << 30
THREADS = max(1, os.cpu_count() or 1)


@pytest.fixture(scope="module")
def ck():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_05797_gb300 import Chunker
    c = Chunker(0)
    yield c
    c.close()


def test_mixed_4gib_all_pairs_full(ck):
    import torch
    from paper_2508_05797_gb300 import cdc
    n = 4 * GIB
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    data = synth.mixed_range(1, n, 0, n, out=host.numpy())
    pairs = [(alg, mean) for alg in ("ram", "ae", "maxp") for mean in (4096, 8192, 16384)]
    with ThreadPoolExecutor(min(THREADS, len(pairs))) as ex:
        futs = {p: ex.submit(oracle.chunk, p[0], data, *params("mixed_4g_seed1", *p)) for p in pairs}
        dev = host.cuda()
        got = {}
        for pipe in (0, 2):
            ck.set_option(cdc.OPT_PIPELINE, pipe)
            for alg, mean in pairs:
                w, mn, mx = params("mixed_4g_seed1", alg, mean)
                got[(pipe, alg, mean)] = ck.chunk(dev, alg, w, mn, mx).cpu().numpy().astype(np.uint64)
        ck.set_option(cdc.OPT_PIPELINE, 0)
        del dev
        for p in pairs:
            exp = futs[p].result()
            for pipe in (0, 2):
                assert np.array_equal(got[(pipe,) + p], exp), (pipe, p, got[(pipe,) + p].size, exp.size)


def _host_dedup(pieces):
    """Exact dedup of (bytes, boundaries) pieces: unique chunks and bytes by
    (length, BLAKE2b-128), hashed on host threads."""
    def keys(piece):
        data, bounds = piece
        mv = memoryview(data)
        s, out = 0, []
        for e in bounds.tolist():
            out.append((e - s, hashlib.blake2b(mv[s:e], digest_size=16).digest()))
            s = e
        return out
    seen, uniq_bytes, chunks = set(), 0, 0
    with ThreadPoolExecutor(THREADS) as ex:
        for ks in ex.map(keys, pieces):
            for k in ks:
                chunks += 1
                if k not in seen:
                    seen.add(k)
                    uniq_bytes += k[0]
    return chunks, len(seen), uniq_bytes


def test_versions_1gib_base_dedup_equal_oracle(ck):
    import torch
    from paper_2508_05797_gb300 import dedup_report
    vs = synth.versions(2, GIB, 15)
    total = sum(v.size for v in vs)
    for alg in ("ae", "ram"):
        w, mn, mx = params("uniform_16m_seed0", alg, 8192)
        with ThreadPoolExecutor(THREADS) as ex:
            exp = list(ex.map(lambda v: oracle.chunk(alg, v, w, mn, mx), vs))
        pieces_gpu = []
        for v, e in zip(vs, exp):
            d = torch.from_numpy(v).cuda()
            b = ck.chunk(d, alg, w, mn, mx)
            assert np.array_equal(b.cpu().numpy().astype(np.uint64), e), (alg, v.size)
            pieces_gpu.append((d, b))
        rep = dedup_report(pieces_gpu)
        del pieces_gpu
        torch.cuda.empty_cache()
        chunks, uniq, uniq_bytes = _host_dedup(list(zip(vs, exp)))
        assert rep["chunks"] == chunks and rep["unique_chunks"] == uniq, (alg, rep, chunks, uniq)
        assert abs(rep["savings"] - (total - uniq_bytes) / total) < 1e-12, (alg, rep["savings"])


def test_batched_100k_files_each_equal_oracle(ck):
    import torch
    n_files = 100_000
    sizes = synth.lognormal_sizes(3, n_files, 65536, 1.5, 1, 256 * MIB).astype(np.int64)
    off = np.zeros(n_files + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    total = int(off[-1])
    arena = synth.mixed(3, total)
    dev = torch.from_numpy(arena).cuda()
    d_off = torch.from_numpy(off).cuda()
    groups = np.array_split(np.arange(n_files), THREADS * 4)
    for alg in ("maxp", "ram"):
        w, mn, mx = params("mixed_4g_seed1", alg, 8192)
        b, idx = ck.chunk_batch(dev, d_off, alg, w, mn, mx)
        b = b.cpu().numpy().astype(np.uint64)
        idx = idx.cpu().numpy()

        def check(files):
            bad = []
            for f in files.tolist():
                e = oracle.chunk(alg, arena[off[f]:off[f + 1]], w, mn, mx)
                if not np.array_equal(b[idx[f]:idx[f + 1]], e):
                    bad.append(f)
            return bad

        with ThreadPoolExecutor(THREADS) as ex:
            bad = [f for r in ex.map(check, groups) for f in r]
        assert not bad, (alg, bad[:10])
        assert idx[-1] == b.size


def test_serving_every_request_equals_oracle():
    import torch
    from paper_2508_05797_gb300 import Server
    n = 4 * GIB
    host = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    hnp = synth.mixed_range(1, n, 0, n, out=host.numpy())
    n_req = 20_000
    sizes = synth.lognormal_sizes(4, n_req, 65536, 1.5, 4096, 64 * MIB).astype(np.int64)
    algs = synth.choice(4, n_req, 3)
    starts = (synth.lognormal_sizes(6, n_req, 1 << 30, 4.0, 0, n) % np.maximum(1, n - sizes)).astype(np.int64)
    names = ("ram", "ae", "maxp")
    prm = [params("mixed_4g_seed1", a, 8192) for a in names]
    outs = [np.zeros(int(sizes[i]) // prm[int(algs[i])][1] + 2, dtype=np.uint64) for i in range(n_req)]
    srv = Server(0, 40 << 30, 4)
    try:
        for i in range(n_req):
            w, mn, mx = prm[int(algs[i])]
            srv.submit(hnp[starts[i]:starts[i] + sizes[i]], names[int(algs[i])], w, mn, mx, outs[i], tag=i)
        res = {}
        while len(res) < n_req:
            for r in srv.poll(4096, wait_ms=200):
                res[r["tag"]] = r
    finally:
        srv.close()
    assert all(r["status"] == 0 for r in res.values())

    def check(ids):
        bad = []
        for i in ids.tolist():
            w, mn, mx = prm[int(algs[i])]
            e = oracle.chunk(names[int(algs[i])], hnp[starts[i]:starts[i] + sizes[i]], w, mn, mx)
            if not np.array_equal(outs[i][:res[i]["n_bounds"]], e):
                bad.append(i)
        return bad

    with ThreadPoolExecutor(THREADS) as ex:
        bad = [i for r in ex.map(check, np.array_split(np.arange(n_req), THREADS * 4)) for i in r]
    assert not bad, bad[:10]
