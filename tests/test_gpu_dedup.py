"""Chunk fingerprints and the deduplication report: equal chunks get equal
fingerprints, a one-byte change gives a different one, and the report over
dedup-shaped versions (Section 2.2, Eq. 1) equals an exact host dedup of the
oracle's chunks (length + 128-bit digest)."""
import hashlib

import numpy as np
import pytest

import oracle
import synth
from gpu_util import params, to_device

pytestmark = pytest.mark.gpu


def test_fingerprints_equal_iff_bytes_equal():
    import torch
    import paper_2508_05797_gb300 as pkg
    rng = np.random.default_rng(0)
    x = synth.uniform(4, 10_000)
    for off in (0, 1, 3):
        for L in (1, 2, 3, 4, 5, 63, 64, 65, 1000, 9999):
            data = np.concatenate([x[:L], x[:L], x[:L]])
            data[2 * L + L // 2] ^= 0x5A  # the third copy differs in one byte
            d = to_device(data, off)
            b = torch.tensor([L, 2 * L, 3 * L], dtype=torch.int64, device="cuda")
            fp = pkg.fingerprint(d, b).cpu().numpy()
            assert (fp[0] == fp[1]).all(), (off, L)
            assert (fp[0] != fp[2]).any(), (off, L)
    # chunks of equal bytes at different offsets, lengths differing only by trailing zeros
    z = np.zeros(100, dtype=np.uint8)
    d = to_device(np.concatenate([z[:8], z[:9]]), 1)
    fp = pkg.fingerprint(d, torch.tensor([8, 17], dtype=torch.int64, device="cuda")).cpu().numpy()
    assert (fp[0] != fp[1]).any()


def test_dedup_report_equals_host_dedup_of_oracle_chunks():
    import torch
    import paper_2508_05797_gb300 as pkg
    vs = synth.versions(2, 16 << 20, 5)
    for alg in ("ae", "ram"):
        w, mn, mx = params("uniform_16m_seed0", alg, 8192)
        pieces, seen, total, ubytes = [], set(), 0, 0
        for v in vs:
            d = torch.from_numpy(v).cuda()
            b = pkg.chunk(d, alg, w, mn, mx)
            pieces.append((d, b))
            o = oracle.chunk(alg, v, w, mn, mx)
            assert np.array_equal(b.cpu().numpy().astype(np.uint64), o)
            s = 0
            mv = memoryview(v)
            for e in o.tolist():
                key = (e - s, hashlib.blake2b(mv[s:e], digest_size=16).digest())
                if key not in seen:
                    seen.add(key)
                    ubytes += e - s
                s = e
            total += v.size
        rep = pkg.dedup_report(pieces)
        assert rep["total_bytes"] == total
        assert rep["unique_chunks"] == len(seen) and rep["unique_bytes"] == ubytes, (alg, rep, len(seen), ubytes)
        assert abs(rep["savings"] - (1 - ubytes / total)) < 1e-12
