"""Helpers shared by the GPU tests (device uploads, the w table, oracle jobs)."""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def wtable():
    with open(os.path.join(HERE, "golden", "wtable.json")) as f:
        return json.load(f)


def params(sample: str, alg: str, mean: int):
    e = wtable()[sample][alg][str(mean)]
    return e["w"], e["min"], e["max"]


def to_device(arr: np.ndarray, offset: int = 0):
    """Copy a host uint8 array to the GPU at a chosen misalignment (bytes past
    a 256-byte aligned allocation)."""
    import torch
    t = torch.empty(arr.size + offset + 64, dtype=torch.uint8, device="cuda")
    v = t[offset:offset + arr.size]
    if arr.size:
        v.copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    return v


def gpu_chunk(ck, arr, alg, w, mn, mx, offset=0):
    t = to_device(arr, offset)
    return ck.chunk(t, alg, w, mn, mx).cpu().numpy().astype(np.uint64)


def _oracle_job(job):
    """Runs in a spawned process: regenerate the input and chunk it."""
    import sys
    sys.path[:0] = [ROOT, HERE]
    import oracle
    import synth
    kind, seed, total, n, alg, w, mn, mx = job
    if kind == "mixed":
        data = synth.mixed_range(seed, total, 0, n)
    else:
        data = synth.uniform(seed, n)
    return oracle.chunk(alg, data, w, mn, mx)


def oracle_pool_map(jobs, procs: int | None = None):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs or min(len(jobs), os.cpu_count() or 1)) as pool:
        return pool.map(_oracle_job, jobs)
