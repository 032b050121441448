"""Calibrate the window size w per (algorithm, target mean chunk size).

The paper gives no formula from the window size to the mean chunk size (it
only notes that MAXP needs windows 70-80% smaller than AE and RAM for the
same mean, Section 2.1). So w is calibrated on a sample of each workload with
the CPU oracle: the integer w whose mean chunk size (sample length / number
of chunks) is closest to the target, found by a binary search for the first
w reaching the target and a scan of the 8 values on either side; ties go to
the smaller w. The table is then a fixed input for both the oracle and the
GPU path.

Run:  python tests/golden/make_wtable.py   (writes tests/golden/wtable.json)
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path[:0] = [ROOT]

SAMPLES = {
    # 16 MiB of uniform bytes, seed 0 (the single-buffer RAM workload)
    "uniform_16m_seed0": dict(kind="uniform", seed=0, n=16 << 20, means=(8192,),
                              algs=("ram", "ae", "maxp"), fixed_min_max=(2048, 65536)),
    # first 256 MiB of the 4 GiB mixed stream, seed 1
    "mixed_4g_seed1": dict(kind="mixed", seed=1, total=4 << 30, n=256 << 20,
                           means=(4096, 8192, 16384), algs=("ram", "ae", "maxp"),
                           fixed_min_max=None),
}


def _sample(spec):
    import synth
    if spec["kind"] == "uniform":
        return synth.uniform(spec["seed"], spec["n"])
    return synth.mixed_range(spec["seed"], spec["total"], 0, spec["n"])


def calibrate(job):
    name, alg, mean = job
    import oracle
    spec = SAMPLES[name]
    data = _sample(spec)
    mn, mx = spec["fixed_min_max"] or (mean // 4, mean * 8)
    cache = {}

    def avg(w):
        if w not in cache:
            cache[w] = data.size / oracle.count(alg, data, w, mn, mx)
        return cache[w]

    hi_w = mx - 1 if alg != "maxp" else mean
    lo, hi = 1, hi_w
    while lo < hi:                       # first w with mean >= target
        mid = (lo + hi) // 2
        if avg(mid) >= mean:
            hi = mid
        else:
            lo = mid + 1
    best = None
    for w in range(max(1, lo - 8), min(hi_w, lo + 8) + 1):
        d = abs(avg(w) - mean)
        if best is None or d < best[0] or (d == best[0] and w < best[1]):
            best = (d, w)
    w = best[1]
    return name, alg, mean, w, avg(w), mn, mx


def main():
    jobs = [(name, alg, mean) for name, spec in SAMPLES.items()
            for alg in spec["algs"] for mean in spec["means"]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(calibrate, jobs)
    table = {"method": __doc__.strip().splitlines()[0],
             "samples": {k: {kk: vv for kk, vv in v.items() if kk != "fixed_min_max"}
                         for k, v in SAMPLES.items()}}
    for name, alg, mean, w, got, mn, mx in res:
        table.setdefault(name, {}).setdefault(alg, {})[str(mean)] = dict(
            w=w, min=mn, max=mx, sample_mean=round(got, 2))
    with open(os.path.join(HERE, "wtable.json"), "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
