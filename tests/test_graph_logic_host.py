"""The candidate-graph rules (graph_logic.cuh), built for the host, against the oracle.

The graph chain stage evaluates, for every candidate position y (a position
where some chunk can end by a natural cut), F(y) = the next candidate on the
chain that starts at y, and then follows y -> F(y) from the start of the data.
These tests check, without a GPU:

* the block-by-block candidate enumeration equals the candidate set written
  out from its definition with numpy (sliding window maxima), for RAM, AE and
  MAXP on uniform, mixed, text-like, zero-run, low-alphabet and ramp bytes;
* F(y) equals walking the oracle's next() from y until the first candidate;
* the chain the graph gives, candidate after candidate, equals the oracle's
  boundaries (so every natural cut of the true chain is a candidate).
"""
import ctypes

import numpy as np
import pytest
from scipy.ndimage import maximum_filter1d

import hostcheck
import oracle
import synth
from test_chain_logic_host import ALG_RULE, Arena, _superblocks


def _window_max_after(v, w):
    """m[p] = max v[p+1 .. p+w] (bytes past the end count as -1)."""
    x = np.concatenate([v.astype(np.int16), np.full(w + 1, -1, dtype=np.int16)])
    # maximum over [i - w//2 + origin ...]: use origin so the window is [i, i + w)
    f = maximum_filter1d(x, size=w, mode="constant", cval=-1, origin=-(w // 2))
    return f[1:v.size + 1]


def _window_max_before(v, w):
    """m[j] = max v[j-w .. j-1] (bytes before the start count as -1)."""
    x = np.concatenate([np.full(w, -1, dtype=np.int16), v.astype(np.int16)])
    f = maximum_filter1d(x, size=w, mode="constant", cval=-1, origin=-(w // 2))
    return f[:v.size]


def expected_cands(alg, data, w):
    """Candidate positions y (offsets into data), from the definitions."""
    v = data if alg != "ae_min" else (255 - data)
    n = v.size
    if alg == "ram":
        if n <= w + 1:
            return np.zeros(0, dtype=np.int64)
        pm = _window_max_before(v, w)
        j = np.arange(w, n - 1)
        ok = (v[j] > 0) & (v[j].astype(np.int16) >= pm[j])
        return j[ok] + 1
    if alg in ("ae", "ae_min"):
        if n <= w + 1:
            return np.zeros(0, dtype=np.int64)
        am = _window_max_after(v, w)
        p = np.arange(0, n - w - 1)
        ok = (v[p] > 0) & (v[p].astype(np.int16) >= am[p])
        return p[ok] + w + 1
    t = oracle.maxp_targets(data, w)
    return np.asarray(t, dtype=np.int64) + 1


def _lib_args(ar, sup, alg, w, mn, mx, flo, fhi):
    base, sm, sa = ar.ptrs()
    return (ALG_RULE[alg][0], base, sm, sa, sup.ctypes.data, ar.inv, w, mn, mx, flo, fhi)


def _datasets(n, seed):
    rng = np.random.default_rng(seed)
    zeros = np.zeros(n, dtype=np.uint8)
    k = max(n // 20000, 3)
    zeros[rng.integers(0, n, size=k)] = rng.integers(1, 256, size=k)
    return {
        "uniform": synth.uniform(seed, n),
        "mixed": synth.mixed_range(seed, 64 << 20, 3 << 20, n),
        "text": synth.mixed_range(1, 4 << 30, 6 << 20, n),  # block 6 of the 4 GiB stream is text-like
        "zero_runs": zeros,
        "ternary": rng.integers(0, 3, size=n).astype(np.uint8),
        "ramp": (np.arange(n) % 251).astype(np.uint8),
        # random bytes, then text-like bytes: RAM chains from the random part
        # meet forced cuts in the text before their next natural cut
        "uniform_then_text": np.concatenate([synth.uniform(seed + 1, n // 2),
                                             synth.mixed_range(1, 4 << 30, 6 << 20, n - n // 2)]),
    }


CASES = [
    # alg, w, min, max  (RAM / AE: w >= 64 and min <= w + 1; MAXP: w >= 63)
    ("ram", 64, 1, 2000), ("ram", 700, 128, 8192), ("ram", 3000, 900, 30000), ("ram", 7101, 2048, 65536),
    ("ae", 64, 65, 1000), ("ae", 700, 128, 8192), ("ae", 3000, 2000, 30000),
    ("maxp", 63, 1, 2000), ("maxp", 150, 512, 8192), ("maxp", 291, 2048, 65536),
]


@pytest.mark.parametrize("alg,w,mn,mx", CASES)
def test_graph_candidates_and_chain(alg, w, mn, mx):
    lib = hostcheck.load()
    orc = oracle.get()
    n = 300_000
    for k, (name, data) in enumerate(_datasets(n, seed=w + mn).items()):
        lo = (11 * k + w) % 64
        ar = Arena(data, lo, alg, w)
        sup = _superblocks(ar, alg)
        for (a, b) in ((0, n), (777, 777 + 123_457), (5000, 5000 + w + 1)):
            fd = np.ascontiguousarray(data[a:b])
            flo, fhi = lo + a, lo + b
            args = _lib_args(ar, sup, alg, w, mn, mx, flo, fhi)
            # 1. enumeration equals the definition
            exp_c = expected_cands(alg, fd, w)
            out = np.zeros(exp_c.size + 8, dtype=np.uint64)
            got_n = lib.hc_cands(*args, out.ctypes.data, out.size)
            got_c = out[:got_n].astype(np.int64) - flo
            assert got_n == exp_c.size and np.array_equal(got_c, exp_c), (alg, name, a, b, got_n, exp_c.size)
            # 2. the graph's chain equals the oracle's boundaries
            exp = orc.chunk(alg, fd, w, mn, mx)
            ob = np.zeros(exp.size + 8, dtype=np.uint64)
            nb = lib.hc_graph_chain(*args, ob.ctypes.data, ob.size)
            assert nb == exp.size and np.array_equal(ob[:nb], exp), (alg, name, a, b)
            # every natural cut of the true chain past a non-zero byte is a candidate
            cset = set(exp_c.tolist())
            # 3. F(y) from sampled candidates equals walking next() to the next candidate
            rng = np.random.default_rng(k)
            ys = exp_c[rng.integers(0, exp_c.size, size=min(40, exp_c.size))] if exp_c.size else []
            for y in list(ys) + [0]:
                y = int(y)
                cnt, s = 0, y
                while True:
                    s = orc.next(alg, fd, s, w, mn, mx)
                    cnt += 1
                    if s >= fd.size or s in cset:
                        break
                c = ctypes.c_uint32()
                e = lib.hc_cand_next(*args, flo + y, ctypes.byref(c))
                assert (e - flo, c.value) == (min(s, fd.size), cnt), (alg, name, y)


@pytest.mark.parametrize("alg,w", [("ram", 700), ("ae", 700), ("maxp", 150)])
def test_is_cand_matches_enumeration(alg, w):
    lib = hostcheck.load()
    data = synth.mixed_range(2, 64 << 20, 1 << 20, 200_000)
    lo = 29
    ar = Arena(data, lo, alg, w)
    sup = _superblocks(ar, alg)
    args = _lib_args(ar, sup, alg, w, 1, 60_000, lo, lo + data.size)
    cset = set(expected_cands(alg, data, w).tolist())
    rng = np.random.default_rng(5)
    ys = np.unique(np.concatenate([np.array(sorted(cset))[:3000], rng.integers(0, data.size + 1, size=3000)]))
    for y in ys.tolist():
        assert lib.hc_is_cand(*args, lo + y) == (1 if y in cset else 0), (alg, y)


@pytest.mark.parametrize("alg,w,mn,mx", [("ram", 200, 100, 4000), ("ram", 7101, 2048, 65536), ("ae", 700, 128, 8192),
                                          ("ae", 3000, 2000, 30000), ("ram", 3548, 1024, 32768),
                                          ("ae", 15599, 4096, 131072)])
def test_graph_chain_with_superblock_maxima(alg, w, mn, mx):
    """Window maxima from the running maxima inside 4 KiB superblocks (prefix
    and suffix per block, as the summary kernel writes them) give the same
    chain as the block-by-block summaries."""
    lib = hostcheck.load()
    orc = oracle.get()
    n = 300_000
    for k, (name, data) in enumerate(_datasets(n, seed=w).items()):
        lo = (5 * k + 3) % 64
        ar = Arena(data, lo, alg, w)
        sup = _superblocks(ar, alg)
        nb = ar.smax.size
        m = ar.smax.copy()
        pre = np.zeros(nb + 64, dtype=np.uint8)
        suf = np.zeros(nb + 64, dtype=np.uint8)
        for q0 in range(0, nb, 64):
            blk = m[q0:q0 + 64]
            pre[q0:q0 + blk.size] = np.maximum.accumulate(blk)
            suf[q0:q0 + blk.size] = np.maximum.accumulate(blk[::-1])[::-1]
        base, sm, sa = ar.ptrs()
        exp = orc.chunk(alg, data, w, mn, mx)
        out = np.zeros(exp.size + 8, dtype=np.uint64)
        got = lib.hc_graph_chain_t(ALG_RULE[alg][0], base, sm, sa, sup.ctypes.data, ar.inv, w, mn, mx, lo, lo + n,
                                   pre.ctypes.data, suf.ctypes.data, out.ctypes.data, out.size)
        assert got == exp.size and np.array_equal(out[:got], exp), (alg, name)


@pytest.mark.parametrize("alg,w,mn,mx", CASES)
def test_list_next_equals_cand_next(alg, w, mn, mx):
    """F from the sorted candidate list (the natural cuts) equals F by stepping
    the chain, for every candidate the list decides; the list decides most of
    them on random and text-like bytes."""
    lib = hostcheck.load()
    n = 300_000
    for k, (name, data) in enumerate(_datasets(n, seed=w + 3).items()):
        lo = (3 * k + 1) % 64
        ar = Arena(data, lo, alg, w)
        sup = _superblocks(ar, alg)
        args = _lib_args(ar, sup, alg, w, mn, mx, lo, lo + n)
        cands = expected_cands(alg, data, w) + lo
        cands = np.concatenate([[lo], cands]).astype(np.uint64)  # the chain start is listed first
        vals = np.zeros(cands.size, dtype=np.uint8)
        v = data if alg != "ae_min" else 255 - data
        shift = 1 if alg in ("ram", "maxp") else w + 1
        vals[1:] = v[(cands[1:] - lo - shift).astype(np.int64)]
        pos = (cands - lo).astype(np.uint32)
        out = np.zeros(max(cands.size, 1), dtype=np.uint32)
        got = lib.hc_list_check(*args, pos.ctypes.data, vals.ctypes.data, cands.size, lo, out.ctypes.data)
        assert got < (1 << 63), (alg, name, "candidate %d disagrees" % ((1 << 64) - 1 - got))
        if name in ("uniform", "text") and cands.size > 100:
            assert got >= 0.9 * (cands.size - 1), (alg, name, got, cands.size)
