"""The chain stage's per-thread rules, built for the host, against the oracle.

The GPU chain stage calls next_cut<RULE>() from chain_logic.cuh for every
step. These tests compile that header for the CPU (tests/hostcheck), feed it
block summaries computed here with numpy (and MAXP targets from the oracle),
and compare next(s) and whole chains with the oracle: bit-exact, for every
algorithm, at start offsets 0..63 inside a 64-byte block, with files placed
inside a larger arena so that summary blocks straddle file edges.
"""
import numpy as np
import pytest

import hostcheck
import oracle
import synth

ALG_RULE = {"ram": (hostcheck.RULE_RAM, hostcheck.RULE_RAM_BYTES),
            "ae": (hostcheck.RULE_AE, hostcheck.RULE_AE_BYTES),
            "ae_min": (hostcheck.RULE_AE, hostcheck.RULE_AE_BYTES),
            "maxp": (hostcheck.RULE_MAXP, hostcheck.RULE_MAXP_BYTES)}


class Arena:
    """Bytes placed at physical offset lo of a 64-byte aligned buffer, with
    block summaries as the summary kernel defines them."""

    def __init__(self, data, lo, alg, w):
        n = data.size
        self.lo, self.hi = lo, lo + n
        nblk = (self.hi + 63) // 64
        self.nblk_pad = (nblk + 15) // 16 * 16
        raw = np.zeros(self.nblk_pad * 64 + 256 + 64, dtype=np.uint8)
        off = (-raw.ctypes.data) % 64
        self.buf = raw[off:off + self.nblk_pad * 64 + 256]
        self.buf[lo:lo + n] = data
        self.inv = 0xFFFFFFFF if alg == "ae_min" else 0
        vals = self.buf[:nblk * 64].copy()
        if alg == "ae_min":
            vals = 255 - vals
        vals[:lo] = 0
        vals[self.hi:] = 0
        blocks = vals.reshape(nblk, 64)
        self.smax = np.zeros(self.nblk_pad + 64, dtype=np.uint8)
        self.sarg = np.zeros(self.nblk_pad + 64, dtype=np.uint8)
        if alg == "maxp":
            self.smax[:] = 0xFF
            if w >= 63:
                for t in oracle.maxp_targets(data, w):
                    p = int(t) + lo
                    assert self.smax[p >> 6] == 0xFF  # at most one target per block
                    self.smax[p >> 6] = p & 63
        else:
            self.smax[:nblk] = blocks.max(axis=1)
            self.sarg[:nblk] = blocks.argmax(axis=1)

    def ptrs(self):
        return self.buf.ctypes.data, self.smax.ctypes.data, self.sarg.ctypes.data


def _check(alg, data, w, mn, mx, lo, files, rules, n_starts=300, seed=0):
    lib = hostcheck.load()
    orc = oracle.get()
    ar = Arena(data, lo, alg, w)
    base, sm, sa = ar.ptrs()
    rng = np.random.default_rng(seed)
    for (a, b) in files:
        fd = np.ascontiguousarray(data[a:b])
        flo, fhi = lo + a, lo + b
        exp = orc.chunk(alg, fd, w, mn, mx)
        for rule in rules:
            out = np.zeros(exp.size + 4, dtype=np.uint64)
            n = lib.hc_chain(rule, base, sm, sa, ar.inv, w, mn, mx, flo, fhi, out.ctypes.data, out.size)
            assert n == exp.size and np.array_equal(out[:n], exp), (alg, rule, w, mn, mx, lo, a, b)
            if b - a == 0:
                continue
            ss = np.unique(np.concatenate([np.arange(min(b - a, 70)),
                                           rng.integers(0, b - a, size=n_starts)]))
            for s in ss.tolist():
                e = orc.next(alg, fd, s, w, mn, mx)
                g = lib.hc_next(rule, base, sm, sa, 0, 0, None, None, ar.inv, w, mn, mx, flo, fhi, flo + s) - flo
                assert g == e, (alg, rule, w, mn, mx, lo, a, b, s, g, e)
    # a staged window of summaries gives the same answers
    if rules[0] in (hostcheck.RULE_RAM, hostcheck.RULE_AE, hostcheck.RULE_MAXP):
        wb0 = ((lo + data.size // 3) >> 6) & ~15
        wn = 64
        wm = np.ascontiguousarray(ar.smax[wb0:wb0 + wn])
        wa = np.ascontiguousarray(ar.sarg[wb0:wb0 + wn])
        a, b = files[0]
        fd = np.ascontiguousarray(data[a:b])
        for s in rng.integers(0, max(b - a, 1), size=n_starts).tolist():
            if b - a == 0:
                break
            e = orc.next(alg, fd, s, w, mn, mx)
            g = lib.hc_next(rules[0], base, sm, sa, wb0, wn, wm.ctypes.data, wa.ctypes.data, ar.inv, w, mn, mx,
                            lo + a, lo + b, lo + a + s) - (lo + a)
            assert g == e


def _datasets(n, seed):
    rng = np.random.default_rng(seed)
    mixed = synth.mixed_range(seed, 64 << 20, 0, n)
    uni = synth.uniform(seed, n)
    small = rng.integers(0, 3, size=n).astype(np.uint8)
    spikes = np.zeros(n, dtype=np.uint8)
    spikes[rng.integers(0, n, size=n // 500)] = rng.integers(1, 256, size=n // 500)
    ramp = (np.arange(n) % 251).astype(np.uint8)
    return {"uniform": uni, "mixed": mixed, "ternary": small, "spikes": spikes, "ramp": ramp}


CASES = [
    # alg, w, min, max
    ("ram", 1, 1, 9), ("ram", 5, 3, 40), ("ram", 63, 1, 500), ("ram", 64, 64, 2000),
    ("ram", 700, 128, 8192), ("ram", 3000, 900, 30000),
    ("ae", 64, 1, 1000), ("ae", 65, 100, 3000), ("ae", 700, 128, 8192), ("ae", 3000, 2000, 30000),
    ("ae_min", 64, 1, 1000), ("ae_min", 700, 128, 8192),
    ("maxp", 63, 1, 2000), ("maxp", 64, 200, 4000), ("maxp", 150, 512, 8192), ("maxp", 300, 64, 65536),
]


@pytest.mark.parametrize("alg,w,mn,mx", CASES)
def test_summary_rules_match_oracle(alg, w, mn, mx):
    n = 160_000
    for k, (name, data) in enumerate(_datasets(n, seed=w + mn).items()):
        lo = (7 * k + w) % 64
        files = [(0, n), (1000, 1000 + 77_777), (50_001, 50_001 + 123), (90_000, 90_000 + 1)]
        _check(alg, data, w, mn, mx, lo, files, ALG_RULE[alg], n_starts=120, seed=k)


@pytest.mark.parametrize("alg,w,mn,mx", [("ram", 2, 1, 11), ("ae", 3, 2, 17), ("ae_min", 7, 1, 30),
                                          ("maxp", 1, 1, 20), ("maxp", 4, 3, 50), ("maxp", 30, 10, 300)])
def test_byte_rules_small_windows(alg, w, mn, mx):
    n = 20_000
    for k, (name, data) in enumerate(_datasets(n, seed=w).items()):
        lo = (13 * k + 5) % 64
        files = [(0, n), (333, 333 + 4_444), (10_000, 10_000 + 5)]
        _check(alg, data, w, mn, mx, lo, files, (ALG_RULE[alg][1],), n_starts=100, seed=k)


def test_block_max_first_matches_numpy():
    lib = hostcheck.load()
    import ctypes
    rng = np.random.default_rng(3)
    for t in range(2000):
        blk = rng.integers(0, (2, 5, 256)[t % 3], size=64).astype(np.uint8)
        m, f = ctypes.c_uint32(), ctypes.c_uint32()
        lib.hc_block_max_first(blk.ctypes.data, ctypes.byref(m), ctypes.byref(f))
        assert m.value == blk.max() and f.value == int(np.argmax(blk))


def _superblocks(ar, alg):
    nsup = (ar.hi + 4095) // 4096 + 2
    sup = np.zeros(nsup + 32, dtype=np.uint8)  # room for 16-byte reads past the end
    nblk = (ar.hi + 63) // 64
    if alg == "maxp":
        has = (ar.smax[:nblk] != 0xFF).astype(np.int64)
        cnt = np.add.reduceat(has, np.arange(0, nblk, 64)) if nblk else np.zeros(0)
        sup[:cnt.size] = np.minimum(cnt, 255)
    else:
        m = ar.smax[:nblk]
        mx = np.maximum.reduceat(m, np.arange(0, nblk, 64)) if nblk else np.zeros(0)
        sup[:mx.size] = mx
    return sup


@pytest.mark.parametrize("alg,w,mn,mx", [("ram", 700, 128, 8192), ("ram", 3000, 1024, 30000), ("ae", 700, 128, 8192),
                                          ("ae_min", 300, 64, 4096), ("maxp", 150, 512, 8192),
                                          ("maxp", 300, 2048, 65536), ("ram", 64, 65, 2000)])
def test_fast_forward_matches_oracle(alg, w, mn, mx):
    """advance(): many steps at once through zero runs (RAM/AE) and through
    target-less stretches (MAXP), exactly equal to the oracle's chain."""
    lib = hostcheck.load()
    orc = oracle.get()
    rng = np.random.default_rng(w)
    n = 1_500_000
    zeros = np.zeros(n, dtype=np.uint8)
    zeros[rng.integers(0, n, size=40)] = rng.integers(1, 256, size=40)
    ones = np.full(n, 255, dtype=np.uint8)
    ones[rng.integers(0, n, size=40)] = rng.integers(0, 255, size=40)
    mixed = synth.mixed_range(11, 64 << 20, 5 << 20, n)
    text = synth.mixed_range(1, 4 << 30, 6 << 20, n)  # block 6 of the 4 GiB stream is text-like
    total_jumps = 0
    for data in (zeros, ones, mixed, text):
        for lo in (0, 17):
            ar = Arena(data, lo, alg, w)
            sup = _superblocks(ar, alg)
            base, sm, sa = ar.ptrs()
            rule = ALG_RULE[alg][0]
            for (a, b) in ((0, n), (12_345, 12_345 + 400_001)):
                exp = orc.chunk(alg, np.ascontiguousarray(data[a:b]), w, mn, mx)
                for stop_every in (0, 65536, 4096):
                    out = np.zeros(exp.size + 4, dtype=np.uint64)
                    jumps = np.zeros(1, dtype=np.uint64)
                    got_n = lib.hc_chain_adv(rule, base, sm, sa, sup.ctypes.data, ar.inv, w, mn, mx, lo + a, lo + b,
                                             stop_every, out.ctypes.data, out.size, jumps.ctypes.data)
                    assert got_n == exp.size and np.array_equal(out[:got_n], exp), (alg, lo, a, b, stop_every)
                    total_jumps += int(jumps[0])
    assert total_jumps > 0  # the fast path was exercised
