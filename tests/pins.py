"""Checks that pin the CPU oracle to the paper and to mathematics.

Every function takes an ``oracle.Oracle`` instance and raises AssertionError
on a mismatch, so the same checks run against the real oracle (the pin tests)
and against deliberately broken copies of it (the mutation test, which shows
that each planted mistake is caught by at least one pin).
"""
from __future__ import annotations

import math
import os

import numpy as np

import brute

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ALGS = ("ram", "ae", "ae_min", "maxp")


def load_hand_examples():
    cases, cur = [], {}
    with open(os.path.join(GOLDEN, "hand_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                if cur:
                    cases.append(cur)
                    cur = {}
                continue
            key, _, val = line.partition(" ")
            cur[key] = val
    if cur:
        cases.append(cur)
    out = []
    for c in cases:
        out.append(dict(name=c["name"], alg=c["alg"], w=int(c["w"]), min=int(c["min"]),
                        max=int(c["max"]),
                        data=np.array([int(x, 16) for x in c["bytes"].split()], dtype=np.uint8),
                        bounds=[int(x) for x in c["bounds"].split()]))
    return out


def check_hand_examples(orc):
    for c in load_hand_examples():
        got = orc.chunk(c["alg"], c["data"], c["w"], c["min"], c["max"]).tolist()
        assert got == c["bounds"], (c["name"], got, c["bounds"])


def _valid_params(alg, w, mn, mx):
    if mn < 1 or mn > mx or w < 1:
        return False
    if alg != "maxp" and w >= mx:
        return False
    return True


def check_brute_small(orc, seed=1234, trials=120, max_len=48):
    """next(s) for every s, and whole chains, against brute force."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        alg = ALGS[t % len(ALGS)]
        alphabet = (2, 3, 4, 256)[(t // 4) % 4]
        n = int(rng.integers(0, max_len + 1))
        B = rng.integers(0, alphabet, size=n).astype(np.uint8)
        if alphabet < 256 and t % 3 == 0:
            B = (B * 85 + 3).astype(np.uint8)   # spread over the byte range
        w = int(rng.integers(1, 7))
        mn = int(rng.integers(1, 10))
        mx = int(rng.integers(max(mn, w + 1), 40))
        if not _valid_params(alg, w, mn, mx):
            continue
        Bl = [int(x) for x in B]
        targets = brute.maxp_targets(Bl, w) if alg == "maxp" else None
        for s in range(n):
            exp = brute.next_cut(alg, Bl, s, w, mn, mx, targets)
            got = orc.next(alg, B, s, w, mn, mx)
            assert got == exp, (alg, Bl, s, w, mn, mx, got, exp)
        assert orc.chunk(alg, B, w, mn, mx).tolist() == brute.chunk(alg, Bl, w, mn, mx)


def check_alternative_forms(orc, seed=99, trials=80, max_len=60):
    """RAM as 'first weak record past the window' and AE-Max as 'first clear
    target' (both when min is within w + 1), and the MAXP target set."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        n = int(rng.integers(1, max_len + 1))
        B = rng.integers(0, (3, 8, 256)[t % 3], size=n).astype(np.uint8)
        Bl = [int(x) for x in B]
        w = int(rng.integers(1, 8))
        mn = int(rng.integers(1, w + 2))
        mx = int(rng.integers(w + 1, 50))
        for s in range(n):
            assert orc.next("ram", B, s, w, mn, mx) == brute.ram_next_weak_record(Bl, s, w, mn, mx)
            assert orc.next("ae", B, s, w, mn, mx) == brute.ae_next_records(Bl, s, w, mn, mx)
        assert orc.maxp_targets(B, w).tolist() == brute.maxp_targets(Bl, w)


def check_closed_forms(orc):
    # Constant input with min <= w+1: RAM and AE cut every w+1 bytes (the
    # window maximum equals every byte; no byte exceeds a target). MAXP has
    # no target, so every chunk is max bytes.
    for c in (0, 7, 255):
        for (n, w, mn, mx) in ((100, 4, 1, 50), (257, 9, 10, 33), (64, 1, 2, 5)):
            B = np.full(n, c, dtype=np.uint8)
            # RAM: the last chunk is whatever remains once <= w bytes are left
            ram_exp = []
            s = 0
            while s < n:
                s = n if n - s <= w else s + w + 1
                ram_exp.append(s)
            assert orc.chunk("ram", B, w, mn, mx).tolist() == ram_exp, (c, n, w)
            ae_exp, s = [], 0
            while s < n:
                s = s + w + 1 if s + w < min(n, s + mx) else min(n, s + mx)
                ae_exp.append(s)
            assert orc.chunk("ae", B, w, mn, mx).tolist() == ae_exp, (c, n, w)
            mp = list(range(mx, n, mx)) + [n]
            assert orc.chunk("maxp", B, w, mn, mx).tolist() == mp
    # Strictly increasing ramp: RAM cuts every w+1 bytes (the byte after the
    # window always exceeds it); AE and MAXP never find a cut, so max applies.
    B = np.arange(200, dtype=np.uint8)
    w, mn, mx = 5, 1, 17
    ram, s = [], 0
    while s < 200:
        s = 200 if 200 - s <= w else s + w + 1
        ram.append(s)
    assert orc.chunk("ram", B, w, mn, mx).tolist() == ram
    assert orc.chunk("ae", B, w, mn, mx).tolist() == list(range(mx, 200, mx)) + [200]
    assert orc.chunk("maxp", B, w, mn, mx).tolist() == list(range(mx, 200, mx)) + [200]
    # Single spike in zeros: MAXP cuts right after it exactly when both
    # windows fit and the size is within [min, max].
    n, w = 40, 3
    for i in range(n):
        B = np.zeros(n, dtype=np.uint8)
        B[i] = 9
        # the only target is i itself, when both windows fit
        T = [i] if w <= i <= n - 1 - w else []
        for (mn, mx) in ((1, 100), (6, 100), (1, 12)):
            exp, s = [], 0
            while s < n:
                s = brute.maxp_next([0] * n, s, w, mn, mx, targets=T)
                exp.append(s)
            got = orc.chunk("maxp", B, w, mn, mx).tolist()
            assert got == exp, (i, mn, mx, got, exp)


def check_uniform_statistics(orc, n=1 << 22, seed=7):
    """Closed forms on i.i.d. uniform bytes (within 4 standard errors).

    RAM and AE, large w: the window maximum (or the first target to reach
    it) is 255 with probability ~1, the scan for a byte >= 255 is geometric
    with p = 1/256, so the mean chunk is w + 1 + 255.
    MAXP: a position is a target with probability
    (1/256) * sum_v (v/256)^(2w) (all 2w neighbours strictly below it)."""
    import synth
    B = synth.uniform(seed, n)
    w, mn, mx = 3000, 64, 1 << 20
    for alg in ("ram", "ae"):
        b = orc.chunk(alg, B, w, mn, mx)
        sizes = np.diff(np.concatenate([[0], b[:-1].astype(np.int64)]))
        mean, expect = sizes.mean(), w + 256
        sd = math.sqrt(255 * 256)  # geometric(1/256) standard deviation
        assert abs(mean - expect) < 4 * sd / math.sqrt(len(sizes)), (alg, mean, expect)
    for w in (4, 60, 300):
        p = sum((v / 256.0) ** (2 * w) for v in range(256)) / 256.0
        m = n - 2 * w
        exp = m * p
        got = len(orc.maxp_targets(B, w))
        # targets within distance w exclude each other, so the count is at
        # most binomial in spread; 5 sigma of the binomial bounds it loosely
        assert abs(got - exp) < 5 * math.sqrt(exp) + 2, (w, got, exp)


def check_invariants(orc, seed=5):
    import synth
    rng = np.random.default_rng(seed)
    data = [synth.uniform(11, 300_000), synth.mixed(12, 3 << 20)[1 << 20:(1 << 20) + 400_000],
            np.zeros(50_000, dtype=np.uint8)]
    for B in data:
        for alg, w in (("ram", 700), ("ae", 700), ("ae_min", 700), ("maxp", 90)):
            mn, mx = 256, 4096
            b = orc.chunk(alg, B, w, mn, mx).astype(np.int64)
            assert b[-1] == B.size and np.all(np.diff(b) > 0)
            sizes = np.diff(np.concatenate([[0], b]))
            assert sizes.max() <= mx
            assert sizes[:-1].min() >= mn
    # AE-Min on B equals AE-Max on 255 - B.
    B = rng.integers(0, 256, size=200_000).astype(np.uint8)
    for w in (1, 5, 300):
        a = orc.chunk("ae_min", B, w, 2, 5000)
        b = orc.chunk("ae", (255 - B).astype(np.uint8), w, 2, 5000)
        assert np.array_equal(a, b)


def check_edit_locality(orc, seed=21):
    """A single edit at position p leaves every boundary at or before p - w
    untouched (next(s) reads only bytes below the cut, plus w bytes beyond it
    for MAXP), and after the first common start past the edit the two
    boundary lists agree up to the length change."""
    import synth
    B = synth.uniform(seed, 200_000)
    rng = np.random.default_rng(seed)
    for alg, w in (("ram", 900), ("ae", 900), ("maxp", 120)):
        mn, mx = 128, 8192
        old = orc.chunk(alg, B, w, mn, mx).astype(np.int64)
        for kind in ("insert", "delete", "overwrite"):
            p = int(rng.integers(20_000, 180_000))
            L = int(rng.integers(1, 513))
            ins = rng.integers(0, 256, size=L).astype(np.uint8)
            if kind == "insert":
                N = np.concatenate([B[:p], ins, B[p:]]); delta = L
            elif kind == "delete":
                N = np.concatenate([B[:p], B[p + L:]]); delta = -L
            else:
                N = np.concatenate([B[:p], ins, B[p + L:]]); delta = 0
            new = orc.chunk(alg, N, w, mn, mx).astype(np.int64)
            lim = p - w
            assert np.array_equal(old[old <= lim], new[new <= lim]), (alg, kind)
            # resync: first new boundary past the edit that is an old
            # boundary shifted by delta; from there on the lists agree.
            edit_end = p + max(L, 0) + w
            old_set = set((old + delta).tolist())
            k = next((i for i, x in enumerate(new) if x > edit_end and x in old_set), None)
            assert k is not None, (alg, kind, "no resync")
            j = int(np.searchsorted(old + delta, new[k]))
            assert np.array_equal(new[k:], old[j:] + delta), (alg, kind)


ALL_PINS = (check_hand_examples, check_brute_small, check_alternative_forms,
            check_closed_forms, check_invariants, check_edit_locality)
