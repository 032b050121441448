"""Brute-force statements of the chunk rules, for tiny inputs only.

Each rule is written as "the smallest admissible cut position", evaluated
from scratch for every candidate (O(n^2) or worse). This is a different
formulation from the oracle's single forward scan, so an index, sign or
comparator slip in either one shows up as a disagreement.

Sources (arxiv 2508.05797): Section 2.1 (AE, MAXP and RAM paragraphs) and
Section 3.3 for the rules; Section 2.1 (hash-based paragraph) for min / max.
"""
from __future__ import annotations


def ram_next(B, s, w, mn, mx):
    """RAM: cut e is admissible when byte e-1 lies at or beyond the w-byte
    window at s, is >= the window maximum, and the size e-s is within
    [min, max]; with no admissible cut the chunk is forced to min(len, s+max).
    When at most w bytes remain, they form the last chunk."""
    n = len(B)
    if n - s <= w:
        return n
    M = max(B[s:s + w])
    forced = min(n, s + mx)
    admissible = [e for e in range(s + 1, n + 1)
                  if e - 1 >= s + w and mn <= e - s <= mx and B[e - 1] >= M]
    return min(admissible + [forced])


def ram_next_weak_record(B, s, w, mn, mx):
    """RAM restated without the window maximum (valid when min - 1 <= w): the
    cut follows the first byte at or beyond s+w that no earlier byte of the
    chunk exceeds."""
    n = len(B)
    assert mn - 1 <= w
    if n - s <= w:
        return n
    forced = min(n, s + mx)
    for j in range(s + w, forced):
        if all(B[k] <= B[j] for k in range(s, j)):
            return j + 1
    return forced


def ae_next(B, s, w, mn, mx, direction=+1):
    """AE: position i ends the chunk (cut i+1) when B[i] is not beyond the
    extreme of B[s:i], the first position holding that extreme is at least w
    before i, and the chunk has at least min bytes."""
    n = len(B)
    forced = min(n, s + mx)
    sign = 1 if direction > 0 else -1
    for i in range(s + 1, forced):
        prefix = [sign * b for b in B[s:i]]
        m = max(prefix)
        p = s + prefix.index(m)
        if sign * B[i] <= m and i - p >= w and i + 1 - s >= mn:
            return i + 1
    return forced


def ae_next_records(B, s, w, mn, mx):
    """AE-Max restated over targets (valid when min <= w + 1): the targets
    from s are s and every later byte greater than all before it; the cut is
    p+w+1 for the first target p whose next w bytes hold nothing greater."""
    n = len(B)
    assert mn <= w + 1
    forced = min(n, s + mx)
    for p in range(s, forced):
        is_target = p == s or B[p] > max(B[s:p])
        if not is_target:
            continue
        if p + w < forced and all(B[k] <= B[p] for k in range(p + 1, p + w + 1)):
            return p + w + 1
    return forced


def maxp_targets(B, w):
    """All positions strictly greater than every byte within distance w on
    both sides, with both windows inside the data."""
    n = len(B)
    out = []
    for i in range(n):
        if i - w < 0 or i + w > n - 1:
            continue
        if all(B[k] < B[i] for k in range(i - w, i + w + 1) if k != i):
            out.append(i)
    return out


def maxp_next(B, s, w, mn, mx, targets=None):
    n = len(B)
    T = maxp_targets(B, w) if targets is None else targets
    forced = min(n, s + mx)
    cuts = [c + 1 for c in T if c + 1 - s >= mn and c + 1 <= forced]
    return min(cuts + [forced])


def next_cut(alg, B, s, w, mn, mx, targets=None):
    if alg == "ram":
        return ram_next(B, s, w, mn, mx)
    if alg in ("ae", "ae_max"):
        return ae_next(B, s, w, mn, mx, +1)
    if alg == "ae_min":
        return ae_next(B, s, w, mn, mx, -1)
    if alg == "maxp":
        return maxp_next(B, s, w, mn, mx, targets)
    raise ValueError(alg)


def chunk(alg, B, w, mn, mx):
    B = [int(x) for x in B]
    targets = maxp_targets(B, w) if alg == "maxp" else None
    out, s = [], 0
    while s < len(B):
        s = next_cut(alg, B, s, w, mn, mx, targets)
        out.append(s)
    return out
