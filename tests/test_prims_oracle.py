"""The oracle's Extreme Byte Search and Range Scan (Section 3.1, 3.2) against
numpy: maximum / minimum and first occurrence (numpy argmax / argmin return
the first), and the first position matching each of the five comparators."""
import numpy as np
import pytest

import oracle

CMP = {"gt": np.greater, "lt": np.less, "geq": np.greater_equal, "leq": np.less_equal, "eq": np.equal}


@pytest.mark.parametrize("hi", [2, 7, 256])
def test_ebs_matches_numpy(hi):
    rng = np.random.default_rng(hi)
    orc = oracle.get()
    data = rng.integers(0, hi, size=5000).astype(np.uint8)
    for _ in range(400):
        a = int(rng.integers(0, data.size))
        b = int(rng.integers(a, data.size + 40))
        seg = data[a:min(b, data.size)]
        for op in ("max", "min"):
            v, p = orc.ebs(op, data, a, b)
            if seg.size == 0:
                assert (v, p) == ((0 if op == "max" else 255), a)
            else:
                idx = int(np.argmax(seg) if op == "max" else np.argmin(seg))
                assert v == int(seg[idx]) and p == a + idx


@pytest.mark.parametrize("cmp", sorted(CMP))
def test_rs_matches_numpy(cmp):
    rng = np.random.default_rng(len(cmp))
    orc = oracle.get()
    data = rng.integers(0, 256, size=4000).astype(np.uint8)
    data[100:300] = 0
    data[300:400] = 255
    for _ in range(500):
        a = int(rng.integers(0, data.size))
        b = int(rng.integers(a, data.size + 40))
        t = int(rng.choice([0, 1, 254, 255, int(rng.integers(0, 256))]))
        seg = data[a:min(b, data.size)]
        hits = np.nonzero(CMP[cmp](seg.astype(np.int32), t))[0]
        want = a + int(hits[0]) if hits.size else b
        assert orc.rs(cmp, data, a, b, t) == want, (cmp, a, b, t)
