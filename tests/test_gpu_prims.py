"""cdc_ebs / cdc_rs on the GPU against the oracle's plain loops: every
comparator and both extremes, thresholds at the ends of the byte range,
empty, short, long and out-of-range ranges, and misaligned data."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_device

pytestmark = pytest.mark.gpu


def _ranges(rng, n, size):
    a = rng.integers(0, size, size=n)
    kind = rng.integers(0, 4, size=n)
    ln = np.where(kind == 0, 0, np.where(kind == 1, rng.integers(1, 40, size=n),
                                         np.where(kind == 2, rng.integers(40, 3000, size=n),
                                                  rng.integers(3000, 20000, size=n))))
    b = a + ln
    b[::37] = size + 50  # past the end: clipped
    return np.stack([a, b], axis=1).astype(np.int64)


@pytest.mark.parametrize("offset", [0, 5, 13])
def test_ebs_and_rs_match_oracle(offset):
    import torch
    import paper_2508_05797_gb300 as pkg
    rng = np.random.default_rng(offset)
    orc = oracle.get()
    n = 60_000
    datasets = [synth.uniform(offset, n), synth.mixed_range(2, 4 << 30, 5 << 20, n),
                rng.integers(0, 3, size=n).astype(np.uint8)]
    for data in datasets:
        d = to_device(data, offset)
        r = _ranges(rng, 1500, n)
        dr = torch.from_numpy(r).cuda()
        for op in ("max", "min"):
            v, p = pkg.ebs(d, dr, op)
            v, p = v.cpu().numpy(), p.cpu().numpy()
            for i in range(r.shape[0]):
                ev, ep = orc.ebs(op, data, int(r[i, 0]), int(r[i, 1]))
                assert (int(v[i]), int(p[i])) == (ev, ep), (op, i, r[i])
        thr = rng.integers(0, 256, size=r.shape[0]).astype(np.uint8)
        thr[::11] = 0
        thr[5::11] = 255
        dt = torch.from_numpy(thr).cuda()
        for cmp in ("gt", "lt", "geq", "leq", "eq"):
            p = pkg.rs(d, dr, dt, cmp).cpu().numpy()
            for i in range(r.shape[0]):
                e = orc.rs(cmp, data, int(r[i, 0]), int(r[i, 1]), int(thr[i]))
                assert int(p[i]) == e, (cmp, i, r[i], int(thr[i]))


def test_empty_inputs():
    import torch
    import paper_2508_05797_gb300 as pkg
    d = torch.zeros(0, dtype=torch.uint8, device="cuda")
    r = torch.tensor([[0, 10], [3, 3]], dtype=torch.int64, device="cuda")
    v, p = pkg.ebs(d, r, "min")
    assert v.cpu().tolist() == [255, 255] and p.cpu().tolist() == [0, 3]
    q = pkg.rs(d, r, torch.tensor([0, 0], dtype=torch.uint8, device="cuda"), "geq")
    assert q.cpu().tolist() == [10, 3]


@pytest.mark.parametrize("offset", [0, 3])
def test_byte_shares_match_oracle(offset):
    """cdc_byte_shares over the GPU's boundaries equals the oracle's search /
    scan loop exactly (RAM, AE-Max, AE-Min; several windows)."""
    import paper_2508_05797_gb300 as pkg
    from paper_2508_05797_gb300.cdc import CdcError, ERR_INVALID
    data = synth.mixed_range(12, 64 << 20, 7 << 20, 6 << 20)
    d = to_device(data, offset)
    for alg, w, mn, mx in (("ram", 7936, 2048, 65536), ("ram", 100, 500, 3000), ("ae", 7000, 2048, 65536),
                           ("ae", 64, 32, 700), ("ae_min", 3000, 1024, 20000)):
        b = pkg.chunk(d, alg, w, mn, mx)
        assert pkg.byte_shares(d, b, alg, w, mn, mx) == oracle.byte_shares(alg, data, w, mn, mx), (alg, w)
    with pytest.raises(CdcError) as ei:
        pkg.byte_shares(d, pkg.chunk(d, "maxp", 300, 2048, 65536), "maxp", 300, 2048, 65536)
    assert ei.value.status == ERR_INVALID
