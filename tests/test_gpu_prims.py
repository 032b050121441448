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
    scan loop exactly (RAM, AE-Max, AE-Min, MAXP; several windows; mixed,
    uniform and low-alphabet bytes)."""
    import paper_2508_05797_gb300 as pkg
    from paper_2508_05797_gb300.cdc import CdcError, ERR_INVALID
    rng = np.random.default_rng(offset)
    for data in (synth.mixed_range(12, 64 << 20, 7 << 20, 6 << 20), synth.uniform(13, (1 << 20) + 77),
                 rng.integers(0, 3, size=300_001).astype(np.uint8)):
        d = to_device(data, offset)
        for alg, w, mn, mx in (("ram", 7936, 2048, 65536), ("ram", 100, 500, 3000), ("ae", 7000, 2048, 65536),
                               ("ae", 64, 32, 700), ("ae_min", 3000, 1024, 20000), ("maxp", 291, 2048, 65536),
                               ("maxp", 63, 1, 3000), ("maxp", 7, 40, 300), ("maxp", 1000, 1, 5000)):
            b = pkg.chunk(d, alg, w, mn, mx)
            assert pkg.byte_shares(d, b, alg, w, mn, mx) == oracle.byte_shares(alg, data, w, mn, mx), (alg, w)
    with pytest.raises(CdcError) as ei:
        pkg.byte_shares(d, pkg.chunk(d, "ae", 300, 200, 65536), "ae", 300, 400, 65536)
    assert ei.value.status == ERR_INVALID


def _host_hist(bounds, width, n_bins):
    sizes = np.diff(np.concatenate([[0], np.asarray(bounds, dtype=np.int64)]))
    return np.bincount(np.minimum(sizes // width, n_bins - 1), minlength=n_bins)


def test_size_histogram_equals_oracle_sizes():
    """The device chunk-size histogram of each algorithm's boundaries equals
    the histogram of the oracle's chunk sizes counted on the host (the size
    CDF is its running sum over the chunk count)."""
    import torch
    import paper_2508_05797_gb300 as pkg
    from gpu_util import params
    data = synth.mixed_range(1, 4 << 30, 0, 24 << 20)
    d = torch.from_numpy(data).cuda()
    for alg in ("ram", "ae", "ae_min", "maxp"):
        w, mn, mx = params("mixed_4g_seed1", "ae" if alg == "ae_min" else alg, 8192)
        exp = oracle.chunk(alg, data, w, mn, mx)
        b = pkg.chunk(d, alg, w, mn, mx)
        for width, n_bins in ((1024, 64), (4096, 17), (1, 8192), (1 << 20, 3)):
            h = pkg.size_histogram(b, width, n_bins).cpu().numpy()
            assert np.array_equal(h, _host_hist(exp, width, n_bins)), (alg, width, n_bins)


def test_size_histogram_edges():
    import torch
    import paper_2508_05797_gb300 as pkg
    from paper_2508_05797_gb300.cdc import CdcError, ERR_INVALID
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert pkg.size_histogram(empty, 100, 5).cpu().tolist() == [0] * 5
    b = torch.tensor([1, 1, 101, 5000, 5000 + (1 << 40)], dtype=torch.int64, device="cuda")
    assert pkg.size_histogram(b, 100, 4).cpu().tolist() == [2, 1, 0, 2]
    assert pkg.size_histogram(b, 1 << 50, 1).cpu().tolist() == [5]
    for width, n_bins in ((0, 4), (100, 0), (100, 8193)):
        with pytest.raises(CdcError) as ei:
            pkg.size_histogram(b, width, n_bins)
        assert ei.value.status == ERR_INVALID
