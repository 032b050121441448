"""Chunking one stream split over several ranks: each rank builds its
shard's exit table on its own, one (exit, count) hand-off per shard edge
composes them, and each rank then writes its own boundaries at the global
offset. Run as two gloo processes on CPU with the host build of the
candidate-graph rules (graph_logic.cuh), against the oracle's whole-stream
chunker.

A chain only ever leaves one chunk and enters the next at a candidate
position (or at a forced cut or in a quiet run, which F steps over), so a
shard's table maps every candidate inside the shard to the first candidate
its chain reaches past the shard end and the number of chunk ends on the way.
Rank r needs rank r-1's exit to know where the true chain enters its shard;
that entry is one of its table's candidates (or lies beyond the shard)."""
import ctypes
import os
import socket

import numpy as np
import pytest

import hostcheck
import oracle
import synth

CASES = [("ram", 700, 128, 8192), ("ae", 700, 128, 8192), ("maxp", 150, 512, 8192)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    return np.concatenate([synth.uniform(41, 120_000), synth.mixed_range(1, 4 << 30, 6 << 20, 100_000),
                           synth.mixed_range(1, 4 << 30, 1 << 20, 80_000)])  # random, text-like, zero runs


def _shard_table(alg, w, mn, mx, data, a, b):
    """{candidate position in (a, b], and a itself if it is the stream start:
    (position of the first candidate past b on its chain, or len; chunk ends
    up to it)} -- computed from this shard's candidates only."""
    from test_chain_logic_host import Arena, _superblocks
    from test_graph_logic_host import _lib_args, expected_cands
    lib = hostcheck.load()
    lo = 0
    ar = Arena(data, lo, alg, w)
    sup = _superblocks(ar, alg)
    args = _lib_args(ar, sup, alg, w, mn, mx, lo, lo + data.size)
    cands = expected_cands(alg, data, w)
    mine = [int(y) for y in cands if a < y <= b]
    if a == 0:
        mine = [0] + mine
    table = {}
    c = ctypes.c_uint32()
    for y in mine:
        pos, ends = y, 0
        while pos <= b and pos < data.size:  # F steps until past the shard
            pos = int(lib.hc_cand_next(*args, pos, ctypes.byref(c)))
            ends += c.value
        table[y] = (min(pos, data.size), ends)
    return table


def _worker(rank, world, port, alg, w, mn, mx, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    data = _data()
    n = data.size
    edges = [n * r // world for r in range(world + 1)]
    a, b = edges[rank], edges[rank + 1]
    table = _shard_table(alg, w, mn, mx, data, a, b)  # no communication
    # the hand-off: (entry position, chunk ends before it) from the left neighbour
    msg = torch.zeros(2, dtype=torch.int64)
    if rank > 0:
        dist.recv(msg, src=rank - 1)
        entry, before = int(msg[0]), int(msg[1])
    else:
        entry, before = 0, 0
    if entry <= b and entry < n:
        assert entry in table, (rank, entry)  # the chain enters the shard at one of its candidates
        ex, ends = table[entry]
    else:
        ex, ends = entry, 0  # the chain jumps over this shard
    if rank + 1 < world:
        dist.send(torch.tensor([ex, before + ends], dtype=torch.int64), dst=rank + 1)
    # this rank's boundaries, from the entry up to the exit, at the global offset `before`
    out, s = [], entry
    while s < ex:
        s = oracle.get().next(alg, data, s, w, mn, mx)
        out.append(s)
    np.save(os.path.join(out_dir, "r%d.npy" % rank), np.array([before] + out, dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("alg,w,mn,mx", CASES)
def test_two_shards_compose_to_the_whole_chain(tmp_path, alg, w, mn, mx):
    import torch.multiprocessing as mp
    hostcheck.load()  # build once, before the workers
    port = _free_port()
    mp.spawn(_worker, args=(2, port, alg, w, mn, mx, str(tmp_path)), nprocs=2, join=True)
    exp = oracle.chunk(alg, _data(), w, mn, mx).astype(np.int64)
    got, offset = [], 0
    for r in range(2):
        rec = np.load(tmp_path / ("r%d.npy" % r))
        assert rec[0] == offset, (r, rec[0], offset)  # the composed count is the global offset
        got.extend(rec[1:].tolist())
        offset += rec.size - 1
    assert np.array_equal(np.array(got, dtype=np.int64), exp)
