"""CPU oracle for hashless CDC (RAM, AE-Max, AE-Min, MAXP).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the library's product path never
does. It is the plain sequential statement of the chunkers in ``oracle.c``
(arxiv 2508.05797, Section 2.1 and Section 3.3), compiled with gcc on first
use and called through ctypes. It shares no code with the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_libs: dict = {}

RAM, AE, MAXP, AE_MIN = 0, 1, 2, 3
ALGS = {"ram": RAM, "ae": AE, "ae_max": AE, "maxp": MAXP, "ae_min": AE_MIN}


def alg_id(alg) -> int:
    return ALGS[alg.lower()] if isinstance(alg, str) else int(alg)


def build(src: str = _SRC, out: str = _LIB_PATH, force: bool = False) -> str:
    """Compile an oracle source file into a shared library; returns its path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", src, "-o", tmp])
    os.replace(tmp, out)
    return out


class Oracle:
    """ctypes view of one compiled oracle library (the real one by default)."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.oracle_next.argtypes = [i32, vp, u64, u64, u32, u32, u32]
        lib.oracle_next.restype = u64
        lib.oracle_chunk.argtypes = [i32, vp, u64, u32, u32, u32, vp, u64]
        lib.oracle_chunk.restype = u64
        lib.oracle_maxp_is_target.argtypes = [vp, u64, u64, u32]
        lib.oracle_maxp_is_target.restype = i32
        lib.oracle_maxp_targets.argtypes = [vp, u64, u32, vp, u64]
        lib.oracle_maxp_targets.restype = u64
        lib.oracle_ebs.argtypes = [i32, vp, u64, u64, u64, ctypes.POINTER(u64)]
        lib.oracle_ebs.restype = u32
        lib.oracle_byte_shares.argtypes = [i32, vp, u64, u32, u32, u32, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        lib.oracle_byte_shares.restype = i32
        lib.oracle_rs.argtypes = [i32, vp, u64, u64, u64, u32]
        lib.oracle_rs.restype = u64
        self.lib = lib

    @staticmethod
    def _buf(data) -> np.ndarray:
        a = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8)
                                 if isinstance(data, (bytes, bytearray)) else data, dtype=np.uint8)
        return a

    def next(self, alg, data, s: int, w: int, mn: int, mx: int) -> int:
        a = self._buf(data)
        return int(self.lib.oracle_next(alg_id(alg), a.ctypes.data, a.size, s, w, mn, mx))

    def count(self, alg, data, w: int, mn: int, mx: int) -> int:
        a = self._buf(data)
        return int(self.lib.oracle_chunk(alg_id(alg), a.ctypes.data, a.size, w, mn, mx, None, 0))

    def chunk(self, alg, data, w: int, mn: int, mx: int) -> np.ndarray:
        """Boundaries (chunk ends, increasing, last == len) of the whole buffer."""
        a = self._buf(data)
        if a.size == 0:
            return np.zeros(0, dtype=np.uint64)
        cap = a.size // max(mn, 1) + 2
        if cap > (1 << 26):
            n = self.count(alg, a, w, mn, mx)
            cap = n
        out = np.empty(cap, dtype=np.uint64)
        n = int(self.lib.oracle_chunk(alg_id(alg), a.ctypes.data, a.size, w, mn, mx,
                                      out.ctypes.data, cap))
        assert n <= cap
        return out[:n].copy()

    def is_target(self, data, i: int, w: int) -> bool:
        a = self._buf(data)
        return bool(self.lib.oracle_maxp_is_target(a.ctypes.data, a.size, i, w))

    def maxp_targets(self, data, w: int) -> np.ndarray:
        a = self._buf(data)
        cap = a.size // (w + 1) + 2
        out = np.empty(cap, dtype=np.uint64)
        n = int(self.lib.oracle_maxp_targets(a.ctypes.data, a.size, w, out.ctypes.data, cap))
        assert n <= cap
        return out[:n].copy()


    def ebs(self, op, data, a: int, b: int):
        """(extreme byte, offset of its first occurrence) of data[a:b]; op 'max' or 'min'."""
        arr = self._buf(data)
        pos = ctypes.c_uint64()
        v = self.lib.oracle_ebs(EBS_OPS[op], arr.ctypes.data if arr.size else None, arr.size, a, b,
                                ctypes.byref(pos))
        return int(v), int(pos.value)

    def rs(self, cmp, data, a: int, b: int, t: int) -> int:
        """First offset in [a, b) whose byte compares true against t, else b."""
        arr = self._buf(data)
        return int(self.lib.oracle_rs(RS_CMPS[cmp], arr.ctypes.data if arr.size else None, arr.size, a, b, t))

    def byte_shares(self, alg, data, w: int, mn: int, mx: int):
        """(bytes read by Extreme Byte Searches, bytes read by Range Scans)
        while the whole buffer is chunked, as Section 3.3 composes the
        algorithms; None for AE with min > w + 1 (undefined there). The MAXP
        procedure checks each of its cuts against next() and raises if one
        differs."""
        a = self._buf(data)
        e, r = ctypes.c_uint64(0), ctypes.c_uint64(0)
        st = self.lib.oracle_byte_shares(alg_id(alg), a.ctypes.data if a.size else None, a.size, w, mn, mx,
                                         ctypes.byref(e), ctypes.byref(r))
        if st == -2:
            raise AssertionError("MAXP share procedure cut differs from next()")
        return None if st else (int(e.value), int(r.value))

    def horizon(self, alg, w: int, mx: int) -> int:
        """Bytes after a chunk start s that decide the chunk from s: RAM and AE
        never look at or past s + max (the forced cut, Section 2.1); a MAXP
        target also needs its w right neighbours (Section 2.1), so max + w."""
        return mx + (w if alg_id(alg) == MAXP else 0)

    def chunk_pieces(self, alg, pieces, w: int, mn: int, mx: int, horizon: int | None = None) -> list:
        """The stream chunked while it arrives piece by piece (the last piece
        ends it). For each piece: the chunk ends (offsets from the stream
        start) that the bytes received so far settle, i.e. those of the
        chunks whose start s has s + horizon <= bytes received; the last
        piece adds the rest, up to the stream's length. Each chunk is one step
        s -> next(s) of the sequential loop (Section 3.3) over the bytes
        received so far. `horizon` overrides the rule's horizon (tests plant
        a wrong one)."""
        H = self.horizon(alg, w, mx) if horizon is None else horizon
        buf = np.zeros(0, dtype=np.uint8)
        s, out = 0, []
        for i, piece in enumerate(pieces):
            buf = np.concatenate([buf, self._buf(piece)])
            L = buf.size
            final = i == len(pieces) - 1
            ends = []
            while s < L and (final or s + H <= L):
                s = self.next(alg, buf, s, w, mn, mx)
                ends.append(s)
            out.append(np.array(ends, dtype=np.uint64))
        return out


EBS_OPS = {"max": 0, "min": 1}
RS_CMPS = {"gt": 0, "lt": 1, "geq": 2, "leq": 3, "eq": 4}


def get(lib_path: str | None = None) -> Oracle:
    """The oracle (compiled on first use) or a given compiled variant."""
    path = lib_path or _LIB_PATH
    with _lock:
        if path not in _libs:
            if lib_path is None:
                build()
            _libs[path] = Oracle(path)
        return _libs[path]


def chunk(alg, data, w: int, mn: int, mx: int) -> np.ndarray:
    return get().chunk(alg, data, w, mn, mx)


def count(alg, data, w: int, mn: int, mx: int) -> int:
    return get().count(alg, data, w, mn, mx)


def next_cut(alg, data, s: int, w: int, mn: int, mx: int) -> int:
    return get().next(alg, data, s, w, mn, mx)


def maxp_targets(data, w: int) -> np.ndarray:
    return get().maxp_targets(data, w)


def chunk_pieces(alg, pieces, w: int, mn: int, mx: int, horizon: int | None = None) -> list:
    return get().chunk_pieces(alg, pieces, w, mn, mx, horizon)


def byte_shares(alg, data, w: int, mn: int, mx: int):
    return get().byte_shares(alg, data, w, mn, mx)
