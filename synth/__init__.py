"""Seeded synthetic inputs for the hashless CDC workloads (host side).

The byte streams are written by ``synth.c`` (SplitMix64 in counter form; see
its header). This module compiles it on first use, wraps it with ctypes and
returns numpy arrays. It contains no chunking arithmetic: the oracle and the
GPU path both consume what it produces.

Workloads (the paper's datasets are not available; these stand in for them):

* ``uniform(seed, n)``             -- i.i.d. uniform bytes (16 MiB, seed 0 is
  the single-buffer RAM workload).
* ``mixed(seed, n)``               -- 1 MiB blocks: 50% uniform, 30% text-like
  (Zipf s=1.1 over 64 symbols mapped to 0x20..0x5F), 20% zero runs of
  4-64 KiB each closed by one non-zero byte; seeded block order.
* ``versions(seed_base, n, k)``    -- a uniform base plus k versions, each
  with about 0.1% of its bytes edited by insert / delete / overwrite runs.
* ``lognormal_sizes(...)``         -- file or request sizes.
* ``poisson_arrivals(...)``        -- request arrival times.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None

MIB = 1 << 20
GIB = 1 << 30


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to it; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                           "-pthread", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u64, i32, vp, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
        lib.synth_rand.argtypes = [u64, u64]
        lib.synth_rand.restype = u64
        lib.synth_key.argtypes = [u64, u64, u64]
        lib.synth_key.restype = u64
        lib.synth_uniform.argtypes = [u64, u64, vp, u64, i32]
        lib.synth_uniform.restype = None
        lib.synth_mixed.argtypes = [u64, vp, u64, i32]
        lib.synth_mixed.restype = None
        lib.synth_mixed_range.argtypes = [u64, u64, u64, u64, vp, i32]
        lib.synth_mixed_range.restype = None
        lib.synth_mixed_types.argtypes = [u64, u64, vp]
        lib.synth_mixed_types.restype = None
        lib.synth_edit_count.argtypes = [u64, u64]
        lib.synth_edit_count.restype = u64
        lib.synth_edit_bound.argtypes = [u64, u64]
        lib.synth_edit_bound.restype = u64
        lib.synth_edit.argtypes = [u64, vp, u64, u64, vp]
        lib.synth_edit.restype = u64
        lib.synth_lognormal_sizes.argtypes = [u64, u64, dbl, dbl, u64, u64, vp]
        lib.synth_lognormal_sizes.restype = None
        lib.synth_poisson_arrivals.argtypes = [u64, u64, dbl, vp]
        lib.synth_poisson_arrivals.restype = None
        lib.synth_choice.argtypes = [u64, u64, ctypes.c_uint32, vp]
        lib.synth_choice.restype = None
        _lib = lib
        return lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def uniform(seed: int, n: int, offset: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """Bytes [offset, offset+n) of the uniform stream of ``seed``."""
    lib = _load()
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= n and out.flags.c_contiguous
    lib.synth_uniform(seed, offset, _ptr(out), n, _threads())
    return out


def mixed(seed: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """The mixed (random / text-like / zero-run) stream of ``n`` bytes."""
    lib = _load()
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= n and out.flags.c_contiguous
    lib.synth_mixed(seed, _ptr(out), n, _threads())
    return out


def mixed_range(seed: int, total: int, lo: int, n: int, out: np.ndarray | None = None) -> np.ndarray:
    """Bytes [lo, lo+n) of the mixed stream of total length ``total`` (the
    block order depends on the total length, so a prefix of the 4 GiB stream
    is ``mixed_range(seed, 4 << 30, 0, n)``, not ``mixed(seed, n)``)."""
    lib = _load()
    if out is None:
        out = np.empty(n, dtype=np.uint8)
    assert out.dtype == np.uint8 and out.size >= n and out.flags.c_contiguous
    assert lo + n <= total
    lib.synth_mixed_range(seed, total, lo, n, _ptr(out), _threads())
    return out


def mixed_types(seed: int, n: int) -> np.ndarray:
    """Block type per 1 MiB block of ``mixed(seed, n)``: 0 random, 1 text, 2 zero."""
    lib = _load()
    nb = (n + MIB - 1) // MIB
    t = np.empty(max(nb, 1), dtype=np.uint8)
    lib.synth_mixed_types(seed, n, _ptr(t))
    return t[:nb]


def edit(seed: int, base: np.ndarray, frac_ppm: int = 1000) -> np.ndarray:
    """A version of ``base`` with about frac_ppm/1e6 of its bytes edited."""
    lib = _load()
    base = np.ascontiguousarray(base, dtype=np.uint8)
    n_edits = lib.synth_edit_count(base.size, frac_ppm)
    out = np.empty(lib.synth_edit_bound(base.size, n_edits), dtype=np.uint8)
    m = lib.synth_edit(seed, _ptr(base), base.size, n_edits, _ptr(out))
    return out[:m]


def versions(seed_base: int, n: int, k: int, frac_ppm: int = 1000, edit_seed0: int = 100):
    """A uniform base of n bytes (seed ``seed_base``) and k successive versions;
    version v is ``edit(edit_seed0 + v, version v-1)``."""
    vs = [uniform(seed_base, n)]
    for v in range(1, k + 1):
        vs.append(edit(edit_seed0 + v, vs[-1], frac_ppm))
    return vs


def lognormal_sizes(seed: int, n: int, median: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    lib = _load()
    out = np.empty(max(n, 1), dtype=np.uint64)
    lib.synth_lognormal_sizes(seed, n, float(median), float(sigma), lo, hi, _ptr(out))
    return out[:n]


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    lib = _load()
    out = np.empty(max(n, 1), dtype=np.float64)
    lib.synth_poisson_arrivals(seed, n, float(rate), _ptr(out))
    return out[:n]


def choice(seed: int, n: int, k: int) -> np.ndarray:
    lib = _load()
    out = np.empty(max(n, 1), dtype=np.uint32)
    lib.synth_choice(seed, n, k, _ptr(out))
    return out[:n]


def files_arena(seed: int, n_files: int, median: int = 64 * 1024, sigma: float = 1.5,
                lo: int = 1, hi: int = 256 * MIB, content: str = "mixed"):
    """Files with log-normal sizes packed back to back in one arena.

    Returns (arena bytes, offsets[n_files + 1])."""
    sizes = lognormal_sizes(seed, n_files, median, sigma, lo, hi)
    off = np.zeros(n_files + 1, dtype=np.uint64)
    np.cumsum(sizes, out=off[1:])
    total = int(off[-1])
    arena = mixed(seed, total) if content == "mixed" else uniform(seed, total)
    return arena, off
