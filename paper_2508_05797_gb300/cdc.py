"""ctypes binding of libcdc.so (include/cdc.h) with torch tensors for device memory.

Argument marshalling only: every step of chunking runs in the CUDA library.
If the library cannot be built or loaded, every call raises; there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

ALGS = {"ram": 0, "ae": 1, "ae_max": 1, "maxp": 2, "ae_min": 3}
OPT_SEGMENT, OPT_SPAN, OPT_TIMEOUT_MS, OPT_FORCE_BYTES, OPT_DEBUG_HOLD_ITEM = range(5)
OPT_PROFILE = 5
OPT_STATS = 6
OPT_WARP_CHAINS = 7
OPT_STARTS = 8
OPT_PIPELINE = 9        # 0 automatic, 1 speculative segments, 2 candidate graph
OPT_GRAPH_SEGMENT = 10
OPT_GRAPH_SLOTS = 11
PIPE_AUTO, PIPE_SPECULATE, PIPE_GRAPH = 0, 1, 2
STAT_NAMES = ["segments", "thread_steps", "warp_steps", "merges", "stitch_walks", "stitch_steps", "unknown",
              "hash_full", "scan_follows", "out_steps", "empty", "survivors", "cyc_setup", "cyc_threads",
              "cyc_warps", "cyc_stitch", "rounds", "cyc_rounds", "cyc_surv", "stitch_long", "stitch_maxw",
              "out_passes", "out_recs", "cyc_output", "cyc_out_steps"]
STATUS = ["CDC_OK", "CDC_ERR_INVALID", "CDC_ERR_CAPACITY", "CDC_ERR_CUDA", "CDC_ERR_TIMEOUT",
          "CDC_ERR_NOMEM", "CDC_ERR_INTERNAL"]
OK, ERR_INVALID, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM, ERR_INTERNAL = range(7)

_lock = threading.Lock()
_lib = None


class CdcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        name = STATUS[status] if 0 <= status < len(STATUS) else "status %d" % status
        super().__init__("%s%s" % (name, (": " + what) if what else ""))


class Params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_uint32), ("min", ctypes.c_uint32), ("max", ctypes.c_uint32)]


class Result(ctypes.Structure):
    """cdc_result: one finished serving request."""
    _fields_ = [("tag", ctypes.c_uint64), ("n_bounds", ctypes.c_uint64), ("t_arrive_ms", ctypes.c_double),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("alg", ctypes.c_int32), ("batch_size", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libcdc.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libcdc.so is missing at %s; build it with "
                               "paper_2508_05797_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        vp, sz, u64, i32, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
        P = Params
        sig = {
            "cdc_create": ([ctypes.POINTER(vp), i32], i32),
            "cdc_destroy": ([vp], i32),
            "cdc_chunk": ([vp, i32, P, vp, sz, vp, ctypes.POINTER(sz), vp], i32),
            "cdc_chunk_async": ([vp, i32, P, vp, sz, vp, sz, vp, vp], i32),
            "cdc_chunk_batch": ([vp, i32, P, vp, sz, vp, sz, vp, vp, sz, ctypes.POINTER(sz), vp], i32),
            "cdc_chunk_host": ([vp, i32, P, vp, sz, vp, ctypes.POINTER(sz), vp], i32),
            "cdc_reserve": ([vp, i32, P, sz, sz], i32),
            "cdc_sync_status": ([vp, vp], i32),
            "cdc_set_option": ([vp, i32, i64], i32),
            "cdc_get_option": ([vp, i32, ctypes.POINTER(i64)], i32),
            "cdc_last_timing": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)], i32),
            "cdc_last_launches": ([vp, ctypes.POINTER(i32)], i32),
            "cdc_last_stage": ([vp, ctypes.POINTER(i32)], i32),
            "cdc_profile_collect": ([vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(i64)], i32),
            "cdc_stats": ([vp, vp, i32, vp], i32),
            "cdc_chunk_static": ([i32, P, vp, sz, vp, ctypes.POINTER(sz), vp], i32),
            "cdc_autotune": ([vp, i32, P, vp, sz, vp, sz, vp, vp, sz, ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(ctypes.c_float), vp], i32),
            "cdc_ebs": ([i32, vp, sz, vp, sz, vp, vp, vp], i32),
            "cdc_rs": ([i32, vp, sz, vp, vp, sz, vp, vp], i32),
            "cdc_fingerprint": ([vp, sz, vp, sz, vp, vp], i32),
            "cdc_byte_shares": ([i32, P, vp, sz, vp, sz, vp, vp], i32),
            "cdc_size_histogram": ([vp, sz, ctypes.c_uint64, ctypes.c_uint32, vp, vp], i32),
            "cdc_feed_create": ([ctypes.POINTER(vp), vp, i32, P], i32),
            "cdc_feed_push": ([vp, vp, sz, i32, vp, ctypes.POINTER(sz), vp], i32),
            "cdc_feed_position": ([vp, ctypes.POINTER(u64), ctypes.POINTER(u64)], i32),
            "cdc_feed_reset": ([vp], i32),
            "cdc_feed_destroy": ([vp], i32),
            "cdc_server_create": ([ctypes.POINTER(vp), i32, sz, i32, sz], i32),
            "cdc_server_submit": ([vp, i32, P, vp, sz, vp, sz, u64, ctypes.c_double], i32),
            "cdc_server_poll": ([vp, ctypes.POINTER(Result), i32, ctypes.POINTER(i32), i32], i32),
            "cdc_server_clock": ([vp, ctypes.POINTER(ctypes.c_double)], i32),
            "cdc_server_destroy": ([vp], i32),
            "cdc_status_string": ([i32], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols() -> list[str]:
    return ["cdc_create", "cdc_destroy", "cdc_chunk", "cdc_chunk_async", "cdc_chunk_batch", "cdc_chunk_host",
            "cdc_reserve", "cdc_sync_status", "cdc_set_option", "cdc_get_option", "cdc_last_timing",
            "cdc_last_launches", "cdc_last_stage", "cdc_profile_collect", "cdc_stats", "cdc_chunk_static", "cdc_autotune", "cdc_ebs", "cdc_rs", "cdc_fingerprint", "cdc_byte_shares",
            "cdc_size_histogram", "cdc_feed_create", "cdc_feed_push",
            "cdc_feed_position", "cdc_feed_reset", "cdc_feed_destroy", "cdc_server_create", "cdc_server_submit",
            "cdc_server_poll", "cdc_server_clock", "cdc_server_destroy", "cdc_status_string"]


def alg_id(alg) -> int:
    return ALGS[alg.lower()] if isinstance(alg, str) else int(alg)


def _check(st: int, what: str = ""):
    if st != OK:
        raise CdcError(st, what)


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def max_boundaries(n: int, mn: int) -> int:
    """Upper bound on the number of chunks of n bytes: all but the last are >= min."""
    return n // max(mn, 1) + 1


class Chunker:
    """One library handle on one CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self.lib.cdc_create(ctypes.byref(h), device), "cdc_create")
        self.h = h

    def close(self):
        if self.h:
            self.lib.cdc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # options
    def set_option(self, opt: int, value: int):
        _check(self.lib.cdc_set_option(self.h, opt, int(value)), "cdc_set_option")

    def get_option(self, opt: int) -> int:
        v = ctypes.c_int64()
        _check(self.lib.cdc_get_option(self.h, opt, ctypes.byref(v)), "cdc_get_option")
        return v.value

    def last_timing(self):
        a, b = ctypes.c_float(), ctypes.c_float()
        _check(self.lib.cdc_last_timing(self.h, ctypes.byref(a), ctypes.byref(b)), "cdc_last_timing")
        return a.value, b.value

    def stats(self, stream=None) -> dict:
        """Work counters of the last call made with OPT_STATS on."""
        arr = (ctypes.c_uint64 * len(STAT_NAMES))()
        _check(self.lib.cdc_stats(self.h, arr, len(STAT_NAMES), _stream_handle(stream)), "cdc_stats")
        return {name: int(arr[i]) for i, name in enumerate(STAT_NAMES)}

    def last_launches(self) -> int:
        n = ctypes.c_int()
        _check(self.lib.cdc_last_launches(self.h, ctypes.byref(n)))
        return n.value

    def last_stage(self) -> int:
        """Chain stage of the last call: 1 speculation, 2 candidate graph (cdc_last_stage)."""
        n = ctypes.c_int()
        _check(self.lib.cdc_last_stage(self.h, ctypes.byref(n)))
        return n.value

    def profile_collect(self):
        """(calls, summary ms, chain ms, speculation-kernel ms, kernel launches)
        recorded since the last collect."""
        n, a, b, c, l = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
        _check(self.lib.cdc_profile_collect(self.h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c), ctypes.byref(l)), "cdc_profile_collect")
        return n.value, a.value, b.value, c.value, l.value

    # chunking
    def chunk(self, data, alg, w: int, mn: int, mx: int, out=None, stream=None):
        """Boundaries of a uint8 CUDA tensor as an int64 CUDA tensor."""
        import torch
        assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
        n = data.numel()
        if out is None:
            out = torch.empty(max_boundaries(n, mn), dtype=torch.int64, device=data.device)
        cap = ctypes.c_size_t(out.numel())
        st = self.lib.cdc_chunk(self.h, alg_id(alg), Params(w, mn, mx), data.data_ptr() if n else None, n,
                                out.data_ptr(), ctypes.byref(cap), _stream_handle(stream))
        _check(st, "cdc_chunk (count %d)" % cap.value)
        return out[:cap.value]

    def chunk_async(self, data, alg, w: int, mn: int, mx: int, out, d_count, stream=None):
        import torch
        assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
        st = self.lib.cdc_chunk_async(self.h, alg_id(alg), Params(w, mn, mx), data.data_ptr(), data.numel(),
                                      out.data_ptr(), out.numel(), d_count.data_ptr(), _stream_handle(stream))
        _check(st, "cdc_chunk_async")

    def chunk_batch(self, arena, file_off, alg, w: int, mn: int, mx: int, out=None, index=None,
                    stream=None, sync: bool = True):
        """Chunk every file of a packed arena. file_off: int64 CUDA tensor of
        n_files + 1 offsets. Returns (boundaries, index) with file f's
        boundaries at boundaries[index[f]:index[f+1]] (relative to its start)."""
        import torch
        assert arena.dtype == torch.uint8 and arena.is_cuda
        n_files = file_off.numel() - 1
        if out is None:
            out = torch.empty(arena.numel() // max(mn, 1) + n_files + 1, dtype=torch.int64, device=arena.device)
        if index is None:
            index = torch.empty(n_files + 1, dtype=torch.int64, device=arena.device)
        total = ctypes.c_size_t(0)
        st = self.lib.cdc_chunk_batch(self.h, alg_id(alg), Params(w, mn, mx), arena.data_ptr(), arena.numel(),
                                      file_off.data_ptr(), n_files, out.data_ptr(), index.data_ptr(), out.numel(),
                                      ctypes.byref(total) if sync else None, _stream_handle(stream))
        _check(st, "cdc_chunk_batch (total %d)" % total.value)
        return (out[:total.value] if sync else out), index

    def chunk_host(self, data, alg, w: int, mn: int, mx: int, out=None, stream=None):
        """End to end from a host numpy uint8 array to a host numpy uint64 array."""
        import numpy as np
        assert data.dtype == np.uint8 and data.flags.c_contiguous
        n = data.size
        if out is None:
            out = np.empty(max_boundaries(n, mn), dtype=np.uint64)
        cap = ctypes.c_size_t(out.size)
        st = self.lib.cdc_chunk_host(self.h, alg_id(alg), Params(w, mn, mx), data.ctypes.data, n,
                                     out.ctypes.data, ctypes.byref(cap), _stream_handle(stream))
        _check(st, "cdc_chunk_host (count %d)" % cap.value)
        return out[:cap.value]

    def autotune(self, data, alg, w: int, mn: int, mx: int, out=None, file_off=None, index=None, stream=None):
        """cdc_autotune on a uint8 CUDA tensor (one stream, or a packed arena
        with file_off). Returns (segment bytes, warp chains, best ms); the
        handle keeps the chosen options."""
        import torch
        assert data.dtype == torch.uint8 and data.is_cuda
        n = data.numel()
        n_files = 0 if file_off is None else file_off.numel() - 1
        if out is None:
            out = torch.empty(n // max(mn, 1) + n_files + 1, dtype=torch.int64, device=data.device)
        if file_off is not None and index is None:
            index = torch.empty(n_files + 1, dtype=torch.int64, device=data.device)
        sg, wc, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_float()
        st = self.lib.cdc_autotune(self.h, alg_id(alg), Params(w, mn, mx), data.data_ptr(), n,
                                   file_off.data_ptr() if file_off is not None else None, n_files, out.data_ptr(),
                                   index.data_ptr() if index is not None else None, out.numel(), ctypes.byref(sg),
                                   ctypes.byref(wc), ctypes.byref(ms), _stream_handle(stream))
        _check(st, "cdc_autotune")
        return sg.value, wc.value, ms.value

    def reserve(self, alg, w: int, mn: int, mx: int, n: int, n_files: int = 0):
        _check(self.lib.cdc_reserve(self.h, alg_id(alg), Params(w, mn, mx), n, n_files), "cdc_reserve")

    def sync_status(self, stream=None):
        _check(self.lib.cdc_sync_status(self.h, _stream_handle(stream)), "device-side status")


class Feed:
    """cdc_feed: resumable chunking of one stream handed over in pieces.
    push() returns the boundaries settled by that piece (offsets from the start
    of the stream); concatenated over all pushes they equal chunk() of the
    whole stream. Borrows the Chunker's handle."""

    def __init__(self, chunker: Chunker, alg, w: int, mn: int, mx: int):
        self.lib = chunker.lib
        self.chunker = chunker
        self.mn = mn
        self.horizon = mx + (w if alg_id(alg) == ALGS["maxp"] else 0)
        h = ctypes.c_void_p()
        _check(self.lib.cdc_feed_create(ctypes.byref(h), chunker.h, alg_id(alg), Params(w, mn, mx)),
               "cdc_feed_create")
        self.f = h

    def position(self):
        """(bytes received, stream offset of the next unsettled chunk start)"""
        r, s = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self.lib.cdc_feed_position(self.f, ctypes.byref(r), ctypes.byref(s)), "cdc_feed_position")
        return r.value, s.value

    def push(self, piece, final: bool = False, out=None, stream=None):
        import torch
        n = 0 if piece is None else piece.numel()
        if piece is not None:
            assert piece.dtype == torch.uint8 and piece.is_cuda and piece.is_contiguous()
        received, start = self.position()
        if out is None:
            out = torch.empty(max_boundaries(received + n - start, self.mn) + 1, dtype=torch.int64,
                              device=torch.device("cuda", self.chunker.device))
        cap = ctypes.c_size_t(out.numel())
        st = self.lib.cdc_feed_push(self.f, piece.data_ptr() if n else None, n, 1 if final else 0,
                                    out.data_ptr(), ctypes.byref(cap), _stream_handle(stream))
        _check(st, "cdc_feed_push (count %d)" % cap.value)
        return out[:cap.value]

    def reset(self):
        """Start a new stream, keeping the feed's device buffers."""
        _check(self.lib.cdc_feed_reset(self.f), "cdc_feed_reset")

    def close(self):
        if self.f:
            self.lib.cdc_feed_destroy(self.f)
            self.f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving engine (cdc_server_*): requests from host memory, admitted under
    a device-memory budget and run with continuous batching on `slots` streams.
    Submitted arrays must stay alive and unchanged until their result is
    polled (the binding keeps references until then)."""

    def __init__(self, device: int = 0, budget_bytes: int = 40 << 30, slots: int = 4, max_batch: int = 0):
        self.lib = load_library()
        h = ctypes.c_void_p()
        _check(self.lib.cdc_server_create(ctypes.byref(h), device, budget_bytes, slots, max_batch),
               "cdc_server_create")
        self.h = h
        self._live = {}

    def submit(self, data, alg, w: int, mn: int, mx: int, out, tag: int, arrive_ms: float = -1.0):
        """Queue `data` (uint8 numpy array) with boundaries into `out` (uint64)."""
        import numpy as np
        assert data.dtype == np.uint8 and data.flags.c_contiguous
        assert out.dtype == np.uint64 and out.flags.c_contiguous
        _check(self.lib.cdc_server_submit(self.h, alg_id(alg), Params(w, mn, mx), data.ctypes.data if data.size else None,
                                          data.size, out.ctypes.data if out.size else None, out.size, int(tag),
                                          float(arrive_ms)), "cdc_server_submit")
        self._live[int(tag)] = (data, out)

    def poll(self, max_results: int = 1024, wait_ms: int = 0) -> list:
        arr = (Result * max(max_results, 1))()
        n = ctypes.c_int()
        _check(self.lib.cdc_server_poll(self.h, arr, max_results, ctypes.byref(n), wait_ms), "cdc_server_poll")
        out = []
        for i in range(n.value):
            r = arr[i]
            self._live.pop(int(r.tag), None)
            out.append({f: getattr(r, f) for f, _ in Result._fields_ if f != "pad"})
        return out

    def clock(self) -> float:
        t = ctypes.c_double()
        _check(self.lib.cdc_server_clock(self.h, ctypes.byref(t)), "cdc_server_clock")
        return t.value

    def close(self):
        if self.h:
            self.lib.cdc_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict = {}


def default_chunker(device: int | None = None) -> Chunker:
    import torch
    d = torch.cuda.current_device() if device is None else device
    if d not in _default:
        _default[d] = Chunker(d)
    return _default[d]


def chunk(data, alg, w: int, mn: int, mx: int, stream=None):
    """Boundaries (int64 CUDA tensor) of a uint8 CUDA tensor on the current stream."""
    return default_chunker(data.device.index).chunk(data, alg, w, mn, mx, stream=stream)


EBS_OPS = {"max": 0, "min": 1}
RS_CMPS = {"gt": 0, "lt": 1, "geq": 2, "leq": 3, "eq": 4}


def ebs(data, ranges, op="max", with_pos=True, stream=None):
    """Extreme Byte Search over ranges (int64 CUDA tensor of shape (n, 2))
    of a uint8 CUDA tensor: (values uint8, first positions int64 or None)."""
    import torch
    assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
    r = ranges.contiguous()
    n = r.shape[0]
    val = torch.empty(n, dtype=torch.uint8, device=data.device)
    pos = torch.empty(n, dtype=torch.int64, device=data.device) if with_pos else None
    _check(load_library().cdc_ebs(EBS_OPS[op], data.data_ptr() if data.numel() else None, data.numel(),
                                  r.data_ptr() if n else None, n, val.data_ptr() if n else None,
                                  pos.data_ptr() if (pos is not None and n) else None, _stream_handle(stream)),
           "cdc_ebs")
    return val, pos


def rs(data, ranges, thresholds, cmp="geq", stream=None):
    """Range Scan: first position in each range whose byte compares true
    against its threshold (uint8 CUDA tensor), or the range end."""
    import torch
    assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
    r = ranges.contiguous()
    t = thresholds.contiguous()
    n = r.shape[0]
    pos = torch.empty(n, dtype=torch.int64, device=data.device)
    _check(load_library().cdc_rs(RS_CMPS[cmp], data.data_ptr() if data.numel() else None, data.numel(),
                                 r.data_ptr() if n else None, t.data_ptr() if n else None, n,
                                 pos.data_ptr() if n else None, _stream_handle(stream)), "cdc_rs")
    return pos


def fingerprint(data, bounds, stream=None):
    """128-bit fingerprints (int64 CUDA tensor of shape (n, 2)) of the chunks
    of a uint8 CUDA tensor given its boundary list (int64 CUDA tensor)."""
    import torch
    assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
    b = bounds.contiguous()
    n = b.numel()
    fp = torch.empty((n, 2), dtype=torch.int64, device=data.device)
    _check(load_library().cdc_fingerprint(data.data_ptr() if data.numel() else None, data.numel(),
                                          b.data_ptr() if n else None, n, fp.data_ptr() if n else None,
                                          _stream_handle(stream)), "cdc_fingerprint")
    return fp


def byte_shares(data, bounds, alg, w: int, mn: int, mx: int, stream=None):
    """(bytes read by Extreme Byte Searches, bytes read by Range Scans) while
    the chunks `bounds` of `data` were found (cdc_byte_shares)."""
    import torch
    lib = load_library()
    assert data.dtype == torch.uint8 and data.is_cuda
    out = torch.empty(2, dtype=torch.int64, device=data.device)
    n = bounds.numel()
    _check(lib.cdc_byte_shares(alg_id(alg), Params(w, mn, mx), data.data_ptr() if data.numel() else None,
                               data.numel(), bounds.data_ptr() if n else None, n, out.data_ptr(),
                               _stream_handle(stream)), "cdc_byte_shares")
    v = out.cpu().tolist()
    return v[0], v[1]


def size_histogram(bounds, bin_width: int, n_bins: int, stream=None):
    """Chunk-size histogram of a boundary list (int64 CUDA tensor, as chunk
    returns): counts of sizes in [k * bin_width, (k + 1) * bin_width) for
    k < n_bins - 1, the last bin taking every larger size (cdc_size_histogram).
    Returns an int64 CUDA tensor of n_bins counts; its cumulative sum over the
    chunk count is the chunk-size CDF."""
    import torch
    lib = load_library()
    assert bounds.dtype == torch.int64 and bounds.is_cuda and bounds.is_contiguous()
    h = torch.empty(n_bins, dtype=torch.int64, device=bounds.device)
    _check(lib.cdc_size_histogram(bounds.data_ptr() if bounds.numel() else None, bounds.numel(), int(bin_width),
                                  int(n_bins), h.data_ptr(), _stream_handle(stream)), "cdc_size_histogram")
    return h


def dedup_report(pieces):
    """Deduplication over a list of (uint8 CUDA tensor, its boundaries):
    chunks are equal when length and fingerprint are (Section 2.2, Eq. 1:
    space savings = 1 - unique bytes / total bytes). Also the chunk-size
    distribution (sizes at the 10/50/90/99th percentiles). Sorting and
    counting use torch on the device."""
    import torch
    keys, sizes = [], []
    for data, b in pieces:
        if b.numel() == 0:
            continue
        fp = fingerprint(data, b)
        sz = torch.diff(b, prepend=torch.zeros(1, dtype=b.dtype, device=b.device))
        keys.append(torch.stack([fp[:, 0], fp[:, 1], sz], dim=1))
        sizes.append(sz)
    if not keys:
        return {"chunks": 0, "unique_chunks": 0, "total_bytes": 0, "unique_bytes": 0, "savings": 0.0}
    k = torch.cat(keys)
    sz = torch.cat(sizes)
    uniq, first = torch.unique(k, dim=0, return_inverse=True)
    total = int(sz.sum().item())
    ubytes = int(uniq[:, 2].sum().item())
    q = torch.quantile(sz.double(), torch.tensor([0.1, 0.5, 0.9, 0.99], dtype=torch.float64, device=sz.device))
    return {"chunks": int(k.shape[0]), "unique_chunks": int(uniq.shape[0]), "total_bytes": total,
            "unique_bytes": ubytes, "savings": 1.0 - ubytes / max(total, 1),
            "size_quantiles": {"p10": float(q[0]), "p50": float(q[1]), "p90": float(q[2]), "p99": float(q[3])},
            "mean_size": total / max(int(k.shape[0]), 1)}


STATIC_MAX_LEN = 16 << 20


def chunk_static(data, alg, w: int, mn: int, mx: int, out=None, stream=None):
    """cdc_chunk_static: boundaries of a uint8 CUDA tensor (at most
    STATIC_MAX_LEN bytes) on the tensor's device, with the library's fixed
    scratch and no handle. The library allocates nothing; `out` (int64 CUDA
    tensor on the same device) is allocated here when not given. Calls must
    not overlap."""
    import torch
    assert data.dtype == torch.uint8 and data.is_cuda and data.is_contiguous()
    lib = load_library()
    n = data.numel()
    if out is None:
        out = torch.empty(max_boundaries(n, mn), dtype=torch.int64, device=data.device)
    assert out.dtype == torch.int64 and out.is_contiguous() and out.device == data.device
    cap = ctypes.c_size_t(out.numel())
    with torch.cuda.device(data.device):
        st = lib.cdc_chunk_static(alg_id(alg), Params(w, mn, mx), data.data_ptr() if n else None, n,
                                  out.data_ptr(), ctypes.byref(cap), _stream_handle(stream))
    _check(st, "cdc_chunk_static (count %d)" % cap.value)
    return out[:cap.value]


def chunk_batch(arena, file_off, alg, w: int, mn: int, mx: int, stream=None):
    return default_chunker(arena.device.index).chunk_batch(arena, file_off, alg, w, mn, mx, stream=stream)
