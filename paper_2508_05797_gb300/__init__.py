"""GB300 (sm_103a) hashless content-defined chunking: RAM, AE, MAXP.

The work runs in libcdc.so (CUDA; C ABI in include/cdc.h); this package is
its Python binding. See ``cdc.Chunker`` and ``cdc.chunk``.
"""
from .cdc import (ALGS, STATIC_MAX_LEN, CdcError, Chunker, Feed, Params, Server, byte_shares, chunk, chunk_batch,
                  chunk_static, dedup_report, ebs,
                  fingerprint, rs, size_histogram,
                  default_chunker, exported_symbols, library_path, load_library, max_boundaries)

__all__ = ["ALGS", "STATIC_MAX_LEN", "CdcError", "Chunker", "Feed", "Params", "Server", "byte_shares", "chunk",
           "chunk_batch", "chunk_static",
           "dedup_report", "ebs", "fingerprint", "rs", "size_histogram",
           "default_chunker",
           "exported_symbols", "library_path", "load_library", "max_boundaries"]
