"""Host (CPU) build of the chain stage's per-thread rules, for tests only."""
import ctypes
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2508_05797_gb300", "csrc")
SRC = os.path.join(HERE, "host_next.cpp")
OUT = os.path.join(HERE, "_build", "libhostnext.so")
_lock = threading.Lock()
_lib = None

RULE_RAM, RULE_AE, RULE_MAXP, RULE_RAM_BYTES, RULE_AE_BYTES, RULE_MAXP_BYTES = range(6)


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        deps = [SRC, os.path.join(CSRC, "chain_logic.cuh"), os.path.join(CSRC, "graph_logic.cuh")]
        if not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in deps):
            tmp = OUT + ".%d.tmp" % os.getpid()
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, SRC, "-o", tmp])
            os.replace(tmp, OUT)
        lib = ctypes.CDLL(OUT)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.hc_next.argtypes = [i32, vp, vp, vp, u64, u64, vp, vp, u32, u32, u32, u32, u64, u64, u64]
        lib.hc_next.restype = u64
        lib.hc_chain.argtypes = [i32, vp, vp, vp, u32, u32, u32, u32, u64, u64, vp, u64]
        lib.hc_chain.restype = u64
        lib.hc_chain_adv.argtypes = [i32, vp, vp, vp, vp, u32, u32, u32, u32, u64, u64, u64, vp, u64, vp]
        lib.hc_chain_adv.restype = u64
        lib.hc_block_max_first.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(u32)]
        lib.hc_block_max_first.restype = None
        gargs = [i32, vp, vp, vp, vp, u32, u32, u32, u32, u64, u64]
        lib.hc_cands.argtypes = gargs + [vp, u64]
        lib.hc_cands.restype = u64
        lib.hc_is_cand.argtypes = gargs + [u64]
        lib.hc_is_cand.restype = i32
        lib.hc_cand_next.argtypes = gargs + [u64, ctypes.POINTER(u32)]
        lib.hc_cand_next.restype = u64
        lib.hc_graph_chain.argtypes = gargs + [vp, u64]
        lib.hc_graph_chain.restype = u64
        lib.hc_graph_chain_t.argtypes = gargs + [vp, vp, vp, u64]
        lib.hc_graph_chain_t.restype = u64
        lib.hc_list_check.argtypes = gargs + [vp, vp, u32, u64, vp]
        lib.hc_list_check.restype = u64
        _lib = lib
        return lib
