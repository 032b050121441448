"""C ABI of libcdc.so without a GPU: it builds, loads and exports every
function include/cdc.h declares (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "cdc.h")).read()
    return sorted(set(re.findall(r"^CDC_API\s+[\w\s\*]+?\b(cdc_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("cdc_create", "cdc_destroy", "cdc_chunk", "cdc_chunk_async", "cdc_chunk_batch",
                 "cdc_status_string"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import paper_2508_05797_gb300 as pkg
    lib = pkg.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(pkg.exported_symbols())


def test_status_strings():
    import paper_2508_05797_gb300 as pkg
    lib = pkg.load_library()
    assert lib.cdc_status_string(0) == b"CDC_OK"
    assert lib.cdc_status_string(2) == b"CDC_ERR_CAPACITY"
    assert lib.cdc_status_string(4) == b"CDC_ERR_TIMEOUT"
    assert lib.cdc_status_string(99) == b"CDC_ERR_UNKNOWN"


def test_build_targets_sm_103a():
    from paper_2508_05797_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
