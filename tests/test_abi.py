"""The C-ABI library loads and exports every entry point include/b2sr.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "b2sr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:b2sr_status|const char\*)\s+(b2sr_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    from paper_2201_08560_gb300 import build
    build.build()
    g.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["b2sr_from_csr", "b2sr_to_csr", "b2sr_info", "b2sr_destroy", "b2sr_spmv",
                     "b2sr_spmm_bits64", "b2sr_spgemm_bool", "b2sr_spgemm_masked_count", "b2sr_bfs",
                     "b2sr_bfs_multi", "b2sr_sssp", "b2sr_pagerank", "b2sr_cc", "b2sr_tc"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment names the paper passage (Sec./Table/Listing) or says it is not in the paper."""
    text = open(HEADER).read()
    blocks = re.findall(r"/\*((?:(?!\*/).)*)\*/\s*(?:b2sr_status|const char\*)\s+(b2sr_\w+)", text, flags=re.S)
    seen = {name for _, name in blocks}
    assert set(declared_functions()) <= seen
    for comment, name in blocks:
        if name in ("b2sr_last_error", "b2sr_version", "b2sr_info", "b2sr_arrays", "b2sr_export",
                    "b2sr_destroy", "b2sr_to_csr"):
            continue
        flat = " ".join(comment.replace("*", " ").split())
        assert re.search(r"Sec\.|Table|Listing|not in the paper|no counterpart", flat), name


def test_host_side_errors_without_gpu(lib):
    lib.b2sr_from_csr.restype = ctypes.c_int
    lib.b2sr_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    st = lib.b2sr_from_csr(ctypes.c_int32(4), None, None, ctypes.c_int64(0), 6, None, ctypes.byref(out))
    assert st == 2  # UNSUPPORTED_TILE
    assert b"tile_dim" in lib.b2sr_last_error()
    st = lib.b2sr_from_csr(ctypes.c_int32(4), None, None, ctypes.c_int64(0), 8, None, None)
    assert st == 1  # INVALID_ARG: out is NULL
    lib.b2sr_info.restype = ctypes.c_int
    assert lib.b2sr_info(None, None) == 1
    lib.b2sr_destroy.restype = ctypes.c_int
    assert lib.b2sr_destroy(None) == 0
    lib.b2sr_spmv.restype = ctypes.c_int
    assert lib.b2sr_spmv(None, 0, 0, None, 0, None, None, 0, None, None) == 1
    lib.b2sr_version.restype = ctypes.c_char_p
    assert lib.b2sr_version().decode().count(".") == 2
    # the max-times, transpose and bit-plane entry points check their handle first
    for name, args in (("b2sr_mis", (None, None, None, 0, None)),
                       ("b2sr_color", (None, None, None, 0, 0, None)),
                       ("b2sr_transpose", (None, None, ctypes.byref(out))),
                       ("b2sr_planes_from_csr", (None, None, None, None, 8, None, None)),
                       ("b2sr_spmv_planes", (None, None, 8, 0, None, 4, None, None, 0, None))):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        assert f(*args) == 1, name  # INVALID_ARG: not a handle
    assert lib.b2sr_transpose(None, None, None) == 1  # out is NULL

