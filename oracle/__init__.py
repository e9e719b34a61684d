"""CPU oracle for the B2SR bit-graph hot path -- TEST INFRASTRUCTURE ONLY.

Plain C (``oracle.c``, fp64 where floating point) wrapped with ctypes and
numpy.  Only the test suite, the smoke check and the benchmark's CPU-baseline
leg may import this package; the library never does, and the two share no
code.  Each wrapper names the paper passage its C function follows; the C file
states the conventions (bit order, mask modes, identities).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KS = (4, 8, 16, 32)
WORD_BYTES = {4: 1, 8: 1, 16: 2, 32: 4}
WORD_DTYPE = {4: np.uint8, 8: np.uint8, 16: np.uint16, 32: np.uint32}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (portable flags only)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-fopenmp", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32, i64, p, d = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
            sig = {
                "orc_csr_validate": (ctypes.c_int, [i32, p, p]),
                "orc_csr_canonicalize": (i64, [i32, p, p, p, p]),
                "orc_b2sr_rowptr": (i64, [i32, p, p, ctypes.c_int, p]),
                "orc_b2sr_fill": (ctypes.c_int, [i32, p, p, ctypes.c_int, p, p, p]),
                "orc_b2sr_bytes": (i64, [i32, ctypes.c_int, i64]),
                "orc_b2sr_to_csr": (i64, [i32, ctypes.c_int, p, p, p, p, p]),
                "orc_spmv_bool": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_count": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_plus": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_minplus": (None, [i32, p, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_min_i32": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_spmm_or64": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_max": (None, [i32, p, p, p, p, p, ctypes.c_int]),
                "orc_b2sr_planes": (ctypes.c_int, [i32, p, p, p, ctypes.c_int, ctypes.c_int, p, p, p]),
                "orc_spmv_wcount": (None, [i32, p, p, p, p, p, p, ctypes.c_int]),
                "orc_spmv_wplus": (None, [i32, p, p, p, p, p, p, ctypes.c_int]),
                "orc_mis_greedy": (ctypes.c_int, [i32, p, p, p, p]),
                "orc_color_levels": (ctypes.c_int, [i32, p, p, p, p]),
                "orc_masked_count": (i64, [i32, p, p, p, p, p, p]),
                "orc_triangle_count": (i64, [i32, p, p]),
                "orc_spgemm_bool": (i64, [i32, p, p, p, p, p, p]),
                "orc_bfs": (ctypes.c_int, [i32, p, p, i32, p]),
                "orc_sssp": (ctypes.c_int, [i32, p, p, p, i32, p]),
                "orc_pagerank": (ctypes.c_int, [i32, p, p, d, ctypes.c_int, p, p]),
                "orc_cc": (ctypes.c_int, [i32, p, p, p]),
                "orc_sample_profile": (ctypes.c_int, [i32, p, p, p, i64, p, p]),
                "orc_set_threads": (ctypes.c_int, [ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def set_threads(threads: int = 0) -> int:
    """Host threads for the oracle's row loops (0 keeps the current count); returns the count in force."""
    return int(_load().orc_set_threads(int(threads)))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _mask_mode(mask, complement: bool) -> int:
    if mask is None:
        return 0
    return 2 if complement else 1


class _G:
    """Contiguous int32 views of a CSR-like object (n, rowptr, colind)."""

    def __init__(self, g):
        self.n = int(g.n)
        self.rowptr = _c(g.rowptr, np.int32)
        self.colind = _c(g.colind, np.int32)
        if self.colind.size == 0:
            self.colind = np.zeros(1, dtype=np.int32)


# --------------------------------------------------------------------------
# CSR plumbing
# --------------------------------------------------------------------------

def canonicalize(g):
    """Sorted, duplicate-free copy of a CSR (duplicates OR-ed: Sec. III, binary matrix)."""
    from types import SimpleNamespace
    G = _G(g)
    rp = np.zeros(G.n + 1, dtype=np.int32)
    ci = np.zeros(max(int(G.rowptr[-1]), 1), dtype=np.int32)
    nnz = _load().orc_csr_canonicalize(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(rp), _ptr(ci))
    if nnz < 0:
        raise ValueError("invalid CSR")
    return SimpleNamespace(n=G.n, rowptr=rp, colind=ci[:nnz].copy())


# --------------------------------------------------------------------------
# B2SR (Sec. III-A/B, Table 1)
# --------------------------------------------------------------------------

def b2sr(g, k: int):
    """Oracle B2SR arrays of a CSR: (tile_rowptr int32[nTR+1], tile_colind int32[T],
    tiles uintK[T, k]) with word dtype uint8/uint8/uint16/uint32 for k=4/8/16/32."""
    G = _G(g)
    lib = _load()
    ntr = (G.n + k - 1) // k
    trp = np.zeros(ntr + 1, dtype=np.int32)
    T = lib.orc_b2sr_rowptr(G.n, _ptr(G.rowptr), _ptr(G.colind), k, _ptr(trp))
    if T < 0:
        raise ValueError("invalid CSR or tile size")
    tci = np.zeros(max(T, 1), dtype=np.int32)
    tiles = np.zeros(max(T, 1) * k * WORD_BYTES[k], dtype=np.uint8)
    rc = lib.orc_b2sr_fill(G.n, _ptr(G.rowptr), _ptr(G.colind), k, _ptr(trp), _ptr(tci), _ptr(tiles))
    if rc != 0:
        raise ValueError("b2sr fill failed")
    words = tiles[: T * k * WORD_BYTES[k]].view(WORD_DTYPE[k]).reshape(T, k)
    return trp, tci[:T].copy(), words.copy()


def b2sr_bytes(n: int, k: int, T: int) -> int:
    """4(nTileRow+1) + 4T + T*k*word_bytes: the size of the three B2SR arrays."""
    return int(_load().orc_b2sr_bytes(n, k, T))


def b2sr_to_csr(n: int, k: int, tile_rowptr, tile_colind, tiles):
    from types import SimpleNamespace
    lib = _load()
    trp = _c(tile_rowptr, np.int32)
    tci = _c(tile_colind, np.int32) if len(tile_colind) else np.zeros(1, np.int32)
    tw = np.ascontiguousarray(tiles, dtype=WORD_DTYPE[k]).reshape(-1)
    tb = tw.view(np.uint8) if tw.size else np.zeros(1, np.uint8)
    rp = np.zeros(n + 1, dtype=np.int32)
    nnz = lib.orc_b2sr_to_csr(n, k, _ptr(trp), _ptr(tci), _ptr(tb), _ptr(rp), None)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.orc_b2sr_to_csr(n, k, _ptr(trp), _ptr(tci), _ptr(tb), _ptr(rp), _ptr(ci))
    return SimpleNamespace(n=n, rowptr=rp, colind=ci[:nnz].copy())


# --------------------------------------------------------------------------
# SpMV (Table 2 schemes over the Table 4 semirings); inputs must be canonical
# --------------------------------------------------------------------------

def spmv_bool(g, x_bits, mask=None, complement=False):
    G = _G(g)
    x = _c(x_bits, np.uint32)
    y = np.zeros((G.n + 31) // 32, dtype=np.uint32)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_bool(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(x), _ptr(y), _ptr(m),
                          _mask_mode(mask, complement))
    return y


def spmv_count(g, x_bits, mask=None, complement=False):
    G = _G(g)
    x = _c(x_bits, np.uint32)
    y = np.zeros(G.n, dtype=np.int32)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_count(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(x), _ptr(y), _ptr(m),
                           _mask_mode(mask, complement))
    return y


def spmv_plus(g, x, mask=None, complement=False):
    G = _G(g)
    xd = _c(x, np.float64)
    y = np.zeros(G.n, dtype=np.float64)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_plus(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(xd), _ptr(y), _ptr(m),
                          _mask_mode(mask, complement))
    return y


def spmv_minplus(g, x, weights=None, mask=None, complement=False):
    G = _G(g)
    xd = _c(x, np.float64)
    w = None if weights is None else _c(weights, np.float32)
    y = np.zeros(G.n, dtype=np.float64)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_minplus(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(xd), _ptr(w), _ptr(y),
                             _ptr(m), _mask_mode(mask, complement))
    return y


def spmv_min_i32(g, x, mask=None, complement=False):
    G = _G(g)
    xi = _c(x, np.int32)
    y = np.zeros(G.n, dtype=np.int32)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_min_i32(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(xi), _ptr(y), _ptr(m),
                             _mask_mode(mask, complement))
    return y


def spmv_max(g, x, mask=None, complement=False):
    """Max-times (Table 4): y_i = max over row i of x_j, -inf if empty or masked out."""
    G = _G(g)
    xd = _c(x, np.float64)
    y = np.zeros(G.n, dtype=np.float64)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_max(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(xd), _ptr(y), _ptr(m),
                         _mask_mode(mask, complement))
    return y


def b2sr_planes(g, w, bits: int, k: int):
    """Bit-planes of integer weights w (CSR order of g, each < 2^bits) over the
    tile index of b2sr(g, k): uint array [T, bits, k] of the tile word dtype."""
    G = _G(g)
    wv = _c(w, np.uint32)
    if wv.size != int(G.rowptr[-1]):
        raise ValueError("one weight per CSR entry")
    wv = wv if wv.size else np.zeros(1, np.uint32)
    trp, tci, _ = b2sr(G, k)
    T = len(tci)
    out = np.zeros(max(T, 1) * bits * k * WORD_BYTES[k], dtype=np.uint8)
    rc = _load().orc_b2sr_planes(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(wv), int(bits), int(k), _ptr(trp),
                                 _ptr(tci if T else np.zeros(1, np.int32)), _ptr(out))
    if rc != 0:
        raise ValueError("weights do not fit the bit width")
    return out[: T * bits * k * WORD_BYTES[k]].view(WORD_DTYPE[k]).reshape(T, bits, k).copy()


def spmv_wcount(g, w, x_bits, mask=None, complement=False):
    """y_i = sum_{j in row i, x_j = 1} w_ij (int64)."""
    G = _G(g)
    wv = _c(w, np.uint32) if len(w) else np.zeros(1, np.uint32)
    x = _c(x_bits, np.uint32)
    y = np.zeros(G.n, dtype=np.int64)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_wcount(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(wv), _ptr(x), _ptr(y), _ptr(m),
                            _mask_mode(mask, complement))
    return y


def spmv_wplus(g, w, x, mask=None, complement=False):
    """y_i = sum_{j in row i} w_ij x_j (fp64)."""
    G = _G(g)
    wv = _c(w, np.uint32) if len(w) else np.zeros(1, np.uint32)
    xd = _c(x, np.float64)
    y = np.zeros(G.n, dtype=np.float64)
    m = None if mask is None else _c(mask, np.uint32)
    _load().orc_spmv_wplus(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(wv), _ptr(xd), _ptr(y), _ptr(m),
                           _mask_mode(mask, complement))
    return y


def mis_greedy(g, prio):
    """Maximal independent set, greedy in decreasing priority (ties: larger id)."""
    G = _G(g)
    pr = _c(prio, np.float64)
    out = np.zeros(G.n, dtype=np.int32)
    if _load().orc_mis_greedy(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(pr), _ptr(out)) != 0:
        raise MemoryError("oracle")
    return out


def color_levels(g, prio):
    """Colour = 1 + the largest colour among higher-priority neighbours (0 if none)."""
    G = _G(g)
    pr = _c(prio, np.float64)
    out = np.zeros(G.n, dtype=np.int32)
    if _load().orc_color_levels(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(pr), _ptr(out)) != 0:
        raise MemoryError("oracle")
    return out


def spmm_or64(g, X, M=None, complement=False):
    G = _G(g)
    Xc = _c(X, np.uint64)
    Y = np.zeros(G.n, dtype=np.uint64)
    Mc = None if M is None else _c(M, np.uint64)
    _load().orc_spmm_or64(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(Xc), _ptr(Y), _ptr(Mc),
                          _mask_mode(M, complement))
    return Y


# --------------------------------------------------------------------------
# SpGEMM (Table 3) and graph algorithms (Sec. V)
# --------------------------------------------------------------------------

def masked_count(a, b, m) -> int:
    A, B, M = _G(a), _G(b), _G(m)
    return int(_load().orc_masked_count(A.n, _ptr(A.rowptr), _ptr(A.colind), _ptr(B.rowptr),
                                        _ptr(B.colind), _ptr(M.rowptr), _ptr(M.colind)))


def triangle_count(g) -> int:
    G = _G(g)
    return int(_load().orc_triangle_count(G.n, _ptr(G.rowptr), _ptr(G.colind)))


def spgemm_bool(a, b):
    from types import SimpleNamespace
    A, B = _G(a), _G(b)
    lib = _load()
    rp = np.zeros(A.n + 1, dtype=np.int32)
    nnz = lib.orc_spgemm_bool(A.n, _ptr(A.rowptr), _ptr(A.colind), _ptr(B.rowptr), _ptr(B.colind),
                              _ptr(rp), None)
    if nnz < 0:
        raise MemoryError("oracle spgemm")
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.orc_spgemm_bool(A.n, _ptr(A.rowptr), _ptr(A.colind), _ptr(B.rowptr), _ptr(B.colind),
                        _ptr(rp), _ptr(ci))
    return SimpleNamespace(n=A.n, rowptr=rp, colind=ci[:nnz].copy())


def bfs(g, src: int):
    G = _G(g)
    lv = np.zeros(G.n, dtype=np.int32)
    if _load().orc_bfs(G.n, _ptr(G.rowptr), _ptr(G.colind), int(src), _ptr(lv)) != 0:
        raise ValueError("bad source")
    return lv


def sssp(g, src: int, weights=None):
    G = _G(g)
    w = None if weights is None else _c(weights, np.float32)
    dist = np.zeros(G.n, dtype=np.float64)
    if _load().orc_sssp(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(w), int(src), _ptr(dist)) != 0:
        raise ValueError("bad source")
    return dist


def pagerank(g, d: float = 0.85, iters: int = 20, teleport=None):
    G = _G(g)
    t = None if teleport is None else _c(teleport, np.float64)
    x = np.zeros(G.n, dtype=np.float64)
    _load().orc_pagerank(G.n, _ptr(G.rowptr), _ptr(G.colind), float(d), int(iters), _ptr(t), _ptr(x))
    return x


def cc(g):
    G = _G(g)
    lab = np.zeros(G.n, dtype=np.int32)
    _load().orc_cc(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(lab))
    return lab


def sample_profile(g, sample_rows):
    """Alg. 1 estimate: (est_compression[4], est_tiles[4]) for k = 4, 8, 16, 32."""
    G = _G(g)
    s = _c(sample_rows, np.int32)
    est = np.zeros(4, dtype=np.float64)
    th = np.zeros(4, dtype=np.float64)
    rc = _load().orc_sample_profile(G.n, _ptr(G.rowptr), _ptr(G.colind), _ptr(s), int(s.size),
                                    _ptr(est), _ptr(th))
    if rc != 0:
        raise ValueError("bad sample")
    return est, th
