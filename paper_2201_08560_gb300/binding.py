"""Thin ctypes binding of libb2sr.so (the C ABI in include/b2sr.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  The functions
keep the C names; a failed call raises B2SRError with the library's message.
Importing this module loads the library and fails loudly if it has not been
built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libb2sr.so")

BOOL_OR_AND, PLUS_TIMES, MIN_PLUS, MAX_TIMES = 0, 1, 2, 3
VEC_BITS, VEC_I32, VEC_F32, VEC_BITS64, VEC_I64 = 0, 1, 2, 3, 4
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_TILE", 3: "OOM", 4: "CUDA", 5: "NOT_CONVERGED",
          6: "ADMISSION_REFUSED", 7: "ABORTED"}
WORD_BYTES = {4: 1, 8: 1, 16: 2, 32: 4}


class B2SRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("tile_dim", ctypes.c_int32), ("n_tile_rows", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("n_tiles", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("bytes", ctypes.c_int64)]


class TuneReport(ctypes.Structure):
    _fields_ = [("est_ratio", ctypes.c_double * 4), ("est_tiles", ctypes.c_double * 4),
                ("trial_us", (ctypes.c_double * 2) * 4), ("tiles", ctypes.c_int64 * 4),
                ("tile_dim", ctypes.c_int32), ("schedule", ctypes.c_int32)]

    def as_dict(self):
        return {"est_ratio": list(self.est_ratio), "est_tiles": list(self.est_tiles),
                "trial_us": [list(r) for r in self.trial_us], "tiles": list(self.tiles),
                "tile_dim": self.tile_dim, "schedule": self.schedule}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("refused", ctypes.c_int64), ("steps", ctypes.c_int64), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("queries_per_s", ctypes.c_double), ("bytes_in_use", ctypes.c_int64),
                ("budget", ctypes.c_int64)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"the CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    p, i32, i64, c_int, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_float
    pp = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "b2sr_last_error": (ctypes.c_char_p, []),
        "b2sr_version": (ctypes.c_char_p, []),
        "b2sr_from_csr": (c_int, [i32, p, p, i64, c_int, p, pp]),
        "b2sr_to_csr": (c_int, [p, p, p, ctypes.POINTER(i64), p]),
        "b2sr_info": (c_int, [p, ctypes.POINTER(Info)]),
        "b2sr_arrays": (c_int, [p, pp, pp, pp]),
        "b2sr_export": (c_int, [p, p, p, p, p]),
        "b2sr_destroy": (c_int, [p]),
        "b2sr_lower": (c_int, [p, p, pp]),
        "b2sr_transpose": (c_int, [p, p, pp]),
        "b2sr_planes_from_csr": (c_int, [p, p, p, p, c_int, p, p]),
        "b2sr_spmv_planes": (c_int, [p, p, c_int, c_int, p, c_int, p, p, c_int, p]),
        "b2sr_weights_from_csr": (c_int, [p, p, p, p, p, p]),
        "b2sr_spmv": (c_int, [p, c_int, c_int, p, c_int, p, p, c_int, p, p]),
        "b2sr_spmm_bits64": (c_int, [p, p, p, p, c_int, p]),
        "b2sr_spmv_bool_noalloc": (c_int, [p, p, p, p, c_int, p]),
        "b2sr_spmm_f32x4": (c_int, [p, p, p, p, c_int, p]),
        "b2sr_spgemm_masked_count": (c_int, [p, p, p, p, p]),
        "b2sr_spgemm_masked_count_work": (c_int, [p, p, p, p, p, p]),
        "b2sr_spgemm_bool": (c_int, [p, p, p, pp]),
        "b2sr_set_schedule": (c_int, [p, c_int]),
        "b2sr_sample_profile": (c_int, [i32, p, p, i64, p, i64, p, p, p]),
        "b2sr_autotune": (c_int, [i32, p, p, i64, p, i64, c_int, c_int, ctypes.c_double, c_int, p, pp,
                                  ctypes.POINTER(TuneReport)]),
        "b2sr_bfs": (c_int, [p, i32, p, c_int, p]),
        "b2sr_bfs_multi": (c_int, [p, p, c_int, p, c_int, p]),
        "b2sr_bfs_diropt": (c_int, [p, p, i32, p, c_int, p]),
        "b2sr_bfs_sources": (c_int, [p, p, c_int, p, c_int, p]),
        "b2sr_from_csr_batch": (c_int, [c_int, p, p, p, p, c_int, p, pp, p]),
        "b2sr_sssp": (c_int, [p, p, i32, p, c_int, p]),
        "b2sr_sssp_push": (c_int, [p, p, i32, p, f32, c_int, p]),
        "b2sr_sssp_push_rounds": (c_int, [p, p]),
        "b2sr_pagerank": (c_int, [p, f32, c_int, p, p, p]),
        "b2sr_cc": (c_int, [p, p, c_int, p]),
        "b2sr_mis": (c_int, [p, p, p, c_int, p]),
        "b2sr_color": (c_int, [p, p, p, c_int, c_int, p]),
        "b2sr_tc": (c_int, [p, p, p]),
        "b2sr_server_create": (c_int, [i64, c_int, c_int, pp]),
        "b2sr_server_add_graph": (c_int, [p, p, ctypes.POINTER(i32)]),
        "b2sr_server_graph_bytes": (c_int, [p, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "b2sr_server_submit_bfs": (c_int, [p, i32, i32, p, ctypes.POINTER(i64)]),
        "b2sr_server_submit_pagerank": (c_int, [p, i32, i32, f32, c_int, p, ctypes.POINTER(i64)]),
        "b2sr_server_wait": (c_int, [p, i64, ctypes.c_double, ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_double)]),
        "b2sr_server_drain": (c_int, [p, ctypes.c_double]),
        "b2sr_server_stats": (c_int, [p, ctypes.POINTER(ServerStats)]),
        "b2sr_server_reset_stats": (c_int, [p]),
        "b2sr_server_destroy": (c_int, [p]),
        "b2sr_launch_count": (i64, []),
        "b2sr_timing_enable": (None, [c_int]),
        "b2sr_timing_read": (c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_double)]),
        "b2sr_timing_reset": (c_int, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int):
    if status != 0:
        raise B2SRError(status, lib.b2sr_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def bitset_words(n: int) -> int:
    return (n + 31) // 32


class Matrix:
    """Owner of a b2sr_handle; released by close() or garbage collection."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        inf = Info()
        _check(lib.b2sr_info(self._h, ctypes.byref(inf)))
        self.n = inf.n
        self.tile_dim = inf.tile_dim
        self.n_tile_rows = inf.n_tile_rows
        self.n_tiles = inf.n_tiles
        self.nnz = inf.nnz
        self.bytes = inf.bytes

    @property
    def schedule(self) -> int:
        inf = Info()
        _check(lib.b2sr_info(self.handle, ctypes.byref(inf)))
        return inf.schedule

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("matrix is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None  # never destroyed twice, even if this call fails
            _check(lib.b2sr_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# storage
# ---------------------------------------------------------------------------

def b2sr_from_csr(n: int, rowptr: torch.Tensor, colind: torch.Tensor, tile_dim: int, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(lib.b2sr_from_csr(int(n), _ptr(rowptr), _ptr(colind), int(colind.numel()), int(tile_dim),
                             _stream(stream), ctypes.byref(h)))
    return Matrix(h)


def b2sr_from_csr_batch(graphs_csr: Sequence, tile_dim: int, stream=None):
    """Block-diagonal arena of several graphs.  graphs_csr: (n, rowptr, colind)
    per graph with device int32 tensors.  Returns (Matrix, bases) where bases
    is a list of ngraphs+1 row offsets."""
    g = len(graphs_csr)
    ns = (ctypes.c_int32 * g)(*[int(n) for n, _, _ in graphs_csr])
    rps = (ctypes.c_void_p * g)(*[_ptr(rp) for _, rp, _ in graphs_csr])
    cis = (ctypes.c_void_p * g)(*[_ptr(ci) for _, _, ci in graphs_csr])
    nnz = (ctypes.c_int64 * g)(*[int(ci.numel()) for _, _, ci in graphs_csr])
    bases = (ctypes.c_int64 * (g + 1))()
    h = ctypes.c_void_p()
    _check(lib.b2sr_from_csr_batch(g, ns, rps, cis, nnz, int(tile_dim), _stream(stream), ctypes.byref(h), bases))
    return Matrix(h), list(bases)


SCHED_AUTO, SCHED_STAGED, SCHED_DIRECT = 0, 1, 2


def b2sr_set_schedule(m: Matrix, schedule: int) -> None:
    _check(lib.b2sr_set_schedule(m.handle, int(schedule)))


def b2sr_sample_profile(n: int, rowptr: torch.Tensor, colind: torch.Tensor, sample, stream=None):
    """Alg. 1 estimate on the device: (est_ratio[4], est_tiles[4]) for k = 4, 8, 16, 32."""
    import numpy as np
    smp = np.ascontiguousarray(np.asarray(sample, dtype=np.int32))
    est = (ctypes.c_double * 4)()
    th = (ctypes.c_double * 4)()
    _check(lib.b2sr_sample_profile(int(n), _ptr(rowptr), _ptr(colind), int(colind.numel()),
                                   smp.ctypes.data_as(ctypes.c_void_p), int(smp.size), est, th, _stream(stream)))
    return list(est), list(th)


def b2sr_autotune(n: int, rowptr: torch.Tensor, colind: torch.Tensor, sample, semiring: int, in_kind: int,
                  keep_ratio: float = 0.0, trials: int = 5, stream=None):
    """Returns (Matrix with the chosen tile_dim and schedule, report dict)."""
    import numpy as np
    smp = np.ascontiguousarray(np.asarray(sample, dtype=np.int32))
    rep = TuneReport()
    h = ctypes.c_void_p()
    _check(lib.b2sr_autotune(int(n), _ptr(rowptr), _ptr(colind), int(colind.numel()),
                             smp.ctypes.data_as(ctypes.c_void_p), int(smp.size), int(semiring), int(in_kind),
                             float(keep_ratio), int(trials), _stream(stream), ctypes.byref(h), ctypes.byref(rep)))
    return Matrix(h), rep.as_dict()


def b2sr_to_csr(m: Matrix, stream=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    rowptr = torch.empty(m.n + 1, dtype=torch.int32, device=dev)
    nnz = ctypes.c_int64()
    _check(lib.b2sr_to_csr(m.handle, _ptr(rowptr), None, ctypes.byref(nnz), _stream(stream)))
    colind = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    _check(lib.b2sr_to_csr(m.handle, _ptr(rowptr), _ptr(colind), ctypes.byref(nnz), _stream(stream)))
    return rowptr, colind[: nnz.value]


def b2sr_export(m: Matrix, stream=None):
    """(TileRowPtr int32, TileColInd int32, BitTiles uint8 bytes) as new CUDA tensors."""
    dev = torch.device("cuda", torch.cuda.current_device())
    trp = torch.empty(m.n_tile_rows + 1, dtype=torch.int32, device=dev)
    tci = torch.empty(max(m.n_tiles, 1), dtype=torch.int32, device=dev)
    tiles = torch.empty(max(m.n_tiles * m.tile_dim * WORD_BYTES[m.tile_dim], 1), dtype=torch.uint8, device=dev)
    _check(lib.b2sr_export(m.handle, _ptr(trp), _ptr(tci), _ptr(tiles), _stream(stream)))
    return trp, tci[: m.n_tiles], tiles[: m.n_tiles * m.tile_dim * WORD_BYTES[m.tile_dim]]


def b2sr_planes_from_csr(m: Matrix, rowptr: torch.Tensor, colind: torch.Tensor, w_csr: torch.Tensor, bits: int,
                         stream=None) -> torch.Tensor:
    """Bit-planes of integer weights (uint32 values in an int32 tensor, CSR
    order): uint8 tensor of n_tiles * bits * tile_bytes bytes."""
    tb = m.tile_dim * (1 if m.tile_dim <= 8 else m.tile_dim // 8)
    out = torch.empty(max(m.n_tiles * bits * tb, 4), dtype=torch.uint8, device=w_csr.device)
    _check(lib.b2sr_planes_from_csr(m.handle, _ptr(rowptr), _ptr(colind), _ptr(w_csr), int(bits), _ptr(out),
                                    _stream(stream)))
    return out


def b2sr_spmv_planes(m: Matrix, planes: torch.Tensor, bits: int, in_kind: int, x: torch.Tensor, out_kind: int,
                     y: torch.Tensor, mask: Optional[torch.Tensor] = None, mask_complement: bool = False,
                     stream=None) -> torch.Tensor:
    _check(lib.b2sr_spmv_planes(m.handle, _ptr(planes), int(bits), int(in_kind), _ptr(x), int(out_kind), _ptr(y),
                                _ptr(mask), int(bool(mask_complement)), _stream(stream)))
    return y


def b2sr_transpose(m: Matrix, stream=None) -> Matrix:
    """B2SR of A^T (CSC order of the tile index, each tile's bits transposed)."""
    h = ctypes.c_void_p()
    _check(lib.b2sr_transpose(m.handle, _stream(stream), ctypes.byref(h)))
    return Matrix(h)


def b2sr_lower(m: Matrix, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(lib.b2sr_lower(m.handle, _stream(stream), ctypes.byref(h)))
    return Matrix(h)


def b2sr_weights_from_csr(m: Matrix, rowptr: torch.Tensor, colind: torch.Tensor, w_csr: torch.Tensor,
                          stream=None) -> torch.Tensor:
    out = torch.empty(max(m.nnz, 1), dtype=torch.float32, device=w_csr.device)
    _check(lib.b2sr_weights_from_csr(m.handle, _ptr(rowptr), _ptr(colind), _ptr(w_csr), _ptr(out),
                                     _stream(stream)))
    return out[: m.nnz]


# ---------------------------------------------------------------------------
# SpMV / SpMM
# ---------------------------------------------------------------------------

def b2sr_spmv(m: Matrix, semiring: int, in_kind: int, x: torch.Tensor, out_kind: int, y: torch.Tensor,
              mask: Optional[torch.Tensor] = None, mask_complement: bool = False,
              weights: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    _check(lib.b2sr_spmv(m.handle, int(semiring), int(in_kind), _ptr(x), int(out_kind), _ptr(y), _ptr(mask),
                         int(bool(mask_complement)), _ptr(weights), _stream(stream)))
    return y


def b2sr_spmv_bool_noalloc(m: Matrix, x: torch.Tensor, y: torch.Tensor, mask: Optional[torch.Tensor] = None,
                           mask_complement: bool = False, stream=None) -> torch.Tensor:
    """Boolean SpMV with the library's fixed scratch array: no device allocation."""
    _check(lib.b2sr_spmv_bool_noalloc(m.handle, _ptr(x), _ptr(y), _ptr(mask), int(bool(mask_complement)),
                                      _stream(stream)))
    return y


def b2sr_spmm_bits64(m: Matrix, X: torch.Tensor, Y: torch.Tensor, M: Optional[torch.Tensor] = None,
                     complement: bool = False, stream=None) -> torch.Tensor:
    _check(lib.b2sr_spmm_bits64(m.handle, _ptr(X), _ptr(Y), _ptr(M), int(bool(complement)), _stream(stream)))
    return Y


def b2sr_spmm_f32x4(m: Matrix, X: torch.Tensor, Y: torch.Tensor, mask: Optional[torch.Tensor] = None,
                    complement: bool = False, stream=None) -> torch.Tensor:
    """X, Y: float32 tensors of shape (n, 4), contiguous."""
    _check(lib.b2sr_spmm_f32x4(m.handle, _ptr(X), _ptr(Y), _ptr(mask), int(bool(complement)), _stream(stream)))
    return Y


# ---------------------------------------------------------------------------
# SpGEMM
# ---------------------------------------------------------------------------

def b2sr_spgemm_masked_count(A: Matrix, B: Matrix, M: Matrix, count: Optional[torch.Tensor] = None,
                             stream=None) -> torch.Tensor:
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))
    _check(lib.b2sr_spgemm_masked_count(A.handle, B.handle, M.handle, _ptr(count), _stream(stream)))
    return count


def b2sr_spgemm_masked_count_work(A: Matrix, B: Matrix, M: Matrix, stream=None):
    """(count, pairs): the masked count and its AND-popc word operations, as int64 device tensors."""
    count = torch.empty(1, dtype=torch.int64, device=_dev())
    pairs = torch.empty(1, dtype=torch.int64, device=_dev())
    _check(lib.b2sr_spgemm_masked_count_work(A.handle, B.handle, M.handle, _ptr(count), _ptr(pairs), _stream(stream)))
    return count, pairs


def b2sr_spgemm_bool(A: Matrix, B: Matrix, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    _check(lib.b2sr_spgemm_bool(A.handle, B.handle, _stream(stream), ctypes.byref(h)))
    return Matrix(h)


# ---------------------------------------------------------------------------
# graph algorithms
# ---------------------------------------------------------------------------

def _dev():
    return torch.device("cuda", torch.cuda.current_device())


def b2sr_bfs(m: Matrix, src: int, levels: Optional[torch.Tensor] = None, max_iters: int = 0,
             stream=None) -> torch.Tensor:
    if levels is None:
        levels = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_bfs(m.handle, int(src), _ptr(levels), int(max_iters), _stream(stream)))
    return levels[: m.n]


def b2sr_bfs_diropt(m: Matrix, src: int, mT: Optional[Matrix] = None, levels: Optional[torch.Tensor] = None,
                    max_iters: int = 0, stream=None) -> torch.Tensor:
    """Direction-optimising BFS; mT is the transpose (None: m is symmetric)."""
    if levels is None:
        levels = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_bfs_diropt(m.handle, None if mT is None else mT.handle, int(src), _ptr(levels), int(max_iters),
                               _stream(stream)))
    return levels[: m.n]


def b2sr_bfs_sources(m: Matrix, srcs: Sequence[int], levels: Optional[torch.Tensor] = None, max_iters: int = 0,
                     stream=None) -> torch.Tensor:
    srcs = [int(s) for s in srcs]
    arr = (ctypes.c_int32 * len(srcs))(*srcs)
    if levels is None:
        levels = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_bfs_sources(m.handle, arr, len(srcs), _ptr(levels), int(max_iters), _stream(stream)))
    return levels[: m.n]


def b2sr_bfs_multi(m: Matrix, srcs: Sequence[int], levels: Optional[torch.Tensor] = None, max_iters: int = 0,
                   stream=None) -> torch.Tensor:
    srcs = [int(s) for s in srcs]
    arr = (ctypes.c_int32 * len(srcs))(*srcs)
    if levels is None:
        levels = torch.empty((len(srcs), max(m.n, 1)), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_bfs_multi(m.handle, arr, len(srcs), _ptr(levels), int(max_iters), _stream(stream)))
    return levels


def b2sr_sssp(m: Matrix, src: int, weights: Optional[torch.Tensor] = None, dist: Optional[torch.Tensor] = None,
              max_iters: int = 0, stream=None) -> torch.Tensor:
    if dist is None:
        dist = torch.empty(max(m.n, 1), dtype=torch.float32, device=_dev())
    _check(lib.b2sr_sssp(m.handle, _ptr(weights), int(src), _ptr(dist), int(max_iters), _stream(stream)))
    return dist[: m.n]


def b2sr_pagerank(m: Matrix, d: float = 0.85, iters: int = 20, teleport: Optional[torch.Tensor] = None,
                  pr: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if pr is None:
        pr = torch.empty(max(m.n, 1), dtype=torch.float32, device=_dev())
    _check(lib.b2sr_pagerank(m.handle, float(d), int(iters), _ptr(teleport), _ptr(pr), _stream(stream)))
    return pr[: m.n]


def b2sr_cc(m: Matrix, labels: Optional[torch.Tensor] = None, max_iters: int = 0, stream=None) -> torch.Tensor:
    if labels is None:
        labels = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_cc(m.handle, _ptr(labels), int(max_iters), _stream(stream)))
    return labels[: m.n]


def _priority(m: Matrix, priority: torch.Tensor) -> torch.Tensor:
    if priority.dtype != torch.float32 or not priority.is_cuda or priority.numel() < m.n:
        raise ValueError("priority must be a float32 CUDA tensor of n entries")
    return priority.contiguous()


def b2sr_mis(m: Matrix, priority: torch.Tensor, in_set: Optional[torch.Tensor] = None, max_iters: int = 0,
             stream=None) -> torch.Tensor:
    """Maximal independent set: 1 for members (the greedy set in decreasing
    (priority, id) order)."""
    pr = _priority(m, priority)
    if in_set is None:
        in_set = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_mis(m.handle, _ptr(pr), _ptr(in_set), int(max_iters), _stream(stream)))
    return in_set[: m.n]


COLOR_AUTO, COLOR_MAX_TIMES, COLOR_PUSH = 0, 1, 2


def b2sr_color(m: Matrix, priority: torch.Tensor, colors: Optional[torch.Tensor] = None,
               method: int = COLOR_AUTO, max_iters: int = 0, stream=None) -> torch.Tensor:
    """Colouring by priority levels: 0 without a larger (priority, id)
    neighbour, else 1 + the largest colour among the larger neighbours."""
    pr = _priority(m, priority)
    if colors is None:
        colors = torch.empty(max(m.n, 1), dtype=torch.int32, device=_dev())
    _check(lib.b2sr_color(m.handle, _ptr(pr), _ptr(colors), int(method), int(max_iters), _stream(stream)))
    return colors[: m.n]


def b2sr_sssp_push(mT: Matrix, src: int, weights_t: Optional[torch.Tensor] = None,
                   dist: Optional[torch.Tensor] = None, delta: float = 0.0, max_iters: int = 0,
                   stream=None) -> torch.Tensor:
    """Push SSSP on the transpose handle (the matrix itself when symmetric);
    delta > 0 turns on delta-stepping buckets."""
    if dist is None:
        dist = torch.empty(max(mT.n, 1), dtype=torch.float32, device=_dev())
    _check(lib.b2sr_sssp_push(mT.handle, _ptr(weights_t), int(src), _ptr(dist), float(delta), int(max_iters),
                              _stream(stream)))
    return dist[: mT.n]


def b2sr_sssp_push_rounds(with_rows: bool = False):
    """Rounds run by this thread's most recent b2sr_sssp_push; with
    with_rows, (rounds, active tile-rows summed over the rounds)."""
    r = ctypes.c_int64(0)
    a = ctypes.c_int64(0)
    _check(lib.b2sr_sssp_push_rounds(ctypes.byref(r), ctypes.byref(a)))
    return (int(r.value), int(a.value)) if with_rows else int(r.value)


def b2sr_tc(m: Matrix, count: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=_dev())
    _check(lib.b2sr_tc(m.handle, _ptr(count), _stream(stream)))
    return count


def version() -> str:
    return lib.b2sr_version().decode()


# ---------------------------------------------------------------------------
# measurement support
# ---------------------------------------------------------------------------

def b2sr_launch_count() -> int:
    return int(lib.b2sr_launch_count())


def b2sr_timing_enable(on: bool = True):
    lib.b2sr_timing_enable(1 if on else 0)


def b2sr_timing_read(family: str):
    """(device ms, launches, algorithmic bytes) summed over the recorded launches of `family`."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    by = ctypes.c_double()
    _check(lib.b2sr_timing_read(family.encode(), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by)))
    return ms.value, n.value, by.value


def b2sr_timing_reset():
    _check(lib.b2sr_timing_reset())


# ---------------------------------------------------------------------------
# query server
# ---------------------------------------------------------------------------

class Server:
    """Owner of a b2sr_server_t.  Keeps the registered matrices and every
    query's output tensor alive until the query has been waited for."""

    def __init__(self, budget_bytes: int, max_bfs_lanes: int = 64, max_pr_blocks: int = 2):
        h = ctypes.c_void_p()
        _check(lib.b2sr_server_create(int(budget_bytes), int(max_bfs_lanes), int(max_pr_blocks), ctypes.byref(h)))
        self._h = h
        self._graphs = []
        self._outs = {}

    def add_graph(self, m: Matrix) -> int:
        gid = ctypes.c_int32()
        _check(lib.b2sr_server_add_graph(self._h, m.handle, ctypes.byref(gid)))
        self._graphs.append(m)
        return gid.value

    def _n(self, graph: int) -> int:
        return self._graphs[graph].n if 0 <= graph < len(self._graphs) else 1

    def graph_bytes(self, graph: int):
        """(resident, bfs_batch, pr_block) bytes the budget counts for a graph."""
        r, b, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.b2sr_server_graph_bytes(self._h, int(graph), ctypes.byref(r), ctypes.byref(b), ctypes.byref(p)))
        return r.value, b.value, p.value

    def submit_bfs(self, graph: int, src: int, levels: Optional[torch.Tensor] = None):
        if levels is None:
            levels = torch.empty(max(self._n(graph), 1), dtype=torch.int32, device=_dev())
            # the server writes on its own streams: the block must be free of earlier work
            torch.cuda.current_stream().synchronize()
        qid = ctypes.c_int64()
        _check(lib.b2sr_server_submit_bfs(self._h, int(graph), int(src), _ptr(levels), ctypes.byref(qid)))
        self._outs[qid.value] = levels
        return qid.value, levels

    def submit_pagerank(self, graph: int, src: int = -1, d: float = 0.85, iters: int = 20,
                        pr: Optional[torch.Tensor] = None):
        if pr is None:
            pr = torch.empty(max(self._n(graph), 1), dtype=torch.float32, device=_dev())
            torch.cuda.current_stream().synchronize()
        qid = ctypes.c_int64()
        _check(lib.b2sr_server_submit_pagerank(self._h, int(graph), int(src), float(d), int(iters), _ptr(pr),
                                               ctypes.byref(qid)))
        self._outs[qid.value] = pr
        return qid.value, pr

    def wait(self, qid: int, timeout: float = 60.0) -> float:
        """Latency in microseconds; raises B2SRError if the query failed or timed out."""
        done = ctypes.c_int()
        lat = ctypes.c_double()
        try:
            _check(lib.b2sr_server_wait(self._h, int(qid), float(timeout), ctypes.byref(done), ctypes.byref(lat)))
        except B2SRError:
            self._outs.pop(qid, None)
            raise
        if not done.value:
            raise B2SRError(5, f"query {qid} not done after {timeout} s")
        self._outs.pop(qid, None)
        return lat.value

    def poll(self, qid: int) -> bool:
        done = ctypes.c_int()
        _check(lib.b2sr_server_wait(self._h, int(qid), 0.0, ctypes.byref(done), None))
        return bool(done.value)

    def drain(self, timeout: float = 0.0) -> None:
        _check(lib.b2sr_server_drain(self._h, float(timeout)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib.b2sr_server_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def reset_stats(self) -> None:
        _check(lib.b2sr_server_reset_stats(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            self._outs.clear()
            _check(lib.b2sr_server_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
