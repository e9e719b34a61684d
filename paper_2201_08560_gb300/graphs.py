"""Seeded synthetic graph generators (inputs only).

This module produces the inputs that both the CUDA path and the CPU oracle
consume: binary adjacency matrices in CSR form (int32 ``rowptr``/``colind``),
optional per-entry fp32 weights, and seeded source lists.  It contains none of
the B2SR method's arithmetic: no tiling, packing, products or graph
algorithms.

The paper evaluates on SuiteSparse binary matrices (Sec. VI-A); those are not
available here, so seeded R-MAT and 2D-grid graphs with the workload shapes of
the benchmark configurations stand in for them, plus textbook families
(complete, path, cycle, star, torus, Mycielski) whose properties are known in
closed form.  The Mycielski construction reproduces the paper's
``mycielskian12`` storage figures (Sec. III-C).

Every generator is deterministic given its seed: numpy's PCG64
``default_rng`` yields the same stream on x86-64 and aarch64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class CSR:
    """A square binary matrix in CSR form.

    ``rowptr`` has n+1 int32 entries, ``colind`` nnz int32 entries.  Rows are
    sorted and duplicate-free unless a generator states otherwise.  ``weights``
    (optional) holds one fp32 value per stored entry, in CSR order.
    """

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    weights: Optional[np.ndarray] = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)


# ----------------------------------------------------------------------------
# edge-list -> CSR plumbing
# ----------------------------------------------------------------------------

def from_edges(n: int, src: np.ndarray, dst: np.ndarray, *, symmetric: bool = True,
               drop_self_loops: bool = True, dedup: bool = True, name: str = "") -> CSR:
    """Build a CSR from an edge list (sorted rows, optionally symmetrised)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if symmetric:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    if drop_self_loops:
        keep = src != dst
        src, dst = src[keep], dst[keep]
    key = np.sort(src * np.int64(n) + dst)
    if dedup and key.size:
        first = np.empty(key.size, dtype=bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        key = key[first]
    rows = (key // n).astype(np.int64)
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("graph too large for int32 CSR")
    return CSR(n, rowptr.astype(np.int32), cols, None, name)


def from_dense(a: np.ndarray, name: str = "") -> CSR:
    """CSR of a dense 0/1 matrix (entries are kept exactly as given)."""
    a = np.asarray(a) != 0
    n = a.shape[0]
    rows, cols = np.nonzero(a)
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols.astype(np.int32), None, name)


def to_dense(g: CSR) -> np.ndarray:
    a = np.zeros((g.n, g.n), dtype=np.int64)
    for i in range(g.n):
        for e in range(g.rowptr[i], g.rowptr[i + 1]):
            a[i, g.colind[e]] = 1
    return a


def permute(g: CSR, seed: int) -> CSR:
    """Relabel vertices with a seeded random permutation (rows stay sorted)."""
    rng = np.random.default_rng(seed)
    p = rng.permutation(g.n).astype(np.int64)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    out = from_edges(g.n, p[rows], p[g.colind.astype(np.int64)], symmetric=False,
                     drop_self_loops=False, dedup=True, name=g.name + "-perm")
    return out


# ----------------------------------------------------------------------------
# R-MAT (Chakrabarti et al.), Graph500-style parameters without noise
# ----------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, permute_seed: Optional[int] = None,
         symmetric: bool = True) -> CSR:
    """Seeded R-MAT graph with 2**scale vertices and edge_factor*2**scale tuples.

    For each of the ``scale`` bit levels every tuple picks a quadrant with
    probabilities a/b/c/d (d = 1-a-b-c); the result is symmetrised with
    self-loops and duplicate edges removed.  ``permute_seed`` relabels the
    vertices with a seeded random permutation ("perm" variants).
    """
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        u = rng.random(m, dtype=np.float32)
        bit = np.int64(1) << np.int64(scale - 1 - level)
        # quadrant: [0,a) -> (0,0); [a,a+b) -> (0,1); [a+b,a+b+c) -> (1,0); else (1,1)
        sbit = u >= ab
        dbit = ((u >= a) & (u < ab)) | (u >= abc)
        src += sbit * bit
        dst += dbit * bit
        del u, sbit, dbit
    name = f"rmat{scale}-ef{edge_factor}"
    if permute_seed is not None:
        p = np.random.default_rng(permute_seed).permutation(n).astype(np.int64)
        src, dst = p[src], p[dst]
        name += "-perm"
    return from_edges(n, src, dst, symmetric=symmetric, name=name)


# ----------------------------------------------------------------------------
# meshes and textbook families
# ----------------------------------------------------------------------------

def grid2d(rows: int, cols: int) -> CSR:
    """4-neighbour 2D grid, vertex id = r*cols + c (row-major)."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    right = (ids[:, :-1].ravel(), ids[:, 1:].ravel())
    down = (ids[:-1, :].ravel(), ids[1:, :].ravel())
    src = np.concatenate([right[0], down[0]])
    dst = np.concatenate([right[1], down[1]])
    return from_edges(rows * cols, src, dst, name=f"grid{rows}x{cols}")


def torus2d(rows: int, cols: int) -> CSR:
    """4-regular 2D torus (rows, cols >= 3)."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    src = np.concatenate([ids.ravel(), ids.ravel()])
    dst = np.concatenate([np.roll(ids, -1, axis=1).ravel(), np.roll(ids, -1, axis=0).ravel()])
    return from_edges(rows * cols, src, dst, name=f"torus{rows}x{cols}")


def complete(n: int) -> CSR:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, name=f"K{n}")


def path(n: int) -> CSR:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"P{n}")


def cycle(n: int) -> CSR:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"C{n}")


def star(n: int) -> CSR:
    """Star with centre 0 and n-1 leaves."""
    leaves = np.arange(1, n)
    return from_edges(n, np.zeros(n - 1, dtype=np.int64), leaves, name=f"S{n}")


def mycielski(k: int) -> CSR:
    """Mycielski graph M_k (M_2 = K_2) in its natural vertex order.

    M_{k+1} keeps the vertices v_0..v_{n-1} of M_k, adds shadows u_i = n+i and
    an apex w = 2n; each edge (v_i, v_j) adds (u_i, v_j) and (v_i, u_j), and
    every u_i is joined to w.  M_k is triangle-free and connected, with
    3*2**(k-2) - 1 vertices.
    """
    if k < 2:
        raise ValueError("k >= 2")
    src = np.array([0], dtype=np.int64)
    dst = np.array([1], dtype=np.int64)
    n = 2
    for _ in range(k - 2):
        u_src = np.concatenate([src + n, src])
        u_dst = np.concatenate([dst, dst + n])
        apex_src = np.arange(n, 2 * n, dtype=np.int64)
        apex_dst = np.full(n, 2 * n, dtype=np.int64)
        src = np.concatenate([src, u_src, apex_src])
        dst = np.concatenate([dst, u_dst, apex_dst])
        n = 2 * n + 1
    return from_edges(n, src, dst, name=f"mycielski{k}")


def disjoint_union(*graphs: CSR) -> CSR:
    offs = np.cumsum([0] + [g.n for g in graphs])
    srcs, dsts = [], []
    for off, g in zip(offs, graphs):
        rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
        srcs.append(rows + off)
        dsts.append(g.colind.astype(np.int64) + off)
    n = int(offs[-1])
    return from_edges(n, np.concatenate(srcs), np.concatenate(dsts), symmetric=False,
                      drop_self_loops=False, name="union")


def random_directed(n: int, density: float, seed: int, self_loops: bool = True) -> CSR:
    """Erdos-Renyi style directed 0/1 matrix (asymmetric), for brute-force checks."""
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < density
    if not self_loops:
        np.fill_diagonal(a, False)
    return from_dense(a, name=f"er{n}-{density}-{seed}")


def random_symmetric(n: int, density: float, seed: int) -> CSR:
    rng = np.random.default_rng(seed)
    a = np.triu(rng.random((n, n)) < density, 1)
    a = a | a.T
    return from_dense(a, name=f"ers{n}-{density}-{seed}")


def with_duplicates(g: CSR, seed: int, frac: float = 0.3) -> CSR:
    """Same pattern with some entries repeated and rows shuffled (unsorted CSR)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(g.n):
        c = g.colind[g.rowptr[i]:g.rowptr[i + 1]].tolist()
        extra = [x for x in c if rng.random() < frac]
        c = c + extra
        rng.shuffle(c)
        rows += [i] * len(c)
        cols += c
    counts = np.bincount(np.asarray(rows, dtype=np.int64), minlength=g.n)
    rowptr = np.zeros(g.n + 1, dtype=np.int32)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(g.n, rowptr, np.asarray(cols, dtype=np.int32), None, g.name + "-dup")


# ----------------------------------------------------------------------------
# edge weights, sources, vectors
# ----------------------------------------------------------------------------

def symmetric_weights(g: CSR, seed: int, lo: float = 1.0, hi: float = 100.0,
                      grid: Optional[int] = 16) -> np.ndarray:
    """fp32 weight per stored entry, equal for (i,j) and (j,i).

    With ``grid=16`` the weights are uniform on the 1/16 lattice in [lo, hi):
    every path sum below 2**20 is then exact in fp32.  ``grid=None`` draws
    continuous uniform weights.
    """
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    cols = g.colind.astype(np.int64)
    lo_id = np.minimum(rows, cols)
    hi_id = np.maximum(rows, cols)
    key = lo_id * np.int64(g.n) + hi_id
    order = np.argsort(key, kind="stable")
    sk = key[order]
    first = np.ones(sk.size, dtype=bool)
    if sk.size:
        np.not_equal(sk[1:], sk[:-1], out=first[1:])
    group = np.cumsum(first) - 1          # undirected edge id of each sorted entry
    nuniq = int(first.sum())
    if grid is None:
        w = rng.uniform(lo, hi, size=nuniq).astype(np.float32)
    else:
        steps = int(round((hi - lo) * grid))
        w = (lo + rng.integers(0, steps, size=nuniq) / grid).astype(np.float32)
    inv = np.empty(key.size, dtype=np.int64)
    inv[order] = group
    return w[inv].astype(np.float32)


def sources(g: CSR, count: int, seed: int) -> np.ndarray:
    """Seeded BFS sources drawn from vertices of degree > 0 (Graph500 style)."""
    rng = np.random.default_rng(seed)
    cand = np.nonzero(np.diff(g.rowptr) > 0)[0]
    if cand.size == 0:
        return np.zeros(count, dtype=np.int32)
    return cand[rng.integers(0, cand.size, size=count)].astype(np.int32)


def random_bits(n: int, density: float, seed: int) -> np.ndarray:
    """LSB-first uint32 bitset of n bits with the given fill density (bits >= n are 0)."""
    rng = np.random.default_rng(seed)
    b = rng.random(n) < density
    return pack_bits(b)


def pack_bits(b: np.ndarray) -> np.ndarray:
    """Pack a bool vector into LSB-first uint32 words (bit i of word w = element 32w+i)."""
    n = b.size
    words = (n + 31) // 32
    padded = np.zeros(words * 32, dtype=np.uint8)
    padded[:n] = b.astype(np.uint8)
    by = np.packbits(padded, bitorder="little")
    return by.view(np.uint32).copy() if by.size else np.zeros(0, dtype=np.uint32)


def unpack_bits(w: np.ndarray, n: int) -> np.ndarray:
    by = np.asarray(w, dtype=np.uint32).view(np.uint8)
    return np.unpackbits(by, bitorder="little")[:n].astype(bool)
