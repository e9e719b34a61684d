"""Helpers shared by the GPU parity tests (device transfer, graph fixtures).

Unsigned bitsets travel as int32 tensors (torch has no uint32 arithmetic on
every supported version); the bits are reinterpreted, never converted.
"""
import functools

import numpy as np
import pytest
import torch

from paper_2201_08560_gb300 import graphs


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch.device("cuda", 0)


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a.copy()).to(dev())


def to_np(t: torch.Tensor, dtype=None) -> np.ndarray:
    a = t.detach().cpu().numpy()
    if dtype is not None:
        a = a.view(dtype)
    return a


def csr_dev(g):
    return to_dev(g.rowptr.astype(np.int32)), to_dev(g.colind.astype(np.int32) if g.colind.size else
                                                       np.zeros(0, np.int32))


@functools.lru_cache(maxsize=1)
def small_graphs():
    """Edge cases of the tile walk: ragged n, empty leading/trailing/inner rows,
    rows spanning many chunks, a single vertex, no edges, asymmetric."""
    out = []
    out.append(graphs.rmat(12, 16, seed=1))                     # the 4096-vertex R-MAT workload
    out.append(graphs.rmat(11, 8, seed=3, permute_seed=4))      # permuted ids
    out.append(graphs.star(20000))                              # one row spans many chunks
    out.append(graphs.grid2d(37, 41))                           # n = 1517, not a multiple of any k
    u = graphs.disjoint_union(graphs.from_dense(np.zeros((70, 70))), graphs.complete(40),
                              graphs.from_dense(np.zeros((300, 300))), graphs.cycle(33),
                              graphs.from_dense(np.zeros((90, 90))))
    u.name = "gaps"
    out.append(u)                                               # empty leading/inner/trailing tile-rows
    out.append(graphs.random_directed(300, 0.05, seed=9))       # asymmetric, with self-loops
    out.append(graphs.from_dense(np.ones((1, 1))))              # n = 1
    out.append(graphs.from_dense(np.zeros((45, 45))))           # no edges (T = 0)
    out.append(graphs.mycielski(9))
    return tuple(out)


GRAPH_IDS = ["rmat12", "rmat11perm", "star20k", "grid37x41", "gaps", "directed300", "n1", "empty45",
             "mycielski9"]
