"""GB300-native B2SR bit-graph library (Bit-GraphBLAS, arXiv 2201.08560).

``paper_2201_08560_gb300.binding`` is the ctypes binding of the CUDA library
(loaded on first use, so that importing the seeded generators in
``paper_2201_08560_gb300.graphs`` needs no GPU); ``build`` compiles it.
"""
import importlib

__all__ = ["binding", "graphs", "build"]


def __getattr__(name):
    if name in ("binding", "graphs", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
