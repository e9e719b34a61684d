"""GB300-native B2SR bit-graph library (Bit-GraphBLAS, arXiv 2201.08560)."""
