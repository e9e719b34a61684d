"""Writes fullsize_tc.json: the oracle's triangle count of the full-size
triangle-counting workload (R-MAT scale 18, edge factor 32, seed 2), with the
input's sizes and a digest of its CSR so that a test can check it is counting
the same graph.  Calls only the oracle and the seeded generator.

    python tests/golden/make_fullsize_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2201_08560_gb300 import graphs  # noqa: E402

SCALE, EF, SEED = 18, 32, 2


def csr_digest(g):
    h = hashlib.sha256()
    h.update(g.rowptr.astype("<i8").tobytes())
    h.update(g.colind.astype("<i4").tobytes())
    return h.hexdigest()


def main():
    g = graphs.rmat(SCALE, EF, seed=SEED)
    out = {"workload": f"R-MAT scale {SCALE} ef{EF} seed {SEED}, symmetrised, no self-loops/duplicates",
           "n": int(g.n), "nnz": int(len(g.colind)), "csr_sha256": csr_digest(g),
           "triangles": int(oracle.triangle_count(g)), "source": "oracle.triangle_count (sorted-merge count over L)"}
    with open(os.path.join(HERE, "fullsize_tc.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
