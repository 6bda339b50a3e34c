"""Writes tests/golden/graphs.json.

Uses only the seeded input generators (graphgen) and the oracle: for each
small graph it stores the CSR's SHA-256 and size, and for each of a few
sources the SHA-256 of the oracle's int32 distance array together with the
reached count and eccentricity.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402
import oracle  # noqa: E402

CALLS = {
    "rmat_s12": "rmat(12, 16, 0.57, 0.19, 0.19, 1, 1)",
    "rmat_s16": "rmat(16, 16, 0.57, 0.19, 0.19, 1, 1)",
    "er_2e14_d16": "erdos_renyi(16384, 16.0, 2)",
    "grid_64x64": "grid2d(64, 64)",
    "rgg_2e14_d3": "rgg(16384, 0.007634414248483124, 3)",
}


def main():
    out = {"note": "written by tests/golden/make_golden.py from graphgen + oracle only", "graphs": {}}
    for name, call in CALLS.items():
        rp, col = eval("graphgen." + call)
        srcs = graphgen.sources(rp, 4, 1001)
        rec = {"call": call, "n": int(len(rp) - 1), "m": int(len(col)),
               "csr_sha256": graphgen.csr_sha256(rp, col), "sources": [int(s) for s in srcs], "dist": []}
        for s in srcs:
            d = oracle.bfs(rp, col, int(s))
            rec["dist"].append({"sha256": hashlib.sha256(d.astype(np.int32).tobytes()).hexdigest(),
                                "reached": int((d >= 0).sum()), "eccentricity": int(d.max())})
        out["graphs"][name] = rec
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "graphs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
