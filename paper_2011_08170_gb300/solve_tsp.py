"""The GD program of Section 5.1: a TSPLIB problem in, the F2M optimum out.

    python -m paper_2011_08170_gb300.solve_tsp problem.tsp [-k 10] [-o out.txt]
                                                [--pricing 1|2] [--no-pricing]

Reads the node coordinates (TSPLIB, EUC_2D), builds the k-nearest-neighbour
candidate graph on the GPU (Section 5.3), solves the fractional 2-matching LP
by GDP with pricing and the exact finisher, and writes the solution: one
line "u v x" per edge with x = 1 or x = 0.5 (TSPLIB node ids), after header
lines giving the optimum.  Every step is a call of this library's C ABI.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import (f2m_create, f2m_default_params, f2m_destroy, f2m_get_x, f2m_knn_csr,
               f2m_solve, read_tsplib)


def solve_file(path: str, k: int = 10, pricing: int = 1):
    """Returns (xy, info dict, edges int32 [m, 2] (0-based, u < v), x2 uint8 [m])."""
    xy, _ = read_tsplib(path)
    if xy.shape[0] <= k:
        raise ValueError(f"the problem has {xy.shape[0]} nodes; k must be below that")
    rp, col = f2m_knn_csr(xy, k)
    ctx = f2m_create(xy, rp, col, f2m_default_params(pricing=pricing))
    try:
        info = f2m_solve(ctx).as_dict()
        rp2, col2, x2, _ = f2m_get_x(ctx)
    finally:
        f2m_destroy(ctx)
    src = np.repeat(np.arange(xy.shape[0], dtype=np.int32), np.diff(rp2))
    keep = (src < col2) & (x2 > 0)
    return xy, info, np.stack([src[keep], col2[keep]], axis=1), x2[keep]


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("problem")
    ap.add_argument("-k", type=int, default=10, help="nearest neighbours per node in the candidate graph")
    ap.add_argument("-o", "--output", default="-")
    ap.add_argument("--pricing", type=int, default=1, choices=[1, 2])
    ap.add_argument("--no-pricing", action="store_true",
                    help="solve on the candidate graph only (no scan of all pairs)")
    a = ap.parse_args(argv)
    xy, info, edges, x2 = solve_file(a.problem, a.k, 0 if a.no_pricing else a.pricing)
    opt = info["bound2"] / (2.0 * (1 << info["frac_bits"]))
    out = sys.stdout if a.output == "-" else open(a.output, "w")
    try:
        out.write(f"# nodes {xy.shape[0]}\n# optimum {opt:.6f}\n")
        out.write(f"# certified {'all pairs' if info['certified'] == 2 else 'candidate graph'}\n")
        out.write(f"# edges with x = 1: {int(np.sum(x2 == 2))}, x = 1/2: {int(np.sum(x2 == 1))}\n")
        for (u, v), x in zip(edges.tolist(), x2.tolist()):
            out.write(f"{u + 1} {v + 1} {'1' if x == 2 else '0.5'}\n")
    finally:
        if out is not sys.stdout:
            out.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
