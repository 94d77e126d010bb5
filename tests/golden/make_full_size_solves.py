"""Writes full_size_solves.json: the CPU oracle's solves of the full-size
single-instance workloads, at the default of 128 sweeps per GDP phase.

Calls only the oracle (and the seeded instance generator).  Two solves per
instance:
  before_finisher: the solve with the finisher off, which stops at the first
    rule (7) extraction that leaves a row off -- every step up to there (GDP
    phases, pricing scans, merges, the sign rule) is the same integer algorithm
    in the library, so the GPU test compares its counters, bound and SHA-256
    digests of the candidate graph, x and lambda bit for bit;
  solve: the complete solve with the oracle's plain min-cost-flow finisher --
    its lambda and x are one optimum among several, so only the counters and
    the optimum (bound2 at frac_bits) are kept; oracle_seconds is its time.
One complete oracle solve takes about a minute (n = 100,000) and several
minutes (n = 200,000) on one core.

    python tests/golden/make_full_size_solves.py [name ...]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import instances as I  # noqa: E402
import oracle  # noqa: E402

CASES = {
    "uniform_n100000_k10_seed0": ("uniform", 100_000, 0, 10),
    "mixture_n200000_k12_seed0": ("mixture", 200_000, 0, 12),
}
MAX_ITERS = 128
OUT = os.path.join(HERE, "full_size_solves.json")


def digest(a, dtype):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def record(kind, n, seed, k):
    d = I.make_instance(kind, n, seed, k)
    rec = {"kind": kind, "n": n, "seed": seed, "k": k, "max_iters": MAX_ITERS}
    b = oracle.solve(d["xy"], d["row_ptr"], d["col"], max_iters=MAX_ITERS, finisher=False)
    bf = {f: int(getattr(b, f)) for f in ("status", "iterations", "phases", "pricing_rounds",
                                          "edges_added", "bound2", "frac_bits")}
    bf["nnz"] = int(b.row_ptr[-1])
    bf["sha256"] = {"row_ptr": digest(b.row_ptr, "<i4"), "col": digest(b.col, "<i4"),
                    "x2": digest(b.x2, "u1"), "lam": digest(b.lam, "<i4")}
    rec["before_finisher"] = bf
    t = time.time()
    r = oracle.solve(d["xy"], d["row_ptr"], d["col"], max_iters=MAX_ITERS)
    rec["oracle_seconds"] = round(time.time() - t, 1)
    sv = {f: int(getattr(r, f)) for f in ("status", "iterations", "phases", "pricing_rounds",
                                          "edges_added", "finisher_calls", "augmentations", "bound2",
                                          "frac_bits", "certified")}
    sv["nnz"] = int(r.row_ptr[-1])
    rec["solve"] = sv
    return rec


def main(names):
    oracle.build()
    out = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names or list(CASES):
        out[name] = record(*CASES[name])
        print(name, out[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
