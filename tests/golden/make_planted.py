"""Writes tests/golden/planted_8x2p20.json: the CPU oracle's result on the planted-cut
workload at its full size (8 Erdos-Renyi blocks of 2^20 vertices, average degree 48,
64 bridges, weights uniform in [1, 100], generator seed 1), method seed 1, two
label-propagation rounds per level, n0 = 10000, eight Padberg-Rinaldi runs per level.

Only the oracle and the input generator run here (no GPU code); the oracle needs tens
of minutes at this size, so its result is stored once and the GPU test compares with
it.  The file holds the cut value, the whole contraction trace, the side bitmap's
SHA-256 and popcount, and a SHA-256 of the generated graph so that a test on another
host first checks that it draws the same graph.

    python tests/golden/make_planted.py [--out PATH]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

PARAMS = {"blocks": 8, "block_n": 1 << 20, "avg_deg": 48, "bridges": 64, "graph_seed": 1, "wlo": 1, "whi": 100,
          "seed": 1, "lp_iters": 2, "n0": 10000, "pr_runs_max": 8}


def graph_sha256(g) -> str:
    h = hashlib.sha256()
    for a in (g.offsets, g.adj, g.w):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def side_sha256(bits: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(bits, dtype=np.uint64).tobytes()).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "planted_8x2p20.json"))
    args = ap.parse_args()
    p = PARAMS
    g = gg.planted(p["blocks"], p["block_n"], p["avg_deg"], p["bridges"], p["graph_seed"], p["wlo"], p["whi"])
    t0 = time.time()
    ref = oracle.viecut(g.offsets, g.adj, g.w, seed=p["seed"], lp_iters=p["lp_iters"], n0=p["n0"],
                        pr_runs_max=p["pr_runs_max"])
    dt = time.time() - t0
    side = ref.side(g.n)
    out = {"params": p, "n": g.n, "nnz": g.nnz, "graph_sha256": graph_sha256(g), "cut": ref.cut,
           "trace": [list(s) for s in ref.trace], "side_sha256": side_sha256(ref.side_bits),
           "side_popcount": int(side.sum()), "oracle_seconds": round(dt, 1),
           "written_by": "tests/golden/make_planted.py (CPU oracle only)"}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"cut {ref.cut}, {len(ref.trace)} steps, {dt:.0f} s -> {args.out}")


if __name__ == "__main__":
    main()
