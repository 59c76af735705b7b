"""Writes planted21_noi.json: the oracle's exact minimum cut of the planted
configuration (two G(2^21, avg degree 42) blocks, each cut to its 30-core,
joined by 25 unit cross edges; seed 3), computed by the oracle's sequential
NOI (Algorithm 2 with one CAPFOREST pass per round, App. B) on one core.

Only the generator and the oracle run here; no GPU code is involved.  The
graph is identified by its size and a checksum of its CSR so that a later
change of the generator invalidates the stored value.  Run from the
repository root:  python tests/golden/make_planted21_golden.py  (about two
minutes of CPU and 4 GB of RAM)."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.graphs import csr_checksum  # noqa: E402


def main() -> None:
    g = synth.workload_planted(21, 42, 30, 25, 3)
    block = np.asarray(g.meta["block"], dtype=np.uint8)
    t0 = time.time()
    lam, side, rounds = oracle.noi(g.n, g.row_ptr, g.col, g.w)
    secs = time.time() - t0
    side = np.asarray(side, dtype=np.uint8)
    cut = oracle.cut_weight(g.n, g.row_ptr, g.col, g.w, side)
    split = bool(np.array_equal(side, block) or np.array_equal(side, 1 - block))
    out = {
        "config": "planted cut: two G(2^21, avg degree 42) blocks, 30-cores, 25 unit cross edges, seed 3",
        "generator": "synth.workload_planted(21, 42, 30, 25, 3)",
        "n": int(g.n),
        "m": int(g.m),
        "csr_checksum": csr_checksum(g),
        "lambda": int(lam),
        "oracle": "oracle.noi (sequential NOI, Algorithm 2 with one CAPFOREST pass per round)",
        "oracle_rounds": int(rounds),
        "oracle_seconds_one_core": round(secs, 1),
        "side_sizes": [int(g.n - side.sum()), int(side.sum())],
        "side_cut_weight": int(cut),
        "side_is_block_split": split,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "planted21_noi.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
