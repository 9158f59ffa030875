"""Writes tests/golden/optimal_costs.json: exact optimal costs of seeded
instances, computed only by the oracle's Hungarian method (with its dual
certificate checked), plus SHA-256 digests of the generated int32 matrices
so that a platform whose generator drifted is caught before any parity claim.

Run: python tests/golden/make_golden.py   (about two minutes on one core)
"""

import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1110_6231_gb300 import synth  # noqa: E402

CASES = (
    [("uniform-n256-c1000", s, None) for s in range(100)]
    + [("uniform-n4096-c2^20", s, None) for s in range(10)]
    + [("geometric-n8192", s, 1024) for s in range(4)]
    + [("geometric-n8192", s, None) for s in range(8)]    # the full n = 8192 workload
)


def digest(C):
    return hashlib.sha256(C.tobytes()).hexdigest()


def main():
    out = []
    for name, seed, n in CASES:
        C = synth.instance(name, seed, n)
        cost, match, u, v = oracle.hungarian(C)
        assert oracle.check_duals(C, match, u, v) == 0
        out.append(dict(workload=name, seed=seed, n=int(C.shape[0]), cost=cost, sha256=digest(C)))
        print(name, seed, C.shape[0], cost, flush=True)
    with open(os.path.join(HERE, "optimal_costs.json"), "w") as f:
        json.dump({"source": "oracle.hungarian (dual certificate checked)", "cases": out}, f, indent=1)


if __name__ == "__main__":
    main()
