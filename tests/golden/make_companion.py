"""Writes c0_companion.json: eigenvalues of the n=1000 quadratic workload
(benchmark recipe: K = n*tridiag(-1,2,-1), M = tridiag(1,4,1)/(6n), C = diag(u),
u ~ U[0, 0.1] seed 1000) from the oracle's companion linearisation, restricted
to the two circles used by the tests (centre 50 radius 40, and centre
-25+50i radius 40), plus the smallest relative distance of any eigenvalue to
each circle.  Run from the repository root:  python tests/golden/make_companion.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    p = workloads.config("c0")
    ev = oracle.companion_eigvals(p)
    out = {"recipe": "workloads.config('c0') (n=1000, seed_c=1000)", "circles": []}
    for center, r in ((50.0 + 0.0j, 40.0), (-25.0 + 50.0j, 40.0)):
        rel = np.abs(ev - center) / r - 1.0
        ins = ev[rel < 0]
        out["circles"].append({
            "center": [center.real, center.imag], "radius": r,
            "inside": [[z.real, z.imag] for z in ins],
            "min_rel_boundary_distance": float(np.min(np.abs(rel))),
        })
    with open(os.path.join(os.path.dirname(__file__), "c0_companion.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
