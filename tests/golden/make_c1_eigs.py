"""Writes tests/golden/c1_eigs.json: the eigenvalues of the full-size grid
rational workload (200 x 200 five-point grid, n = 40000, T(z) = K - z M +
z/(z - 300) E, ellipse centre 100, semi-axes 80 / 20, N = 64, L = 32) from
two oracle routes that share no arithmetic:

  * Sylvester inertia: T(x) is real symmetric for real x and T'(x) =
    -M - 300/(x - 300)^2 E is negative definite, so the number of eigenvalues
    in (a, b) is nu(T(b)) - nu(T(a)) (negative pivots of a band LDL^T), and
    bisection on nu gives every eigenvalue in (20, 180), the real interval the
    ellipse encloses;
  * the oracle's RSRR (Section 4.3 steps 1-5) on the same workload.

Calls only oracle/ and workloads/.  Takes several minutes on a few cores."""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle            # noqa: E402
import workloads as W    # noqa: E402


def main():
    p = W.config("c1")
    lo, hi = 20.0, 180.0
    t0 = time.time()
    count = oracle.negative_inertia_band(p, hi) - oracle.negative_inertia_band(p, lo)
    bis = oracle.bisect_real_eigenvalues(p, lo, hi, rtol=1e-13)
    t1 = time.time()
    out = oracle.rsrr(p)
    t2 = time.time()
    lam = out["lam"]
    order = np.argsort(lam.real)
    lam, res = lam[order], out["res"][order]
    assert len(bis) == count == len(lam), (len(bis), count, len(lam))
    err = np.max(np.abs(lam - bis) / np.abs(bis))
    gold = {
        "workload": "grid rational NEP, g = 200 (n = 40000), sigma = 300, E positions seed 2000, "
                    "U seed 2001, ellipse centre 100 semi-axes 80/20, N = 64, L = 32",
        "source": "tests/golden/make_c1_eigs.py (oracle only)",
        "count_in_region": int(count),
        "count_cite": "Sylvester inertia nu(T(180)) - nu(T(20)), band LDL^T (oracle/band_inertia.c)",
        "bisection_eigenvalues": [float(x) for x in bis],
        "bisection_rtol": 1e-13,
        "oracle_rsrr_eigenvalues": [[float(z.real), float(z.imag)] for z in lam],
        "oracle_rsrr_residuals": [float(r) for r in res],
        "oracle_rsrr_k": int(out["k"]),
        "oracle_vs_bisection_max_rel": float(err),
        "seconds": {"inertia": round(t1 - t0, 1), "rsrr": round(t2 - t1, 1)},
    }
    with open(os.path.join(HERE, "c1_eigs.json"), "w") as f:
        json.dump(gold, f, indent=1)
    print(json.dumps(gold, indent=1))


if __name__ == "__main__":
    main()
