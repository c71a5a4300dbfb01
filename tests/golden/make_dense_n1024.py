"""Writes tests/golden/dense_n1024.json: for the dense single-layer kernel on
1024 Fibonacci-sphere points (rotation seed 3000, probe seed 3001, circle
centre 3, radius 1, N = 32, L = 16) the number of eigenvalues inside the
circle by the argument principle (winding number of det T(z) on the circle),
and the oracle's RSRR eigenvalues and residuals (Section 4.3, Taylor
projection of the kernel).  Calls only oracle/ and workloads/."""
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
    p = W.helmholtz_sphere(n=1024, N=32, L=16)
    t0 = time.time()
    count = oracle.argument_principle_count_dense(p, npts=2048)
    t1 = time.time()
    out = oracle.rsrr_dense(p, NQ=500)
    t2 = time.time()
    lam = out["lam"]
    assert len(lam) == count, (len(lam), count)
    gold = {
        "workload": "dense kernel exp(i z r)/(4 pi r), n = 1024 Fibonacci sphere, rotation seed 3000, "
                    "probe seed 3001, circle centre 3 radius 1, N = 32, L = 16, NQ = 500",
        "source": "tests/golden/make_dense_n1024.py (oracle only)",
        "count_in_region": int(count),
        "count_cite": "argument principle: winding number of det T(z) along the circle",
        "oracle_rsrr_eigenvalues": [[float(z.real), float(z.imag)] for z in lam],
        "oracle_rsrr_residuals": [float(r) for r in out["res"]],
        "oracle_rsrr_k": int(out["k"]),
        "seconds": {"argument_principle": round(t1 - t0, 1), "rsrr": round(t2 - t1, 1)},
    }
    with open(os.path.join(HERE, "dense_n1024.json"), "w") as f:
        json.dump(gold, f, indent=1)
    print(json.dumps(gold, indent=1))


if __name__ == "__main__":
    main()
