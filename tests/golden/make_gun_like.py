"""Writes tests/golden/gun_like.json from the oracle alone: the gun-type NEP
of workloads.gun_like (Section 5.4's T(z) = K - z^2 M + i sqrt(z^2) W_1 +
i sqrt(z^2 - kappa_2^2) W_2, synthetic, n = 10^4, half-bandwidth 100) on the
rectangle [215, 330] x [-10, 40]:

* the number of eigenvalues inside by the argument principle along the
  rectangle (phase of det T from banded LU, refined until every step is
  below pi/4);
* RSRR with N = 80 Gauss-Legendre points (27 / 13 per side), L = 2,
  N_Q = 500 composite Gauss nodes, K_Q = 2 (the paper's "contour" run);
* the two-stage run: 30 points (10 / 5 per side), then its eigenvalues added
  as sampling points (the paper's "adapt" run).

Run: python tests/golden/make_gun_like.py   (about a minute on one core)"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def pairs(z):
    return [[float(v.real), float(v.imag)] for v in np.asarray(z)]


def main():
    t0 = time.time()
    p = W.gun_like()
    reg = p.region
    count = oracle.argument_principle_count(p, reg, npts=256, band=True)
    t_count = time.time() - t0
    full = oracle.rsrr(p, NQ=500, KQ=2)
    t_full = time.time() - t0 - t_count
    s1 = W.gun_like(N=30, nx=10)
    st1 = oracle.rsrr(s1, NQ=500, KQ=2)
    z2 = np.concatenate([oracle.sample_points(s1.region, 30), st1["lam"]])
    s2 = W.gun_like(N=len(z2), nx=10)
    s2.region = W.Region(reg.center, reg.a, reg.b, kind="rect", nx=10, points=z2)
    st2 = oracle.rsrr(s2, NQ=500, KQ=2)
    out = {
        "workload": "gun-type NEP, grid 100 x 100 (n = 10000), alpha 2405, beta 3295, w1 = w2 = 1e4, "
                    "kappa2 108.8774, U seed 9001, rectangle [215, 330] x [-10, 40]",
        "source": "tests/golden/make_gun_like.py (oracle only)",
        "count_in_region": count,
        "count_cite": "argument principle along the rectangle, phase of det T from banded LU",
        "contour_N80_L2": {"eigenvalues": pairs(full["lam"]), "residuals": full["res"].tolist(),
                           "k": int(full["k"])},
        "stage1_N30_L2": {"eigenvalues": pairs(st1["lam"]), "residuals": st1["res"].tolist()},
        "stage2_points": pairs(z2),
        "stage2_L2": {"eigenvalues": pairs(st2["lam"]), "residuals": st2["res"].tolist(),
                      "k": int(st2["k"])},
        "seconds": {"count": round(t_count, 1), "contour": round(t_full, 1)},
    }
    with open(os.path.join(HERE, "gun_like.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(count, len(full["lam"]), len(st1["lam"]), len(st2["lam"]), max(full["res"]), max(st2["res"]))


if __name__ == "__main__":
    main()
