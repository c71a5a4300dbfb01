"""Parity at the benchmark sizes, through the C ABI.

* Grid rational workload at full size (n = 40000, half-bandwidth 200, N = 64,
  L = 32; the configuration bench.py times): the whole method -- sampling,
  the multi-level Gram basis, the projection, SS-FULL -- against eigenvalues
  that Sylvester inertia fixes (band LDL^T counts and bisection, written by
  tests/golden/make_c1_eigs.py from the oracle alone).
* Dense kernel at full size (n = 4096, N = 32, L = 64): every column's
  backward error, and two sampling points' X element by element against the
  oracle's dense LAPACK solves.
* Dense kernel at n = 1024: the eigenvalue count against the argument
  principle and the eigenvalues against the oracle's RSRR
  (tests/golden/make_dense_n1024.py)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from util import match_eigs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EIG_TOL = 1e-9   # relative eigenvalue agreement
RES_TOL = 1e-10  # normalised residual of every eigenpair
ETA_TOL = 1e-10  # per-column backward error of the mixed-precision samples


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_full_size_grid_rational_eigenpairs_match_sylvester_inertia(rs):
    g = _gold("c1_eigs.json")
    p = W.config("c1")
    s = rs.Solver(p, rs.default_opts())
    s.sample()
    s.check()
    assert s.eta().max() <= ETA_TOL
    s.project()
    out = s.solve()
    st = s.stats()
    s.close()
    bis = np.array(g["bisection_eigenvalues"])
    assert len(out["lam"]) == g["count_in_region"] == len(bis)
    assert match_eigs(bis.astype(complex), out["lam"]) <= EIG_TOL
    ref = np.array([complex(*z) for z in g["oracle_rsrr_eigenvalues"]])
    assert match_eigs(ref, out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual(p, lam, v) <= RES_TOL
    assert st["k"] >= g["count_in_region"]


def test_full_size_dense_kernel_sampled_parity(rs):
    p = W.helmholtz_sphere(n=4096, N=32, L=64)
    s = rs.Solver(p, rs.default_opts())
    s.sample()
    assert s.check_status() == rs.RSRR_OK
    eta = s.eta()
    assert eta.max() <= ETA_TOL
    S = s.samples()
    s.close()
    zo = oracle.sample_points(p.region, p.N)
    for j in (0, 19):
        Xr = oracle.resolvent_samples_dense(p, zo[j:j + 1])[0]
        Xg = S[:, j * p.L:(j + 1) * p.L]
        e = oracle.backward_error_inf_dense(p, zo[j], Xg)
        assert e.max() <= ETA_TOL
        assert np.allclose(eta[j * p.L:(j + 1) * p.L], e, rtol=1e-3, atol=1e-14)
        assert np.abs(Xg - Xr).max() <= 1e-6 * np.abs(Xr).max()


def test_dense_kernel_n1024_count_and_eigenvalues(rs):
    g = _gold("dense_n1024.json")
    p = W.helmholtz_sphere(n=1024, N=32, L=16)
    s = rs.Solver(p, rs.default_opts(NQ=500))
    s.sample()
    s.check()
    s.project()
    out = s.solve()
    s.close()
    assert len(out["lam"]) == g["count_in_region"]
    ref = np.array([complex(*z) for z in g["oracle_rsrr_eigenvalues"]])
    assert match_eigs(ref, out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual_dense(p, lam, v) <= RES_TOL
