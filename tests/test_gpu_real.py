"""GPU parity of the real-arithmetic path (RSRR_FLAG_REAL), through the C ABI.

A real NEP sampled at real points (Chebyshev points of the first kind on an
interval, Section 5.1) has real T(z_j): the library then factors and solves in
real arithmetic (float for the mixed path, double for the FP64 path) with the
same FP64 refinement.  Checked against the oracle's complex solves with the
same real probe, against the complex path on the same handle inputs, and the
eigenvalues against Sylvester inertia bisection (the loaded string of
Section 5.1 and the grid rational workload at full size, whose eigenvalues
tests/golden/make_c1_eigs.py fixes from the oracle alone)."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from util import match_eigs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ETA_TOL = 1e-10
EIG_TOL = 1e-9
RES_TOL = 1e-10


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


def string(N, L):
    s = W.loaded_string(N=N, L=L)
    s.region = W.Region(5001.5, 4998.5, 0.1 * 4998.5, kind="interval")
    s.U = np.asfortranarray(s.U.real.astype(np.complex128))  # the real path's probe is real
    return s


@pytest.fixture(scope="module")
def exact_string():
    return oracle.bisect_real_eigenvalues(string(100, 1), 3.0, 1e4).astype(complex)


def run(rs, p, project=True, **kw):
    s = rs.Solver(p, rs.default_opts(**kw))
    s.sample()
    s.check()
    out = dict(S=s.samples(), eta=s.eta(), stats=s.stats())
    if project:
        s.project()
        out.update(s.solve())
    s.close()
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_real_samples_match_the_oracle_and_the_complex_path(rs, prec):
    p = string(100, 4)
    precision = rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64
    re = run(rs, p, project=False, precision=precision, flags=rs.RSRR_FLAG_REAL)
    cx = run(rs, p, project=False, precision=precision)
    S = re["S"]
    assert np.all(S.imag == 0)
    assert re["eta"].max() <= (ETA_TOL if prec == "mixed" else 1e-14)
    zo = oracle.sample_points(p.region, p.N)
    for j in (0, 37, 99):
        Xr = oracle.resolvent_samples(p, zo[j:j + 1])[0]
        Xg = S[:, j * p.L:(j + 1) * p.L]
        assert oracle.backward_error_inf(p, zo[j], Xg).max() <= (ETA_TOL if prec == "mixed" else 1e-14)
        assert np.abs(Xg - Xr).max() <= (1e-6 if prec == "mixed" else 1e-9) * np.abs(Xr).max()
    # the complex path on the same real inputs: the same samples to the accuracy of either
    assert np.abs(S - cx["S"]).max() <= (1e-6 if prec == "mixed" else 1e-9) * np.abs(S).max()
    assert re["stats"]["device_bytes"] < cx["stats"]["device_bytes"]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_real_path_finds_the_string_eigenvalues(rs, exact_string, prec):
    """Section 5.2: L = 1, N = 100 Chebyshev points, SS-FULL with K_Q = 8."""
    precision = rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64
    out = run(rs, string(100, 1), NQ=500, KQ=8, precision=precision, flags=rs.RSRR_FLAG_REAL)
    assert len(out["lam"]) == 32
    assert match_eigs(exact_string, out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL


def test_real_path_with_streaming_and_one_kernel_solves_agree(rs):
    p = string(40, 8)
    a = run(rs, p, project=False, flags=rs.RSRR_FLAG_REAL)
    b = run(rs, p, project=False, flags=rs.RSRR_FLAG_REAL | rs.RSRR_FLAG_PLAIN_SOLVE | rs.RSRR_FLAG_ONE_CTA_LU)
    assert a["eta"].max() <= ETA_TOL and b["eta"].max() <= ETA_TOL
    assert np.abs(a["S"] - b["S"]).max() <= 1e-6 * np.abs(a["S"]).max()


def test_real_path_refusals_on_the_device_handle(rs):
    p = string(16, 2)
    s = rs.Solver(p, rs.default_opts(flags=rs.RSRR_FLAG_REAL))
    s.sample()
    s.check()
    with pytest.raises(rs.RSRRError) as e:
        s.add_points([500.0])
    assert e.value.status == rs.RSRR_EINVAL
    with pytest.raises(rs.RSRRError) as e:
        rs.sample_batch([s])
    assert e.value.status == rs.RSRR_EINVAL
    s.close()


def test_full_size_grid_on_interval_points_matches_sylvester_inertia(rs):
    """The grid rational workload (n = 40000, half-bandwidth 200, N = 64,
    L = 32) sampled at Chebyshev points of [20, 180] in real arithmetic; the
    ten eigenvalues there against the band-LDL^T bisection, on the FP64
    path.  Real points sit on the spectrum's line, 0.13 from the nearest
    eigenvalue here: cond(T(z_j)) is about 2.5e6, and with a half-bandwidth of
    200 a float factorisation's error times that condition is above one, so
    the mixed path's refinement does not contract there (it stops with
    ENOCONV, which the second half checks)."""
    g = json.load(open(os.path.join(GOLD, "c1_eigs.json")))
    p = W.config("c1")
    p.region = W.Region(100.0, 80.0, 20.0, kind="interval")
    p.U = np.asfortranarray(p.U.real.astype(np.complex128))
    out = run(rs, p, precision=rs.RSRR_PREC_FP64, flags=rs.RSRR_FLAG_REAL)
    # an FP64 band LU's backward error grows with the bandwidth (about 200 u
    # here, 2e-14, times the pivot growth)
    assert out["eta"].max() <= 1e-12
    bis = np.array(g["bisection_eigenvalues"]).astype(complex)
    assert len(out["lam"]) == g["count_in_region"] == len(bis)
    assert match_eigs(bis, out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual(p, lam, v) <= RES_TOL
    # the mixed path at the same points: the refinement's failure is reported
    s = rs.Solver(p, rs.default_opts(flags=rs.RSRR_FLAG_REAL))
    s.sample()
    assert s.check_status() == rs.RSRR_ENOCONV
    s.close()
