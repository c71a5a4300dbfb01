"""GPU parity of the comparison methods on the same resident samples, through
the C ABI: SS-RI (Section 3.3) and SSRR-M (Section 4.1) against the oracle's
versions and against exact eigenvalues (Sylvester inertia bisection, closed
forms), on the paper's loaded string with Chebyshev points of the first kind
on the interval [3, 1e4] (RSRR_REGION_INTERVAL, Section 5.1) and on a
decoupled closed-form family."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_pins import exact_roots
from util import match_eigs

pytestmark = pytest.mark.gpu


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
    return s


@pytest.fixture(scope="module")
def exact_string():
    return oracle.bisect_real_eigenvalues(string(200, 10), 3.0, 1e4).astype(complex)


def run(rs, p, project=True, **kw):
    s = rs.Solver(p, rs.default_opts(**kw))
    s.sample()
    s.check()
    z = s.points()
    if project:
        s.project()
    out = s.solve()
    s.close()
    out["z"] = z
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ss_ri_on_the_loaded_string(rs, exact_string, prec):
    """Section 5.1: L = K = 10, N = 200 Chebyshev points: the 32 eigenvalues."""
    p = string(200, 10)
    precision = rs.RSRR_PREC_FP64 if prec == "fp64" else rs.RSRR_PREC_MIXED
    # SS-RI's moments amplify the samples' errors by the condition of T(z_i)
    # at Chebyshev points that fall close to eigenvalues (up to ~1e6 here):
    # the mixed-precision samples are refined to a backward error of 1e-14
    # instead of the usual 1e-10 (complex64 refinement reaches it)
    kw = {} if prec == "fp64" else dict(eta_tol=1e-14, max_refine=24)
    out = run(rs, p, project=False, method=rs.RSRR_METHOD_SS_RI, K=10, precision=precision, **kw)
    assert np.abs(out["z"] - oracle.sample_points(p.region, p.N)).max() <= 1e-11
    assert len(out["lam"]) == 32
    assert match_eigs(exact_string, out["lam"]) <= (1e-9 if prec == "fp64" else 1e-7)
    if prec == "fp64":
        ref = oracle.ss_ri(p, K=10)
        assert match_eigs(ref["lam"], out["lam"]) <= 1e-9
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.plain_residual(p, lam, v) <= 1e-8


def test_rsrr_on_interval_points_finds_the_string_eigenvalues(rs, exact_string):
    """Section 5.2: L = 1, N = 100 Chebyshev points, SS-FULL with K_Q = 8."""
    out = run(rs, string(100, 1), NQ=500, KQ=8)
    assert len(out["lam"]) == 32
    assert match_eigs(exact_string, out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10


def test_ssrr_m_loses_eigenvalues_where_rsrr_does_not(rs, exact_string):
    """Section 5.2: with L = 1 and K = N = 100 the moment scheme's M loses rank;
    the oracle's SSRR-M and the library's agree on missing eigenvalues."""
    out = run(rs, string(100, 1), NQ=500, KQ=8, method=rs.RSRR_METHOD_SSRR_M, K=100)
    ref = oracle.ssrr_m(string(100, 1), K=100, NQ=500, KQ=8)
    assert len(ref["lam"]) < 32
    assert len(out["lam"]) < 32 or match_eigs(exact_string, out["lam"]) > 1e-6


@pytest.mark.parametrize("name", ["diag_quadratic", "diag_rational"])
def test_ssrr_m_matches_closed_form_and_oracle(rs, name):
    p = getattr(W, name)(N=48, L=8)
    out = run(rs, p, NQ=256, method=rs.RSRR_METHOD_SSRR_M, K=6)
    ref = exact_roots(p)
    assert len(out["lam"]) == len(ref)
    assert match_eigs(ref, out["lam"]) <= 1e-9
    assert match_eigs(oracle.ssrr_m(p, K=6, NQ=256)["lam"], out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
