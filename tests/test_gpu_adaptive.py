"""Two-stage sampling through the C ABI (rsrr_add_points; Section 5.4): a
first solve with few contour points gives rough eigenvalues, which become new
sampling points; only they are sampled, the first stage's samples stay
resident and bit for bit unchanged, and the second solve on all points
matches the oracle run on the same points (and the closed-form roots)."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_pins import exact_roots
from util import match_eigs

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-9
RES_TOL = 1e-10
ETA_TOL = 1e-10


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


@pytest.mark.parametrize("name,N1,prec", [("diag_quadratic", 10, "mixed"), ("diag_rational", 10, "mixed"),
                                          ("diag_rational", 10, "fp64")])
def test_second_stage_reuses_the_first_samples_and_matches_the_oracle(rs, name, N1, prec):
    p = getattr(W, name)(N=N1)
    precision = rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64
    # stage 1: rough eigenvalues from N1 contour points (loose acceptance).
    # Samples at points close to eigenvalues are dominated by one eigenvector,
    # and a backward error eta leaves an error of about eta / dist in the
    # components that carry the others, so the refinement target is tighter
    # than the usual 1e-10 (complex64 refinement reaches it in a few sweeps).
    s = rs.Solver(p, rs.default_opts(NQ=256, res_tol=1e-2, precision=precision, eta_tol=1e-13,
                                     max_refine=16))
    s.sample()
    s.check()
    S1 = s.samples()
    s.project()
    lam1 = s.solve()["lam"]
    assert len(lam1) > 0
    # stage 2: the eigenvalues become sampling points; only they are sampled
    s.add_points(lam1)
    assert s.check_status() == rs.RSRR_OK
    z2 = s.points()
    S2 = s.samples()
    eta = s.eta()
    s.project()
    out = s.solve()
    st = s.stats()
    s.close()
    assert st["N"] == N1 + len(lam1) == len(z2)
    assert np.array_equal(S2[:, :N1 * p.L], S1)          # the first stage's samples, untouched
    assert eta.max() <= (1e-13 if prec == "mixed" else 1e-14)
    # the new points' samples against the oracle: backward error at the
    # acceptance level (the points sit near eigenvalues, so T(z) is
    # ill-conditioned there and the forward error is larger by its condition)
    Xr = oracle.resolvent_samples(p, z2[N1:N1 + 2])
    for q, X in enumerate(Xr):
        Xg = S2[:, (N1 + q) * p.L:(N1 + q + 1) * p.L]
        assert oracle.backward_error_inf(p, z2[N1 + q], Xg).max() <= ETA_TOL
        assert np.abs(Xg - X).max() <= 1e-3 * np.abs(X).max()
    # the whole second stage against the oracle on the same points
    q = getattr(W, name)(N=len(z2))
    q.region = W.Region(p.region.center, p.region.a, p.region.b, kind="points", points=z2)
    ref = oracle.rsrr(q, NQ=256, res_tol=1e-2)
    assert len(out["lam"]) == len(ref["lam"]) == len(exact_roots(p))
    assert match_eigs(ref["lam"], out["lam"]) <= EIG_TOL
    assert match_eigs(exact_roots(p), out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL


def test_add_points_before_sampling_is_refused(rs):
    p = W.diag_quadratic(N=8)
    s = rs.Solver(p)
    with pytest.raises(rs.RSRRError) as e:
        s.add_points([0.1 + 0.2j])
    assert e.value.status == rs.RSRR_ESTATE
    s.close()
