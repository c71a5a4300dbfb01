"""GPU parity of the wider boundary, through the C ABI, against the FP64
oracle and closed forms:

* RSRR_NEP_DENSE -- caller-supplied dense complex A_i (a decoupled quadratic
  hidden by a dense unitary similarity: eigenvalues in closed form);
* complex sparse values (held as real and imaginary terms);
* RSRR_F_CALLBACK and RSRR_F_TAYLOR coefficient functions (the same NEP as a
  builtin-function problem, written another way);
* rsrr_copy_result and the probe seed of rsrr_opts."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_host_prepare import callback_rational, taylor_quadratic
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


def quadratic_roots(k, c, m, region):
    disc = np.sqrt((c * c - 4 * m * k).astype(complex))
    r = np.concatenate([(-c + disc) / (2 * m), (-c - disc) / (2 * m)])
    return r[oracle.inside(region, r)]


def whole(rs, p, **kw):
    s = rs.Solver(p, rs.default_opts(NQ=256, **kw))
    s.sample()
    s.check()
    S, eta = s.samples(), s.eta()
    s.project()
    out = s.solve()
    out["copy"] = s.copy_result()
    out["S"], out["eta"] = S, eta
    s.close()
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_dense_terms_kind_matches_closed_form_and_oracle(rs, prec):
    q = W.dense_hidden_quadratic(n=200)
    o = dict(precision=rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64)
    out = whole(rs, q, **o)
    k, c, m = q.meta["diags"]
    ref = quadratic_roots(k, c, m, q.region)
    assert len(ref) >= 3 and len(out["lam"]) == len(ref)
    assert match_eigs(ref, out["lam"]) <= EIG_TOL
    assert match_eigs(oracle.rsrr_terms(q, NQ=256)["lam"], out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual_terms(q, lam, v) <= RES_TOL
    # samples: backward error and element-wise agreement with the oracle's solves
    zo = oracle.sample_points(q.region, q.N)
    for j in (0, 13):
        Xg = out["S"][:, j * q.L:(j + 1) * q.L]
        Xr = oracle.resolvent_samples_terms(q, zo[j:j + 1])[0]
        assert oracle.backward_error_inf_terms(q, zo[j], Xg).max() <= ETA_TOL
        assert np.abs(Xg - Xr).max() <= 1e-6 * np.abs(Xr).max()


def test_complex_sparse_values_match_closed_form_and_oracle(rs):
    p = W.diag_quadratic_complex()
    out = whole(rs, p)
    k, c, m = p.meta["diags"]
    ref = quadratic_roots(k, c, m, p.region)
    assert len(ref) >= 3 and len(out["lam"]) == len(ref)
    assert match_eigs(ref, out["lam"]) <= EIG_TOL
    assert match_eigs(oracle.rsrr(p, NQ=256)["lam"], out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual(p, lam, v) <= RES_TOL
    zo = oracle.sample_points(p.region, p.N)
    Xr = oracle.resolvent_samples(p, zo[5:6])[0]
    Xg = out["S"][:, 5 * p.L:6 * p.L]
    assert oracle.backward_error_inf(p, zo[5], Xg).max() <= ETA_TOL
    assert np.abs(Xg - Xr).max() <= 1e-6 * np.abs(Xr).max()


def test_callback_function_gives_the_builtin_results(rs):
    a = whole(rs, W.diag_rational())
    b = whole(rs, callback_rational())
    assert len(a["lam"]) == len(b["lam"]) > 0
    assert match_eigs(a["lam"], b["lam"]) <= 1e-12
    assert b["res"].max() <= RES_TOL
    # the same coefficient table to rounding, so the same samples to rounding
    assert np.abs(a["S"] - b["S"]).max() <= 1e-10 * np.abs(a["S"]).max()


def test_taylor_functions_give_the_quadratic_eigenvalues(rs):
    q = taylor_quadratic()
    out = whole(rs, q)
    ref = W.diag_quadratic()
    k, c, m = ref.meta["diags"]
    lam = quadratic_roots(k, c, m, ref.region)
    assert len(out["lam"]) == len(lam) > 0
    assert match_eigs(lam, out["lam"]) <= EIG_TOL
    assert out["res"].max() <= RES_TOL


def test_copy_result_returns_the_solve_results(rs):
    out = whole(rs, W.diag_quadratic())
    cp = out["copy"]
    assert np.array_equal(cp["lam"], out["lam"])
    assert np.array_equal(cp["res"], out["res"])
    assert np.array_equal(cp["V"], out["V"])


def test_probe_seed_selects_the_default_probe(rs):
    def samples(seed):
        p = W.random_banded(n=200, kl=3, ku=3, N=2, L=3)
        p.U = None  # keep the library's default probe
        s = rs.Solver(p, rs.default_opts(seed=seed))
        s.sample()
        s.check()
        S = s.samples()
        s.close()
        return S
    a, b, c = samples(0), samples(0), samples(12345)
    assert np.array_equal(a, b)
    assert np.abs(a - c).max() > 1e-3 * np.abs(a).max()
