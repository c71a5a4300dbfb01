"""GPU parity of RSRR steps 3-5 through the C ABI: the orthonormal basis Q,
the projected coefficients P_i = Q^H A_i Q, and the eigenpairs of the whole
method, against the FP64 oracle and the closed forms / inertia counts that
pin it."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from util import match_eigs

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


def gpu_rsrr(rs, p, NQ=256, KQ=2, precision=None, **kw):
    o = rs.default_opts(NQ=NQ, KQ=KQ, **kw)
    if precision is not None:
        o.precision = precision
    s = rs.Solver(p, o)
    s.sample()
    s.check()
    s.project()
    out = s.solve()
    out["Q"] = s.Q()
    out["P"] = s.projected()
    out["stats"] = s.stats()
    s.close()
    return out


FAMILIES = [
    ("diag_quadratic", lambda: W.diag_quadratic(), 256, 2),
    ("diag_rational", lambda: W.diag_rational(), 256, 2),
    ("diag_delay", lambda: W.diag_delay(), 256, 2),
    ("quadratic_c0b", lambda: W.config("c0b"), 500, 2),
    ("grid_g30", lambda: W.rational_grid(g=30, N=64, L=8), 500, 2),
    ("diag_sqrt", lambda: W.diag_sqrt(), 256, 2),
    ("diag_inv", lambda: W.diag_inv(), 256, 2),
]


# the projection's dense products: native FP64, or FP64-accurate slices on
# the bf16 tensor cores (forced here even where the sizes would pick FP64)
GEMMS = [1, 2]
GEMM_IDS = ["fp64gemm", "ozaki"]


@pytest.mark.parametrize("gemm", GEMMS, ids=GEMM_IDS)
@pytest.mark.parametrize("name,make,NQ,KQ", FAMILIES, ids=[f[0] for f in FAMILIES])
def test_eigenpairs_match_oracle(rs, name, make, NQ, KQ, gemm):
    p = make()
    ref = oracle.rsrr(p, NQ=NQ, KQ=KQ)
    out = gpu_rsrr(rs, p, NQ=NQ, KQ=KQ, gemm=gemm)
    assert len(ref["lam"]) > 0
    assert len(out["lam"]) == len(ref["lam"]), (len(out["lam"]), len(ref["lam"]))
    assert match_eigs(ref["lam"], out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
    # residuals re-evaluated by the oracle from the GPU eigenvectors
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual(p, lam, v) <= 1e-10


@pytest.mark.parametrize("gemm", GEMMS, ids=GEMM_IDS)
@pytest.mark.parametrize("name,make,NQ,KQ", FAMILIES[:4], ids=[f[0] for f in FAMILIES[:4]])
def test_basis_is_orthonormal_and_contains_the_eigenvectors(rs, name, make, NQ, KQ, gemm):
    p = make()
    out = gpu_rsrr(rs, p, NQ=NQ, KQ=KQ, gemm=gemm)
    Q = out["Q"]
    k = Q.shape[1]
    assert np.abs(Q.conj().T @ Q - np.eye(k)).max() <= 1e-12
    ref = oracle.rsrr(p, NQ=NQ, KQ=KQ)
    for v in ref["V"].T:
        assert np.linalg.norm(v - Q @ (Q.conj().T @ v)) <= 1e-9 * np.linalg.norm(v)
    # the largest singular value of the normalised S (reported from the
    # level-0 Gram, whose pivoted Cholesky drops a part below 1e-12 of it)
    assert abs(out["stats"]["sigma1"] - ref["sigma"][0]) <= 1e-8 * ref["sigma"][0]


@pytest.mark.parametrize("gemm", GEMMS, ids=GEMM_IDS)
@pytest.mark.parametrize("name,make,NQ,KQ", FAMILIES[:4], ids=[f[0] for f in FAMILIES[:4]])
def test_projected_coefficients_equal_QH_A_Q(rs, name, make, NQ, KQ, gemm):
    p = make()
    out = gpu_rsrr(rs, p, NQ=NQ, KQ=KQ, gemm=gemm)
    P_ref = oracle.project(p, out["Q"])
    for i, (Pg, Pr) in enumerate(zip(out["P"], P_ref)):
        a1 = np.abs(oracle.coeff_matrix(p, i)).sum(axis=0).max()
        assert np.abs(Pg - Pr).max() <= 1e-13 * max(a1, 1e-300), i


def test_count_zero_region_reports_no_eigenpairs(rs):
    out = gpu_rsrr(rs, W.config("c0"), NQ=500)
    assert len(out["lam"]) == 0


@pytest.mark.parametrize("gemm", GEMMS, ids=GEMM_IDS)
@pytest.mark.parametrize("mode", ["fp64", "mixed_tight"])
def test_loaded_string_example_of_the_paper(rs, mode, gemm):
    """The paper's residual level (~1e-11 in ||T v||/||v||) comes from FP64
    solves: the FP64 path reaches it, and so does the mixed path once its
    refinement target is tightened from 1e-10 to 1e-14."""
    gold = json.load(open(os.path.join(GOLD, "loaded_string.json")))
    p = W.loaded_string(n=gold["n"], N=gold["N"], L=gold["L"])
    # the paper's truncation delta = 1e-14 (Section 4.3) as the resolution floor
    if mode == "fp64":
        out = gpu_rsrr(rs, p, NQ=gold["NQ"], KQ=gold["KQ"], precision=rs.RSRR_PREC_FP64,
                       delta_floor=1e-14, gemm=gemm)
    else:
        out = gpu_rsrr(rs, p, NQ=gold["NQ"], KQ=gold["KQ"], eta_tol=1e-14, max_refine=12,
                       delta_floor=1e-14, gemm=gemm)
    lo, hi = gold["interval"]
    lam = out["lam"]
    assert len(lam) == gold["count"]
    assert np.all((lam.real > lo) & (lam.real < hi))
    plain = [oracle.plain_residual(p, l, v) for l, v in zip(lam, out["V"].T)]
    # the paper's level: ~1e-11 typical (Section 5.2), floor around 1e-10 (Section 5.3)
    assert np.median(plain) <= 10 * gold["plain_residual_level"]
    assert max(plain) <= 2 * gold["residual_floor"]
    ref = oracle.rsrr(p, NQ=gold["NQ"], KQ=gold["KQ"])
    assert match_eigs(ref["lam"], lam) <= 1e-9


def test_fp64_path_end_to_end(rs):
    p = W.config("c0b")
    ref = oracle.rsrr(p, NQ=500)
    out = gpu_rsrr(rs, p, NQ=500, precision=rs.RSRR_PREC_FP64)
    assert match_eigs(ref["lam"], out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
