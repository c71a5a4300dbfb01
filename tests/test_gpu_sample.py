"""GPU parity of resolvent sampling (RSRR steps 1-2): sampling points, the
samples X_j = T(z_j)^{-1} U and their backward errors, through the C ABI,
against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

ETA_TOL = 1e-10


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


def run(rs, p, precision, **kw):
    opts = rs.default_opts(precision=precision, **kw)
    s = rs.Solver(p, opts)
    s.sample()
    st = s.check_status()
    out = dict(S=s.samples(), eta=s.eta(), z=s.points(), stats=s.stats(), status=st)
    s.close()
    return out


def compare(p, out, rel_tol, eta_tol):
    z = oracle.sample_points(p.region, p.N)
    assert np.abs(out["z"] - z).max() <= 1e-13 * max(1.0, np.abs(z).max())
    ref = oracle.resolvent_samples(p, z)
    L = p.L
    worst = 0.0
    for j, Xr in enumerate(ref):
        Xg = out["S"][:, j * L:(j + 1) * L]
        # backward error of the GPU result, computed by the oracle in FP64
        eta_cpu = oracle.backward_error_inf(p, z[j], Xg)
        assert eta_cpu.max() <= eta_tol, (j, eta_cpu.max())
        # the library's own eta agrees with the oracle's evaluation
        eg = out["eta"][j * L:(j + 1) * L]
        # (atol: backward errors at the 1e-16 rounding floor differ by rounding order)
        assert np.allclose(eg, eta_cpu, rtol=1e-3, atol=max(1e-3 * eta_tol, 1e-14))
        worst = max(worst, np.abs(Xg - Xr).max() / np.abs(Xr).max())
    assert worst <= rel_tol, worst
    return worst


CASES = [
    ("random_band_7_5", lambda: W.random_banded(n=300, kl=7, ku=5, N=6, L=5)),
    ("random_band_ragged", lambda: W.random_banded(n=67, kl=3, ku=9, N=3, L=17, seed=3)),
    ("tiny_n_below_block", lambda: W.random_banded(n=13, kl=2, ku=2, N=2, L=3, seed=4)),
    ("upper_only", lambda: W.random_banded(n=90, kl=0, ku=4, N=2, L=2, seed=5)),
    ("lower_only", lambda: W.random_banded(n=90, kl=5, ku=0, N=2, L=2, seed=6)),
    ("hidden_quadratic", lambda: W.diag_quadratic()),
    ("hidden_delay", lambda: W.diag_delay()),
    ("quadratic_tridiag_c0b", lambda: W.config("c0b")),
    ("grid_g30", lambda: W.rational_grid(g=30, N=8, L=8)),
    ("grid_g40_kl_above_32", lambda: W.rational_grid(g=40, N=4, L=4)),
    ("loaded_string_real_points", lambda: W.loaded_string(N=12, L=2)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_mixed_precision_samples_match_oracle(rs, name, make):
    p = make()
    out = run(rs, p, rs.RSRR_PREC_MIXED)
    assert out["status"] == rs.RSRR_OK, out["status"]
    assert out["stats"]["converged"] == 1
    compare(p, out, rel_tol=1e-6, eta_tol=ETA_TOL)


@pytest.mark.parametrize("name,make", CASES[:4] + CASES[7:9], ids=[c[0] for c in CASES[:4] + CASES[7:9]])
def test_fp64_samples_match_oracle(rs, name, make):
    p = make()
    out = run(rs, p, rs.RSRR_PREC_FP64)
    assert out["status"] == rs.RSRR_OK
    compare(p, out, rel_tol=1e-9, eta_tol=1e-14)


def test_sampling_point_on_an_eigenvalue_reports_singular(rs):
    """T(z) = diag(d) - z I sampled exactly at z = d[5]: an exact zero pivot."""
    n = 64
    d = np.linspace(1.0, 4.0, n)
    p = W.random_banded(n=n, kl=1, ku=1, N=3, L=2, m=2, seed=9)
    p.values = [np.where(np.repeat(np.arange(n), np.diff(p.row_ptr)) == p.col_idx, 0.0, 0.0)
                for _ in range(2)]
    rows = np.repeat(np.arange(n), np.diff(p.row_ptr))
    diag = rows == p.col_idx
    p.values[0] = np.where(diag, d[rows], 0.0)
    p.values[1] = np.where(diag, -1.0, 0.0)
    p.fns = [W.Fn(W.F_ONE), W.Fn(W.F_ZPOW, 1)]
    p.region = W.Region(2.0 + 0j, 3.0, 1.0, kind="points",
                        points=np.array([0.5 + 0.1j, d[5] + 0j, 7.0 + 0j]))
    for prec in (rs.RSRR_PREC_MIXED, rs.RSRR_PREC_FP64):
        s = rs.Solver(p, rs.default_opts(precision=prec))
        s.sample()
        assert s.check_status() == rs.RSRR_ESINGULAR
        assert s.stats()["singular_point"] == 1
        s.close()


def test_refinement_limit_reports_no_convergence(rs):
    p = W.random_banded(n=120, kl=4, ku=4, N=2, L=2)
    s = rs.Solver(p, rs.default_opts(eta_tol=1e-300, max_refine=2))
    s.sample()
    assert s.check_status() == rs.RSRR_ENOCONV
    assert s.stats()["refine_sweeps"] == 2
    s.close()


def test_results_do_not_depend_on_the_batch(rs):
    """A point's samples are the same whether it is sampled alone or with others."""
    p = W.rational_grid(g=30, N=8, L=4)
    full = run(rs, p, rs.RSRR_PREC_MIXED)["S"]
    z = oracle.sample_points(p.region, p.N)
    q = W.rational_grid(g=30, N=1, L=4)
    q.region = W.Region(p.region.center, p.region.a, p.region.b, kind="points", points=z[3:4])
    one = run(rs, q, rs.RSRR_PREC_MIXED)["S"]
    assert np.array_equal(full[:, 3 * 4:4 * 4], one)


@pytest.mark.slow
def test_full_size_grid_rational_sampled_parity(rs):
    """Benchmark workload at full size (n=40000, half-bandwidth 200, N=64, L=32):
    every column reaches eta <= 1e-10, and two sampled points agree with the
    oracle's banded LAPACK solve."""
    p = W.config("c1")
    opts = rs.default_opts()
    s = rs.Solver(p, opts)
    s.sample()
    assert s.check_status() == rs.RSRR_OK
    eta = s.eta()
    assert eta.max() <= ETA_TOL
    S = s.samples()
    z = s.points()
    s.close()
    zo = oracle.sample_points(p.region, p.N)
    for j in (0, 37):
        Xr = oracle.resolvent_samples(p, zo[j:j + 1])[0]
        Xg = S[:, j * p.L:(j + 1) * p.L]
        assert oracle.backward_error_inf(p, zo[j], Xg).max() <= ETA_TOL
        assert np.abs(Xg - Xr).max() / np.abs(Xr).max() <= 1e-6


# the streaming solve (factor panels through a cp.async ring) against the
# one-kernel solve on the same factors: one solve, no refinement
SOLVE_CASES = [CASES[0], CASES[1], CASES[2], CASES[3], CASES[4],
               ("wide_band_many_blocks", lambda: W.random_banded(n=2000, kl=150, ku=140, N=3, L=19, seed=11)),
               ("band_wider_than_rows", lambda: W.random_banded(n=70, kl=66, ku=60, N=2, L=16, seed=12))]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_streaming_solve_matches_the_one_kernel_solve(rs, name, make, precision):
    p = make()
    a = run(rs, p, precision, max_refine=0)
    b = run(rs, p, precision, max_refine=0, flags=rs.RSRR_FLAG_PLAIN_SOLVE)
    scale = np.abs(b["S"]).max()
    # same factors, same operations in another order: complex64 or complex128 rounding
    tol = 1e-4 if precision == 1 else 1e-11
    assert np.abs(a["S"] - b["S"]).max() <= tol * scale
    # and both are solutions: the refined streaming path reaches the oracle
    if precision == 1:
        out = run(rs, p, precision)
        compare(p, out, rel_tol=1e-6, eta_tol=ETA_TOL)


# the band LU as a cluster of two CTAs per point (the default) against one CTA
# per point: same arithmetic on every element in the same order, so the
# factors, and the samples of one solve, agree bit for bit
LU_CASES = SOLVE_CASES + [("grid_g40", lambda: W.rational_grid(g=40, N=4, L=4)),
                          ("band_above_224", lambda: W.random_banded(n=900, kl=240, ku=30, N=2, L=3, seed=13))]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", LU_CASES, ids=[c[0] for c in LU_CASES])
def test_cluster_lu_matches_the_one_cta_lu_bitwise(rs, name, make, precision):
    p = make()
    a = run(rs, p, precision, max_refine=0)
    b = run(rs, p, precision, max_refine=0, flags=rs.RSRR_FLAG_ONE_CTA_LU)
    assert a["status"] == b["status"]
    assert np.array_equal(a["S"], b["S"])
    if precision == 1:
        compare(p, run(rs, p, precision), rel_tol=1e-6, eta_tol=ETA_TOL)


def test_graph_replay_gives_the_eager_samples(rs):
    """RSRR_FLAG_GRAPH: the eager first call, the captured second call and a
    replay give bit for bit the samples of a handle without the flag."""
    import torch
    p = W.rational_grid(g=40, N=8, L=4)
    stream = torch.cuda.Stream()
    ref = run(rs, p, rs.RSRR_PREC_MIXED)["S"]
    s = rs.Solver(p, rs.default_opts(flags=rs.RSRR_FLAG_GRAPH))
    for _ in range(3):
        s.sample(stream)
        stream.synchronize()
        assert s.check_status(stream) == rs.RSRR_OK
        assert np.array_equal(s.samples(), ref)
    s.close()


def test_autotuned_sampling_reaches_the_oracle(rs):
    """RSRR_FLAG_AUTOTUNE: whichever LU and solve variants the first call
    keeps, the refined samples reach the oracle (and the cached choice serves
    a second handle of the same shape)."""
    p = W.rational_grid(g=40, N=8, L=4)
    for _ in range(2):
        out = run(rs, p, rs.RSRR_PREC_MIXED, flags=rs.RSRR_FLAG_AUTOTUNE)
        compare(p, out, rel_tol=1e-6, eta_tol=ETA_TOL)


def test_narrow_late_sweeps_give_the_wide_samples_bitwise(rs):
    """The refinement sweeps switch to the narrow solve shape (4 right-hand
    sides per CTA) once few points are left; every column sees the same
    operations, so the samples equal those of the wide shape bit for bit."""
    p = W.rational_grid(g=48, N=64, L=16)
    a = run(rs, p, rs.RSRR_PREC_MIXED)
    b = run(rs, p, rs.RSRR_PREC_MIXED, flags=rs.RSRR_FLAG_WIDE_SOLVE_ONLY)
    assert a["status"] == b["status"] == rs.RSRR_OK
    assert a["stats"]["refine_sweeps"] == b["stats"]["refine_sweeps"] >= 2
    assert np.array_equal(a["S"], b["S"])
    compare(p, a, rel_tol=1e-6, eta_tol=ETA_TOL)


@pytest.mark.parametrize("name,make", [("grid_g48", lambda: W.rational_grid(g=48, N=64, L=16)),
                                       ("random_banded", lambda: W.random_banded(n=700, kl=9, ku=6, N=8, L=5))])
def test_gmres_refinement_reaches_the_oracle(rs, name, make):
    """RSRR_REFINE_GMRES: right-preconditioned GMRES cycles on the complex64
    LU reach the same backward error as plain refinement, in fewer cycles
    than plain refinement needs sweeps, and the samples agree with the oracle."""
    p = make()
    ir = run(rs, p, rs.RSRR_PREC_MIXED)
    gm = run(rs, p, rs.RSRR_PREC_MIXED, refine=rs.RSRR_REFINE_GMRES, gmres_m=3)
    assert gm["status"] == rs.RSRR_OK
    assert gm["stats"]["refine_sweeps"] <= ir["stats"]["refine_sweeps"]
    compare(p, gm, rel_tol=1e-6, eta_tol=ETA_TOL)


def test_gmres_refinement_reaches_a_tight_target_near_eigenvalues(rs):
    """Points close to eigenvalues (the second stage of two-stage sampling):
    GMRES refinement reaches eta <= 1e-13."""
    p = W.diag_rational(N=10)
    s = rs.Solver(p, rs.default_opts(NQ=256, res_tol=1e-2))
    s.sample()
    s.check()
    s.project()
    lam1 = s.solve()["lam"]
    s.close()
    q = W.diag_rational(N=len(lam1))
    q.region = W.Region(p.region.center, p.region.a, p.region.b, kind="points", points=lam1)
    out = run(rs, q, rs.RSRR_PREC_MIXED, refine=rs.RSRR_REFINE_GMRES, gmres_m=4, eta_tol=1e-13,
              max_refine=6)
    assert out["status"] == rs.RSRR_OK
    assert out["eta"].max() <= 1e-13
    compare(q, out, rel_tol=1e-3, eta_tol=1e-13)
