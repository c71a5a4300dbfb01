"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, Cauchy's integral, Sylvester inertia, companion linearisation,
Lambert W, the argument principle, the paper's loaded-string example).  None of
these re-types the oracle's formulas or re-calls its library step."""
import json
import os
import sys

import numpy as np
import pytest
from scipy.special import lambertw

import oracle
import workloads as W
from util import match_eigs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ORACLE_MOD = sys.modules["oracle.rsrr"]


# ---------------------------------------------------------------- closed forms
def exact_roots(p):
    """Roots of the decoupled scalar problems behind a hidden_diagonal NEP."""
    d = p.meta["diags"]
    if p.name == "diag_quadratic":          # k + z c + z^2 m
        k, c, m = d
        disc = np.sqrt((c * c - 4 * m * k).astype(complex))
        r = np.concatenate([(-c + disc) / (2 * m), (-c - disc) / (2 * m)])
    elif p.name == "diag_rational":         # k - z m + z e/(z - s)
        k, m, e = d
        s = p.fns[2].param
        A, B, C = -m, k + m * s + e, -k * s
        disc = np.sqrt((B * B - 4 * A * C).astype(complex))
        r = np.concatenate([(-B + disc) / (2 * A), (-B - disc) / (2 * A)])
    elif p.name == "diag_delay":            # z - a - b exp(-tau z)
        _, a, b = d
        tau = p.fns[2].param
        r = np.concatenate([a + lambertw(b * tau * np.exp(-a * tau), br) / tau
                            for br in range(-8, 9)])
    elif p.name == "diag_sqrt":             # k - z m + e sqrt(z^2 - kappa^2)
        k, m, e = d
        kap = p.fns[2].param
        # squaring gives (m^2 - e^2) z^2 - 2 m k z + k^2 + e^2 kappa^2 = 0; of its two
        # real roots only (m k + e sqrt(k^2 - kappa^2 (m^2 - e^2))) / (m^2 - e^2) has
        # z m - k > 0, the sign the principal square root requires
        r = (m * k + e * np.sqrt(k * k - kap * kap * (m * m - e * e))) / (m * m - e * e)
        r = r.astype(complex)
    elif p.name == "diag_inv":              # k - z m + e / (sigma - z)
        k, m, e = d
        s = p.fns[2].param
        # (k - z m)(sigma - z) + e = 0:  m z^2 - (k + m sigma) z + k sigma + e = 0
        B = k + m * s
        disc = np.sqrt((B * B - 4 * m * (k * s + e)).astype(complex))
        r = np.concatenate([(B + disc) / (2 * m), (B - disc) / (2 * m)])
    else:
        raise KeyError(p.name)
    return r[oracle.inside(p.region, r)]


def _family(name):
    return getattr(W, name)()


def check_family(p, NQ=256):
    ref = exact_roots(p)
    out = oracle.rsrr(p, NQ=NQ)
    return ref, out, match_eigs(ref, out["lam"])


# --------------------------------------------------------------------- points
def test_points_lie_on_ellipse_and_weights_integrate_cauchy():
    reg = W.Region(0.3 - 1.0j, 2.0, 0.7)
    z = oracle.sample_points(reg, 256)
    assert np.allclose(((z.real - 0.3) / 2.0) ** 2 + ((z.imag + 1.0) / 0.7) ** 2, 1.0)
    w = oracle.quad_weights(reg, 256)
    # sum_q w_q f(z_q) ~ (1/2pi) contour integral of f: = i for 1/(z-c), c inside
    for c, expect in ((0.5 - 0.9j, 1j), (-0.4 - 1.2j, 1j), (3.5 + 0.0j, 0.0), (0.0 + 1.0j, 0.0)):
        assert abs(np.sum(w / (z - c)) - expect) < 1e-12
    # polynomials integrate to zero on a closed contour
    assert abs(np.sum(w * z ** 3)) < 1e-12


# ------------------------------------------------------------ resolvent (step 2)
@pytest.mark.parametrize("name", ["diag_quadratic", "diag_rational", "diag_delay", "diag_sqrt",
                                  "diag_inv"])
def test_resolvent_matches_decoupled_closed_form(name):
    p = _family(name)
    G1 = W.givens_layers(p.n, p.meta["layers"], p.meta["g_seed"])
    G2 = W.givens_layers(p.n, p.meta["layers"], p.meta["g_seed"] + 100)
    z = np.array([p.region.center + 0.3 * p.region.a, p.region.center - 0.2j * p.region.b])
    X = oracle.resolvent_samples(p, z)
    for zj, Xj in zip(z, X):
        t = sum(oracle.eval_fn(fn, zj) * d for fn, d in zip(p.fns, p.meta["diags"]))
        expect = G2.T @ ((G1 @ p.U) / t[:, None])
        assert np.max(np.abs(Xj - expect)) <= 1e-11 * np.max(np.abs(expect))


def test_resolvent_backward_error_is_fp64_level():
    p = W.random_banded()
    z = oracle.sample_points(p.region, p.N)
    for zj, Xj in zip(z, oracle.resolvent_samples(p, z)):
        assert oracle.backward_error_inf(p, zj, Xj).max() < 1e-15


# --------------------------------------------------- eigenvalues (steps 3..5)
@pytest.mark.parametrize("name", ["diag_quadratic", "diag_rational", "diag_delay", "diag_sqrt",
                                  "diag_inv"])
def test_rsrr_finds_closed_form_eigenvalues(name):
    p = _family(name)
    ref, out, err = check_family(p)
    assert len(ref) >= 5
    assert len(out["lam"]) == len(ref)
    assert err <= 1e-9
    assert out["res"].max() <= 1e-10
    assert out["k"] < p.n  # a genuine projection, not the full space


def test_quadratic_proportional_damping_closed_form_full_size():
    """n=1000 benchmark recipe with C = c0*M: lambda^2 + c0 lambda + mu_k = 0,
    mu_k = 6n^2 (2 - 2cos t_k)/(4 + 2cos t_k), t_k = k pi/(n+1)."""
    n, c0 = 1000, 50.0
    p = W.quadratic_tridiag(n=n, c_scale=c0, center=-25.0 + 50.0j)
    t = np.arange(1, n + 1) * np.pi / (n + 1)
    mu = 6.0 * n * n * (2 - 2 * np.cos(t)) / (4 + 2 * np.cos(t))
    disc = np.sqrt((c0 * c0 - 4 * mu).astype(complex))
    lam = np.concatenate([(-c0 + disc) / 2, (-c0 - disc) / 2])
    rel = np.abs(np.abs(lam - p.region.center) / p.region.a - 1)
    assert rel.min() > 5e-3, "closed-form roots too close to the contour for a pin"
    ref = lam[oracle.inside(p.region, lam)]
    out = oracle.rsrr(p, NQ=500)
    assert len(ref) >= 10
    assert match_eigs(ref, out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10


def test_quadratic_workload_matches_companion_linearisation():
    """Benchmark recipe (random diagonal damping): the oracle's eigenvalues in
    the circle centre -25+50i, radius 40 equal the companion pencil's, and the
    literal circle centre 50, radius 40 holds none (count-0 case)."""
    gold = json.load(open(os.path.join(GOLD, "c0_companion.json")))
    c_empty, c_full = gold["circles"]
    assert len(c_empty["inside"]) == 0 and c_empty["min_rel_boundary_distance"] > 0.01
    assert c_full["min_rel_boundary_distance"] > 0.01
    ref = np.array([complex(a, b) for a, b in c_full["inside"]])
    out = oracle.rsrr(W.config("c0b"), NQ=500)
    assert len(ref) == 21
    assert match_eigs(ref, out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
    out0 = oracle.rsrr(W.config("c0"), NQ=500)
    assert len(out0["lam"]) == 0


def test_grid_rational_inertia_count_and_shifted_closed_form():
    """5-point grid rational NEP (benchmark recipe at g=30).  T(x) is real
    symmetric and decreasing on (20, 180), so the eigenvalue count there is
    nu(T(180)) - nu(T(20)) (Sylvester).  With E = e0*I every grid mode mu
    gives the roots of (mu - z)(z - sigma) + e0 z = 0."""
    p = W.rational_grid(g=30, N=64, L=8)
    count = oracle.negative_inertia(p, 180.0) - oracle.negative_inertia(p, 20.0)
    out = oracle.rsrr(p, NQ=500)
    assert count == 10
    assert len(out["lam"]) == count
    assert np.abs(out["lam"].imag).max() < 1e-8
    assert out["res"].max() <= 1e-10

    g, s, e0 = 30, 300.0, 0.5
    p2 = W.rational_grid(g=g, N=64, L=8, frac_e=1.0, e_value=e0)
    j = np.arange(1, g + 1)
    sj = 4 * np.sin(j * np.pi / (2 * (g + 1))) ** 2
    mu = ((g + 1) ** 2 * (sj[:, None] + sj[None, :])).ravel()
    B = mu + s + e0
    disc = np.sqrt(B * B - 4 * mu * s)
    lam = np.concatenate([(B - disc) / 2, (B + disc) / 2])
    ref = lam[oracle.inside(p2.region, lam)]
    out2 = oracle.rsrr(p2, NQ=500)
    assert len(ref) == len(out2["lam"]) >= 8
    assert match_eigs(ref, out2["lam"]) <= 1e-9


def test_loaded_string_example_of_the_paper():
    gold = json.load(open(os.path.join(GOLD, "loaded_string.json")))
    p = W.loaded_string(n=gold["n"], N=gold["N"], L=gold["L"])
    lo, hi = gold["interval"]
    assert oracle.negative_inertia(p, hi) - oracle.negative_inertia(p, lo) == gold["count"]
    out = oracle.rsrr(p, NQ=gold["NQ"], KQ=gold["KQ"])
    lam = out["lam"]
    assert len(lam) == gold["count"]
    assert np.all((lam.real > lo) & (lam.real < hi))
    assert np.abs(lam.imag).max() < 1e-6 * np.abs(lam).max()
    plain = [oracle.plain_residual(p, l, out["V"][:, c]) for c, l in enumerate(lam)]
    assert max(plain) <= 10 * gold["plain_residual_level"]


def test_argument_principle_count_on_tiny_problem():
    p = W.diag_quadratic(n=14, seed=3, N=16, L=4, layers=2)
    reg = W.Region(0.0 + 0.5j, 4.0, 3.0)
    p.region = reg
    ref = exact_roots(p)
    assert oracle.argument_principle_count(p, reg, npts=1024) == len(ref) > 0
    out = oracle.rsrr(p, NQ=256)
    assert match_eigs(ref, out["lam"]) <= 1e-9


# -------------------------------------------------------------- planted errors
def _planted(monkeypatch, which):
    if which == "weights_sign":
        orig = ORACLE_MOD.quad_weights
        monkeypatch.setattr(ORACLE_MOD, "quad_weights", lambda r, n: -orig(r, n).conj())
    elif which == "drop_scale":
        orig = ORACLE_MOD.eval_fn
        monkeypatch.setattr(ORACLE_MOD, "eval_fn",
                            lambda fn, z: orig(W.Fn(fn.kind, fn.param, 1.0), z))
    elif which == "coefficient_transposed":
        monkeypatch.setattr(ORACLE_MOD, "project",
                            lambda prob, Q: [Q.conj().T @ (ORACLE_MOD.coeff_matrix(prob, i).T @ Q)
                                             for i in range(prob.m)])
    elif which == "no_normalisation":
        monkeypatch.setattr(ORACLE_MOD, "normalize_columns", lambda S: S * 1e6)
    elif which == "hankel_shift":
        orig_svd = np.linalg.svd
        monkeypatch.setattr(ORACLE_MOD.np.linalg, "svd",
                            lambda a, *k, **kw: orig_svd(a.T, *k, **kw))


@pytest.mark.parametrize("which", ["weights_sign", "drop_scale", "coefficient_transposed",
                                   "hankel_shift"])
def test_planted_mistakes_fail_a_pin(monkeypatch, which):
    _planted(monkeypatch, which)
    failed = False
    for name in ("diag_quadratic", "diag_rational", "diag_delay"):
        try:
            ref, out, err = check_family(_family(name))
        except Exception:
            failed = True
            break
        if not (len(out["lam"]) == len(ref) and err <= 1e-9):
            failed = True
            break
    assert failed, f"planted mistake {which!r} went unnoticed"


# ------------------------------------------------------------ dense BEM kernel
def test_taylor_expansion_reproduces_the_kernel_matrix():
    """T(z) = sum_{p<P} (z - c)^p A_p inside the circle: the series of
    exp(i z r) about the centre, truncated where (r_max rho)^P/P! < 1e-17."""
    p = W.helmholtz_sphere(n=96, N=8, L=4)
    R = oracle.distances(p)
    A = oracle.taylor_coefficients(p, R)
    assert len(A) == oracle.taylor_terms(p, R) >= 20
    rng = np.random.default_rng(0)
    for _ in range(4):
        z = p.region.center + 0.95 * p.region.a * np.exp(2j * np.pi * rng.random()) * rng.random()
        T = oracle.assemble_dense(p, z, R)
        Ts = sum((z - p.region.center) ** q * Aq for q, Aq in enumerate(A))
        assert np.abs(T - Ts).max() <= 1e-13 * np.abs(T).max()


@pytest.mark.parametrize("n,count", [(64, 4), (128, 1)])
def test_dense_rsrr_count_equals_argument_principle(n, count):
    p = W.helmholtz_sphere(n=n, N=32, L=16)
    assert oracle.argument_principle_count_dense(p, 512) == count
    out = oracle.rsrr_dense(p, NQ=256)
    assert len(out["lam"]) == count
    assert out["res"].max() <= 1e-10


def test_dense_eigenvalue_drifts_towards_pi():
    """Trend only: the continuum single-layer operator on the unit sphere is
    singular at the zeros of j_0(k) = sin(k)/k, k = pi; the discrete NEP's
    eigenvalue in |z - 3| < 1 approaches pi as n grows."""
    d = []
    for n in (128, 256):
        lam = oracle.rsrr_dense(W.helmholtz_sphere(n=n, N=32, L=16), NQ=256)["lam"]
        assert len(lam) == 1
        d.append(abs(lam[0] - np.pi))
    assert d[1] < d[0]


# -------------------------------------------- dense kernel: two-point closed form
def _pair_problem(r=1.0, im=0.5):
    """Two points at distance r, diagonal d = e^{-im r} / (4 pi r).  Then
    det T(z) = d^2 - (e^{i z r} / (4 pi r))^2 vanishes exactly where
    e^{i z r} = +-e^{-im r}, i.e. at z = k pi / r + i im for every integer k,
    with eigenvectors (1, -+1)."""
    P = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    reg = W.Region(complex(3.0, im), 3.5, 3.5)
    U = np.asfortranarray(W.probe(2, 2, 7))
    p = W.DenseProblem("pair", 2, P, np.exp(-im * r) / (4.0 * np.pi * r), reg, 16, 2, U)
    ks = np.arange(-8, 9)
    ref = ks * np.pi / r + 1j * im
    return p, ref[oracle.inside(reg, ref)]


def _pair_ok(p, ref):
    out = oracle.rsrr_dense(p, NQ=256)
    if len(out["lam"]) != len(ref) or match_eigs(ref, out["lam"]) > 1e-9:
        return False, out
    return True, out


def test_dense_two_point_problem_matches_its_closed_form():
    p, ref = _pair_problem()
    assert len(ref) == 3  # k = 0, 1, 2 inside |z - (3 + 0.5i)| < 3.5
    ok, out = _pair_ok(p, ref)
    assert ok, out["lam"]
    assert out["res"].max() <= 1e-12
    for j, lam in enumerate(out["lam"]):
        v = out["V"][:, j]
        sign = 1.0 if round(lam.real / np.pi) % 2 == 0 else -1.0  # e^{i z r} = +-d 4 pi r
        assert abs(v[1] / v[0] + sign) <= 1e-10


def _planted_dense(monkeypatch, which):
    base_asm, base_tay = ORACLE_MOD.assemble_dense, ORACLE_MOD.taylor_coefficients
    if which == "diagonal_doubled":
        def tay(prob, R=None, P=None):
            A = base_tay(prob, R, P)
            A[0] = A[0] + np.diag(np.full(prob.n, prob.diag))
            return A
        monkeypatch.setattr(ORACLE_MOD, "taylor_coefficients", tay)
    elif which == "exponent_sign":
        monkeypatch.setattr(ORACLE_MOD, "taylor_coefficients",
                            lambda prob, R=None, P=None: [
                                np.where(np.eye(prob.n, dtype=bool), A, A.conj() * (-1) ** q)
                                for q, A in enumerate(base_tay(prob, R, P))])
    elif which == "dropped_4pi":
        def asm(prob, z, R=None):
            T = base_asm(prob, z, R)
            off = ~np.eye(prob.n, dtype=bool)
            T[off] *= 4.0 * np.pi
            return T

        def tay(prob, R=None, P=None):
            A = base_tay(prob, R, P)
            off = ~np.eye(prob.n, dtype=bool)
            for Aq in A:
                Aq[off] *= 4.0 * np.pi
            return A
        monkeypatch.setattr(ORACLE_MOD, "assemble_dense", asm)
        monkeypatch.setattr(ORACLE_MOD, "taylor_coefficients", tay)


@pytest.mark.parametrize("which", ["diagonal_doubled", "exponent_sign", "dropped_4pi"])
def test_planted_dense_mistakes_fail_the_two_point_pin(monkeypatch, which):
    p, ref = _pair_problem()
    _planted_dense(monkeypatch, which)
    try:
        ok, _ = _pair_ok(p, ref)
    except Exception:
        ok = False
    assert not ok, f"planted mistake {which!r} went unnoticed"


# ------------------------------------------------- unit pins of steps 3 and 4
def test_truncated_basis_keeps_the_singular_values_above_delta():
    """S = U diag(sigma) V^H with prescribed sigma: the kept count is the
    number of sigma_j > delta sigma_1 and Q spans the matching columns of U."""
    rng = np.random.default_rng(3)
    n, c = 60, 12
    U, _ = np.linalg.qr(rng.normal(size=(n, c)) + 1j * rng.normal(size=(n, c)))
    V, _ = np.linalg.qr(rng.normal(size=(c, c)) + 1j * rng.normal(size=(c, c)))
    sigma = np.logspace(0, -20, c)  # 1 ... 1e-20
    S = (U * sigma) @ V.conj().T
    Q, sig, k = oracle.truncated_basis(S, delta=1e-8)
    assert k == int(np.sum(sigma > 1e-8)) == 5
    # span(Q) = span(U[:, :k]): the projector difference is at rounding level
    Pq, Pu = Q @ Q.conj().T, U[:, :k] @ U[:, :k].conj().T
    assert np.abs(Pq - Pu).max() <= 1e-7  # sigma_k / sigma_{k+1} = 1e2 bounds the angle
    assert np.abs(sig[:k] - sigma[:k]).max() <= 1e-14


def test_projection_onto_coordinate_vectors_is_a_submatrix():
    """With Q = [e_a, e_b, ...], P_i = Q^H A_i Q is A_i restricted to rows and
    columns a, b, ..."""
    p = W.random_banded(n=50, kl=3, ku=4)
    idx = np.array([0, 7, 8, 31, 49])
    Q = np.zeros((p.n, len(idx)), dtype=np.complex128)
    Q[idx, np.arange(len(idx))] = 1.0
    P = oracle.project(p, Q)
    for i, Pi in enumerate(P):
        dense = np.zeros((p.n, p.n))
        rows = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
        dense[rows, p.col_idx] = p.values[i]
        assert np.array_equal(Pi, dense[np.ix_(idx, idx)])


def test_ss_full_on_a_linear_projected_problem():
    """T_Q(z) = K - z I with K = X diag(mu) X^{-1}: SS-FULL returns the mu
    inside the ellipse and eigenvectors parallel to X's columns."""
    rng = np.random.default_rng(4)
    k = 9
    reg = W.Region(complex(0.5, 0.2), 1.0, 0.6)
    mu = np.array([0.3 + 0.1j, 0.9 + 0.3j, 0.2 + 0.5j, 0.6 - 0.2j,
                   3.0, -2.0 + 1j, 0.5 + 2.0j, 2.5 - 1.5j, -1.2 - 0.9j])
    X = rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k)) + 3 * np.eye(k)
    K = X @ np.diag(mu) @ np.linalg.inv(X)
    fns = [W.Fn(W.F_ONE), W.Fn(W.F_ZPOW, 1, -1.0)]
    lam, G, info = oracle.ss_full([K, np.eye(k)], fns, reg, NQ=256, KQ=2)
    inside = oracle.inside(reg, mu)
    assert len(lam) == inside.sum() == 4
    for l, g in zip(lam, G.T):
        j = int(np.argmin(np.abs(mu - l)))
        assert inside[j] and abs(mu[j] - l) <= 1e-10
        x = X[:, j]
        assert abs(np.vdot(x, g)) / (np.linalg.norm(x) * np.linalg.norm(g)) >= 1 - 1e-10


# ------------------------------------------- acceptance checks (eta and rho)
# The oracle's backward error and residual decide every parity test's
# acceptance; they are pinned to hand-computed values (tests/golden), to the
# Rigal-Gaches characterisation of the normwise backward error, and planted
# mutations of their source must each fail one of these pins.
def _cplx(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


def _checker_gold():
    with open(os.path.join(GOLD, "checker_norms.json")) as f:
        return json.load(f)


def _gold_sparse_problem(g):
    A0 = np.array(g["A0"], dtype=np.float64)
    A1 = np.array(g["A1"], dtype=np.float64)
    pat = (A0 != 0) | (A1 != 0)
    rows, cols = np.nonzero(pat)
    row_ptr = np.concatenate([[0], np.cumsum(pat.sum(axis=1))]).astype(np.int64)
    fns = [W.Fn(W.F_ONE), W.Fn(W.F_ZPOW, 1)]
    return W.Problem("gold3", 3, row_ptr, cols.astype(np.int32), [A0[rows, cols], A1[rows, cols]], fns,
                     W.Region(0j, 1.0, 1.0), 1, 2, np.zeros((3, 2), np.complex128))


def _gold_dense_problem(g):
    return W.DenseProblem("gold2", 2, np.array(g["points"], dtype=np.float64), float(g["diag"]),
                          W.Region(0j, 1.0, 1.0), 1, 1, np.zeros((2, 1), np.complex128))


def _checkers_match_gold():
    g = _checker_gold()
    ok = True
    s = g["sparse"]
    p = _gold_sparse_problem(s)
    e = s["eta"]
    eta = ORACLE_MOD.backward_error_inf(p, complex(*e["z"]), _cplx(e["X"]), _cplx(e["U"]))
    ok &= np.allclose(eta, [c["value"] for c in e["columns"]], rtol=1e-13, atol=0)
    for r in s["residual"]:
        rho = ORACLE_MOD.residual(p, complex(*r["lam"]), _cplx(r["v"]))
        ok &= abs(rho - r["value"]) <= 1e-13 * r["value"]
    d = g["dense"]
    q = _gold_dense_problem(d)
    eta = ORACLE_MOD.backward_error_inf_dense(q, complex(*d["z"]), _cplx(d["eta"]["X"]), _cplx(d["eta"]["U"]))
    ok &= abs(eta[0] - d["eta"]["value"]) <= 1e-13 * d["eta"]["value"]
    r = d["residual"]
    rho = ORACLE_MOD.residual_dense(q, complex(*r["lam"]), _cplx(r["v"]))
    ok &= abs(rho - r["value"]) <= 1e-13 * r["value"]
    return bool(ok)


def test_acceptance_checks_match_hand_computed_values():
    assert _checkers_match_gold()


def _rigal_gaches_holds(T, X, U, eta):
    """eta is the normwise backward error: the rank-one perturbation dT = eta
    ||T|| r y^H/||r||, du = -eta ||u|| r/||r|| (y the dual vector of x, ||y||_1
    = 1, y^H x = ||x||_inf) has relative size eta in both T and u and makes x
    an exact solution of (T + dT) x = u + du; no smaller one can, since
    ||r|| <= eps (||T|| ||x|| + ||u||) for any perturbation of relative size eps."""
    Tinf = np.linalg.norm(T, np.inf)
    for c in range(X.shape[1]):
        x, u = X[:, c], U[:, c]
        r = u - T @ x
        rn = np.abs(r).max()
        k = int(np.argmax(np.abs(x)))
        y = np.zeros_like(x)
        y[k] = x[k] / abs(x[k])
        dT = eta[c] * Tinf * np.outer(r, y.conj()) / rn
        du = -eta[c] * np.abs(u).max() * r / rn
        if not np.isclose(np.linalg.norm(dT, np.inf), eta[c] * Tinf, rtol=1e-12):
            return False
        if np.abs((T + dT) @ x - (u + du)).max() > 1e-8 * rn:
            return False
    return True


def _perturbed_solution(T, U, seed):
    rng = np.random.default_rng(seed)
    X = np.linalg.solve(T, U)
    return X * (1.0 + 1e-4 * (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)))


def test_backward_error_is_the_smallest_relative_perturbation():
    p = W.random_banded(n=60, kl=4, ku=2, N=1, L=3, seed=17)   # non-symmetric
    z = 0.4 + 0.1j
    T = oracle.assemble(p, z).toarray()
    X = _perturbed_solution(T, p.U, 1)
    assert _rigal_gaches_holds(T, X, p.U, oracle.backward_error_inf(p, z, X))
    q = W.helmholtz_sphere(n=40, N=1, L=3, seed=9, seed_u=10)
    z = 3.1 + 0.05j
    T = oracle.assemble_dense(q, z)
    X = _perturbed_solution(T, q.U, 2)
    assert _rigal_gaches_holds(T, X, q.U, oracle.backward_error_inf_dense(q, z, X))


def _mutated(func, old, new):
    """A copy of an oracle function with one plausible mistake planted in its
    source (compiled in the oracle module's namespace)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(func))
    assert old in src, (func.__name__, old)
    ns = {}
    exec(compile(src.replace(old, new, 1), "<mutant>", "exec"), ORACLE_MOD.__dict__.copy(), ns)
    return ns[func.__name__]


CHECKER_MUTANTS = [
    # row sums -> column sums for ||T||_inf
    ("backward_error_inf", "np.abs(T).sum(axis=1).max()", "np.abs(T).sum(axis=0).max()"),
    # the ||u||_inf term dropped from the denominator
    ("backward_error_inf", "+ np.abs(U).max(axis=0)", ""),
    # ||x||_1 in place of ||x||_inf
    ("backward_error_inf", "np.abs(X).max(axis=0) +", "np.abs(X).sum(axis=0) +"),
    # ||A_i||_inf in place of ||A_i||_1
    ("residual", "coeff_matrix(prob, i)).sum(axis=0).max()", "coeff_matrix(prob, i)).sum(axis=1).max()"),
    # |f_i(lam)| dropped from the scale
    ("residual", "scale += abs(eval_fn(fn, lam)) * a1", "scale += a1"),
    # ||v||_2 dropped
    ("residual", "(scale * np.linalg.norm(v))", "scale"),
    # the ||u||_inf term dropped (dense)
    ("backward_error_inf_dense", "+ np.abs(U).max(axis=0)", ""),
    # residual in the 1-norm (dense)
    ("residual_dense", "np.linalg.norm(T @ v)", "np.linalg.norm(T @ v, 1)"),
    # largest entry in place of ||T||_1 (dense)
    ("residual_dense", "np.abs(T).sum(axis=0).max()", "np.abs(T).max()"),
]


@pytest.mark.parametrize("name,old,new", CHECKER_MUTANTS)
def test_planted_checker_mistakes_fail_a_pin(monkeypatch, name, old, new):
    monkeypatch.setattr(ORACLE_MOD, name, _mutated(getattr(ORACLE_MOD, name), old, new))
    try:
        gold = _checkers_match_gold()
    except Exception:
        gold = False
    assert not gold, f"planted mistake in {name} ({old!r} -> {new!r}) went unnoticed"


# ---------------------------------------------- Sylvester inertia (band LDL^T)
def _grid_closed_form(g):
    """Eigenvalues of K = (g+1)^2 (5-point Laplacian) on a g x g grid:
    (g+1)^2 (4 sin^2(j pi / 2(g+1)) + 4 sin^2(k pi / 2(g+1))), 1 <= j, k <= g."""
    j = np.arange(1, g + 1)
    lam1 = 4.0 * np.sin(j * np.pi / (2.0 * (g + 1))) ** 2
    return np.sort(((g + 1) ** 2 * (lam1[:, None] + lam1[None, :])).ravel())


def _band_counts_agree(count_fn):
    p = W.rational_grid(g=30, N=8, L=2)
    for x in (20.0, 55.5, 100.0, 180.0, 250.0):
        if count_fn(p, x) != oracle.negative_inertia(p, x):
            return False
    q = W.rational_grid(g=40, N=8, L=2, frac_e=0.0)   # E = 0: T(x) = K - x I
    ev = _grid_closed_form(40)
    for x in (10.0, 60.0, 123.4, 250.0):
        if count_fn(q, x) != int(np.sum(ev < x)):
            return False
    s = W.loaded_string()
    for x in (3.0, 500.0, 1e4):
        if count_fn(s, x) != oracle.negative_inertia(s, x):
            return False
    return True


def test_band_inertia_matches_dense_count_and_closed_form():
    assert _band_counts_agree(oracle.negative_inertia_band)


def test_bisection_recovers_the_closed_form_grid_eigenvalues():
    q = W.rational_grid(g=30, N=8, L=2, frac_e=0.0)
    ev = _grid_closed_form(30)
    ev = ev[(ev > 20.0) & (ev < 180.0)]
    bis = oracle.bisect_real_eigenvalues(q, 20.0, 180.0)
    assert len(bis) == len(ev) > 5          # includes double eigenvalues (j, k), (k, j)
    assert np.max(np.abs(bis - ev) / ev) < 1e-12


@pytest.mark.parametrize("old,new", [
    ("cj[i - j] -= lj * col[i];", "cj[i - j] -= lj * col[j];"),   # transposed operand
    ("const double lj = col[j] / d;", "const double lj = col[j];"),  # dropped pivot division
])
def test_planted_inertia_mistakes_fail_a_pin(tmp_path, old, new):
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(ORACLE_MOD.__file__), "band_inertia.c")).read()
    assert old in src
    (tmp_path / "m.c").write_text(src.replace(old, new))
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", str(tmp_path / "m.so"), str(tmp_path / "m.c")],
                   check=True)
    lib = ctypes.CDLL(str(tmp_path / "m.so"))
    lib.band_ldlt_negcount.restype = ctypes.c_int
    lib.band_ldlt_negcount.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    saved = ORACLE_MOD._INERTIA_LIB
    ORACLE_MOD._INERTIA_LIB = lib
    try:
        agree = _band_counts_agree(oracle.negative_inertia_band)
    except ZeroDivisionError:
        agree = False
    finally:
        ORACLE_MOD._INERTIA_LIB = saved
    assert not agree, f"planted mistake {old!r} -> {new!r} went unnoticed"


# ------------------------------ SS-RI and SSRR-M (Sections 3.3, 4.1, 5.1, 5.2)
def _string(N, L):
    """The loaded string of Example 1 with N Chebyshev points of the first kind
    on [3, 1e4] (Section 5.1) and L probe columns."""
    s = W.loaded_string(N=N, L=L)
    s.region = W.Region(5001.5, 4998.5, 0.1 * 4998.5, kind="interval")
    return s


def test_chebyshev_points_and_weights():
    reg = W.Region(2.0, 3.0, 0.5, kind="interval")
    z = oracle.sample_points(reg, 7)
    x = np.cos((2 * np.arange(7) + 1) * np.pi / 14)
    assert np.allclose(z, 2.0 + 3.0 * x, rtol=0, atol=1e-15)
    # the Chebyshev weights are the barycentric weights up to a common factor
    w = oracle.interpolation_weights(reg, z)
    wb = oracle.interpolation_weights(W.Region(2.0, 3.0, 0.5, kind="points", points=z), z)
    r = wb / w
    assert np.allclose(r, r[0], rtol=1e-12)
    # barycentric weights: sum_i w_i p(z_i) = leading coefficient of the
    # interpolant, 0 for polynomials of degree < N - 1
    zz = np.array([0.3, -1.1 + 0.4j, 2.0, 0.7 - 0.9j, 1.5j])
    wb = oracle.interpolation_weights(W.Region(0j, 1.0, 1.0, kind="points", points=zz), zz)
    for d in range(4):
        assert abs(np.sum(wb * zz ** d)) <= 1e-13 * np.abs(wb).sum()
    assert abs(np.sum(wb * zz ** 4)) > 1e-3 * np.abs(wb).sum()


def test_ss_ri_on_the_loaded_string_follows_section_5_1():
    """Section 5.1: with L = K = 10 (N = 200) SS-RI reaches about 1e-10 on the
    32 eigenvalues; L = 3, K = 40 loses accuracy; L = 2, K = 60 fails."""
    exact = oracle.bisect_real_eigenvalues(_string(200, 10), 3.0, 1e4).astype(complex)
    assert len(exact) == 32
    good = oracle.ss_ri(_string(200, 10), K=10)
    assert len(good["lam"]) == 32 and match_eigs(exact, good["lam"]) <= 1e-9
    worse = oracle.ss_ri(_string(200, 3), K=40)
    assert len(worse["lam"]) != 32 or match_eigs(exact, worse["lam"]) > 10 * match_eigs(exact, good["lam"])
    bad = oracle.ss_ri(_string(200, 2), K=60)
    assert len(bad["lam"]) < 32


def test_sampling_beats_moments_on_the_loaded_string_section_5_2():
    """Section 5.2: with L = 1 and N = 100 Chebyshev points RSRR finds the 32
    eigenvalues; SSRR-M with K = N does not (its moment matrix loses rank)."""
    exact = oracle.bisect_real_eigenvalues(_string(100, 1), 3.0, 1e4).astype(complex)
    s = oracle.rsrr(_string(100, 1), NQ=500, KQ=8)
    assert len(s["lam"]) == 32 and match_eigs(exact, s["lam"]) <= 1e-9
    m = oracle.ssrr_m(_string(100, 1), K=100, NQ=500, KQ=8)
    assert len(m["lam"]) < 32 or match_eigs(exact, m["lam"]) > 1e-6


@pytest.mark.parametrize("name", ["diag_quadratic", "diag_rational"])
def test_ssrr_m_finds_closed_form_eigenvalues(name):
    p = getattr(W, name)(N=48, L=8)
    ref = exact_roots(p)
    out = oracle.ssrr_m(p, K=6, NQ=256)
    assert len(out["lam"]) == len(ref) and match_eigs(ref, out["lam"]) <= 1e-9


@pytest.mark.parametrize("which", ["weights_sign", "hankel_unshifted"])
def test_planted_moment_mistakes_fail_a_pin(monkeypatch, which):
    ss_ri = ORACLE_MOD.ss_ri
    if which == "weights_sign":   # (-1)^i dropped from the Chebyshev weights
        orig = ORACLE_MOD.interpolation_weights
        monkeypatch.setattr(ORACLE_MOD, "interpolation_weights", lambda r, z: np.abs(orig(r, z)))
    else:   # H^< built from A_{i+j} instead of A_{i+j+1}
        ss_ri = _mutated(ss_ri, "Hs = np.block([[A[i + j + 1]", "Hs = np.block([[A[i + j]")
    exact = oracle.bisect_real_eigenvalues(_string(200, 10), 3.0, 1e4).astype(complex)
    out = ss_ri(_string(200, 10), K=10)
    assert len(out["lam"]) != 32 or match_eigs(exact, out["lam"]) > 1e-9


# ------------------------------------------- stored full-size golden values
def test_full_size_grid_golden_is_consistent():
    """tests/golden/c1_eigs.json: the full-size count recomputed by the band
    inertia, and the oracle's RSRR eigenvalues against the bisected ones."""
    with open(os.path.join(GOLD, "c1_eigs.json")) as f:
        g = json.load(f)
    p = W.config("c1")
    assert oracle.negative_inertia_band(p, 180.0) - oracle.negative_inertia_band(p, 20.0) == g["count_in_region"]
    bis = np.array(g["bisection_eigenvalues"])
    lam = np.array([complex(*z) for z in g["oracle_rsrr_eigenvalues"]])
    assert len(bis) == len(lam) == g["count_in_region"] == 10
    assert match_eigs(bis.astype(complex), lam) <= 1e-11
    assert max(g["oracle_rsrr_residuals"]) <= 1e-14


def test_dense_n1024_golden_is_consistent():
    with open(os.path.join(GOLD, "dense_n1024.json")) as f:
        g = json.load(f)
    assert g["count_in_region"] == len(g["oracle_rsrr_eigenvalues"]) >= 1
    lam = np.array([complex(*z) for z in g["oracle_rsrr_eigenvalues"]])
    assert np.all(np.abs(lam - 3.0) < 1.0)
    assert max(g["oracle_rsrr_residuals"]) <= 1e-12


# ------------------------------------------------ rectangle contour (Section 5.4)
def _rect(nx=27):
    return W.Region(272.5 + 15.0j, 57.5, 25.0, kind="rect", nx=nx)


def test_gauss_legendre_is_exact_to_degree_2n_minus_1():
    """The n-point Gauss-Legendre rule integrates x^k over [-1, 1] exactly
    (2/(k+1) for even k, 0 for odd k) for k <= 2n - 1; for x^(2n) it falls
    short by the rule's error constant 2^(2n+1) (n!)^4 / ((2n+1) ((2n)!)^2)."""
    from math import factorial
    for n in (5, 13, 27):
        x, w = oracle.gauss_legendre(n)
        for k in range(2 * n):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(np.sum(w * x ** k) - exact) <= 1e-14
        if n < 27:
            err = 2.0 / (2 * n + 1) - np.sum(w * x ** (2 * n))
            want = 2 ** (2 * n + 1) * factorial(n) ** 4 / ((2 * n + 1) * factorial(2 * n) ** 2)
            assert abs(err - want) <= 1e-6 * want


def test_rectangle_points_and_weights_integrate_cauchy():
    """(Through the module, so that planted mistakes are seen.)  Sampling
    points: nx Gauss-Legendre nodes on each horizontal side, N/2 -
    nx on each vertical side, counterclockwise; the weights dz/(2 pi) give
    (1/2 pi) of the contour integral: i for 1/(z - c) with c inside, 0 outside
    and 0 for polynomials (Cauchy)."""
    reg = _rect()
    z = ORACLE_MOD.sample_points(reg, 80)
    c, a, b = 272.5 + 15.0j, 57.5, 25.0
    bottom, right, top, left = z[:27], z[27:40], z[40:67], z[67:]
    assert np.allclose(bottom.imag, c.imag - b) and np.all(np.diff(bottom.real) > 0)
    assert np.allclose(right.real, c.real + a) and np.all(np.diff(right.imag) > 0)
    assert np.allclose(top.imag, c.imag + b) and np.all(np.diff(top.real) < 0)
    assert np.allclose(left.real, c.real - a) and np.all(np.diff(left.imag) < 0)
    x27, _ = ORACLE_MOD.gauss_legendre(27)
    assert np.allclose(bottom.real, c.real + a * x27, rtol=0, atol=1e-12)
    # the 80 sampling points (one Gauss rule per side) and the composite rule
    # of SS-FULL (10-point panels), each to its own accuracy
    for (zq, wq), tol, poles in (
            ((z, ORACLE_MOD.interpolation_weights(reg, z)), 1e-6, (c, 250 + 20j, 400 + 0j, 272 + 80j)),
            (ORACLE_MOD.contour_quadrature(reg, 500), 1e-10, (c, 300 - 5j, 220 - 5j, 400 + 0j, 272 + 60j))):
        for pole in poles:
            expect = 1j if ORACLE_MOD.inside(reg, np.array([pole]))[0] else 0.0
            assert abs(np.sum(wq / (zq - pole)) - expect) < tol
        assert abs(np.sum(wq * ((zq - c) / a) ** 5)) < 1e-12
    zq, wq = ORACLE_MOD.contour_quadrature(reg, 500)
    assert 480 <= len(zq) <= 520 and len(zq) % ORACLE_MOD.RECT_PANEL == 0
    assert ORACLE_MOD.inside(reg, np.array([c, c + 57.4, c - 24.9j, c + 58, c + 25.1j])).tolist() == \
        [True, True, True, False, False]
    p = ORACLE_MOD.contour_path(reg, np.array([0.0, 115 / 330, 165 / 330, 280 / 330, 1.0]))
    assert np.allclose(p, [c - a - 1j * b, c + a - 1j * b, c + a + 1j * b, c - a + 1j * b, c - a - 1j * b])


# rectangles with every closed-form eigenvalue at least 0.1 from the contour;
# the quadratic's holds two eigenvalues outside its inscribed ellipse
RECT_REGION = {"diag_quadratic": (0.2 + 0.3j, 0.6, 0.9), "diag_sqrt": (5.0 + 0.0j, 1.35, 0.45)}


def rect_family(name, nx=16, **kw):
    p = getattr(W, name)(**kw)
    c, a, b = RECT_REGION[name]
    p.region = W.Region(c, a, b, kind="rect", nx=nx)
    return p


@pytest.mark.parametrize("name", ["diag_quadratic", "diag_sqrt"])
def test_rsrr_on_a_rectangle_finds_closed_form_eigenvalues(name):
    """RSRR with Gauss-Legendre sampling points on a rectangle and SS-FULL by
    composite Gauss quadrature, on closed-form families; the count inside
    also by the argument principle along the rectangle."""
    p = rect_family(name, N=48, L=6)
    ref = exact_roots(p)
    assert len(ref) >= 4
    out = oracle.rsrr(p, NQ=500)
    assert len(out["lam"]) == len(ref) and match_eigs(ref, out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
    q = rect_family(name, nx=2, n=40, N=8, L=2)
    cnt = len(exact_roots(q))
    assert oracle.argument_principle_count(q, q.region, npts=512) == cnt
    assert oracle.argument_principle_count(q, q.region, npts=512, band=True) == cnt


def test_moment_methods_on_a_rectangle_find_closed_form_eigenvalues():
    """SS-RI's moments are contour integrals of U^H T^{-1} U, accurate only as
    far as the Gauss rule on the sides resolves the poles near the contour:
    128 points reach 1e-13 here (48 give 4e-6); SSRR-M only needs span(M)."""
    p = rect_family("diag_quadratic", nx=44, N=128, L=8)
    ref = exact_roots(p)
    out = oracle.ss_ri(p, K=8)
    assert len(out["lam"]) == len(ref) and match_eigs(ref, out["lam"]) <= 1e-9
    p = rect_family("diag_quadratic", N=48, L=8)
    out = oracle.ssrr_m(p, K=6, NQ=500)
    assert len(out["lam"]) == len(ref) and match_eigs(ref, out["lam"]) <= 1e-9


@pytest.mark.parametrize("which", ["clockwise", "half_weights", "ellipse_contour"])
def test_planted_rectangle_mistakes_fail_a_pin(monkeypatch, which):
    if which == "clockwise":
        orig = ORACLE_MOD.rect_sides
        monkeypatch.setattr(ORACLE_MOD, "rect_sides", lambda reg: [(q, p) for p, q in orig(reg)])
    elif which == "half_weights":
        orig = ORACLE_MOD.gauss_legendre
        monkeypatch.setattr(ORACLE_MOD, "gauss_legendre", lambda n: (orig(n)[0], 0.5 * orig(n)[1]))
    else:   # the ellipse's trapezoid rule for a rectangular region
        orig = ORACLE_MOD.contour_quadrature
        monkeypatch.setattr(ORACLE_MOD, "contour_quadrature",
                            lambda reg, NQ: orig(W.Region(reg.center, reg.a, reg.b), NQ))
    failed = False
    try:
        test_rsrr_on_a_rectangle_finds_closed_form_eigenvalues("diag_quadratic")
        test_rectangle_points_and_weights_integrate_cauchy()
    except (AssertionError, Exception):
        failed = True
    assert failed, f"planted mistake {which!r} went unnoticed"


def test_gun_like_golden_is_consistent():
    """tests/golden/gun_like.json: the argument-principle count equals the
    number of eigenpairs of each run, every stored eigenvalue has a tiny
    normalised residual when recomputed here with an eigenvector from the
    banded null-space iteration, and the three runs agree."""
    with open(os.path.join(GOLD, "gun_like.json")) as f:
        g = json.load(f)
    runs = [np.array([complex(*z) for z in g[k]["eigenvalues"]])
            for k in ("contour_N80_L2", "stage1_N30_L2", "stage2_L2")]
    assert all(len(r) == g["count_in_region"] == 15 for r in runs)
    assert match_eigs(runs[0], runs[2]) <= 1e-11 and match_eigs(runs[0], runs[1]) <= 1e-9
    assert max(g["stage2_L2"]["residuals"]) <= max(g["contour_N80_L2"]["residuals"])
    # inverse iteration at each stored eigenvalue: T(lam) is (numerically)
    # singular, so two solves with a random right-hand side give a vector
    # with a residual at rounding level
    import scipy.sparse.linalg as spla
    p = W.gun_like()
    rng = np.random.default_rng(0)
    for lam in runs[0][:5]:
        lu = spla.splu(ORACLE_MOD.assemble(p, lam).tocsc())
        v = lu.solve(rng.standard_normal(p.n) + 0j)
        v = lu.solve(v / np.linalg.norm(v))
        assert oracle.residual(p, lam, v) <= 1e-13
