"""CPU parity of what rsrr_create prepares on the host (rsrr_describe, no GPU):
the sampling points z_j (step 1, Section 5.1 trapezoid nodes or explicit
points), the coefficient table f_i(z_j) for every function family of the ABI
(Section 2.1: polynomial, z/(z - sigma), 1/(sigma - z), sqrt(z^2 - kappa^2) on
the principal branch, exp(-tau z)) against the oracle, and the half-bandwidths
detected from the pattern against their definition."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1605_07951_gb300", "librsrr.so")


@pytest.fixture(scope="module")
def rsrr():
    if not os.path.exists(LIB):  # a fresh checkout: build the library first
        from paper_1605_07951_gb300 import build
        build.build()
    from paper_1605_07951_gb300 import rsrr as binding
    return binding


FAMILIES = {
    "diag_quadratic": lambda: W.diag_quadratic(),
    "diag_rational": lambda: W.diag_rational(),
    "diag_delay": lambda: W.diag_delay(),
    "diag_sqrt": lambda: W.diag_sqrt(),
    "diag_inv": lambda: W.diag_inv(),
    "grid_g30": lambda: W.rational_grid(g=30, N=64, L=8),
    "random_banded": lambda: W.random_banded(kl=5, ku=9),
    "loaded_string_points": lambda: W.loaded_string(),
    "loaded_string_interval": lambda: _interval_string(),
    "gun_like_rect": lambda: W.gun_like(gx=24, gy=20),
    "gun_like_rect_points": lambda: _rect_points(),
}


def _rect_points():
    p = W.gun_like(gx=24, gy=20, N=8, nx=2)
    r = p.region
    p.region = W.Region(r.center, r.a, r.b, kind="rect", nx=2,
                        points=np.array([250 + 1j, 260 - 2j, 300 + 5j, 320 + 0.5j, 230 + 3j, 228 + 1j, 290, 310 - 1j]))
    return p


def _interval_string():
    s = W.loaded_string(N=37)
    s.region = W.Region(5001.5, 4998.5, 0.1 * 4998.5, kind="interval")
    return s


def bandwidths(p):
    rows = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
    d = rows - np.asarray(p.col_idx)
    return int(max(d.max(), 0)), int(max(-d.min(), 0))


@pytest.mark.parametrize("name", list(FAMILIES))
def test_points_coefficients_and_bandwidths_match(rsrr, name):
    p = FAMILIES[name]()
    z, coef, (kl, ku) = rsrr.prepared(p)
    zo = oracle.sample_points(p.region, p.N)
    assert np.abs(z - zo).max() <= 1e-15 * max(1.0, np.abs(zo).max())
    for i, fn in enumerate(p.fns):
        want = oracle.eval_fn(fn, zo)
        assert np.abs(coef[:, i] - want).max() <= 1e-14 * max(1.0, np.abs(want).max()), (name, i)
    assert (kl, ku) == bandwidths(p)


def test_square_root_takes_the_principal_branch(rsrr):
    # points on both sides of the cut of sqrt(w) (w = z^2 - kappa^2 <= 0 on
    # the real segment |z| < kappa and on the imaginary axis)
    p = W.diag_sqrt(n=16)
    pts = np.array([0.3 + 1e-3j, 0.3 - 1e-3j, -0.3 + 1e-3j, 2e-3 + 0.7j, -2e-3 + 0.7j, 3.0 + 0.5j])
    p.region = W.Region(p.region.center, p.region.a, p.region.b, kind="points", points=pts)
    p.N = len(pts)
    z, coef, _ = rsrr.prepared(p)
    kappa = p.fns[2].param
    got = coef[:, 2] / complex(p.fns[2].scale)
    assert np.all(got.real >= 0.0)  # principal branch: Re sqrt >= 0
    assert np.abs(got ** 2 - (pts ** 2 - kappa ** 2)).max() <= 1e-14
    # across the cut the value jumps sign (the imaginary part flips)
    assert got[0].imag * got[1].imag < 0 and got[3].imag * got[4].imag < 0


def test_describe_validates_like_create(rsrr):
    p = W.diag_quadratic()
    p.row_ptr = p.row_ptr.copy()
    p.row_ptr[0] = 1
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.prepared(p)
    assert e.value.status == rsrr.RSRR_EINVAL


def test_dense_kind_has_points_but_no_table(rsrr):
    p = W.helmholtz_sphere(n=64, N=8, L=4)
    z, coef, (kl, ku) = rsrr.prepared(p)
    assert coef is None and (kl, ku) == (0, 0)
    assert np.abs(z - oracle.sample_points(p.region, p.N)).max() <= 1e-15 * 4


# ------------------------------------------------ the wider boundary (no GPU)
def taylor_quadratic(c0=0.3 + 0.2j, n=240, seed=11):
    """diag_quadratic rewritten in powers of (z - c0): k' = k + c c0 + m c0^2,
    c' = c + 2 m c0, m' = m with TAYLOR functions (same eigenvalues)."""
    p = W.diag_quadratic(n=n, seed=seed)
    k, c, m = p.meta["diags"]
    fns = [W.Fn(W.F_TAYLOR, power=q, shift=c0) for q in range(3)]
    return W.hidden_diagonal([k + c * c0 + m * c0 * c0, c + 2 * m * c0, m.astype(complex)], fns,
                             p.region, p.N, p.L, layers=p.meta["layers"], seed=seed + 1, seed_u=seed + 2,
                             name="taylor_quadratic")


def callback_rational():
    """diag_rational with its z/(z - sigma) term given as a host callback."""
    p = W.diag_rational()
    s = p.fns[2].param
    p.fns[2] = W.Fn(W.F_CALLBACK, scale=p.fns[2].scale, callback=lambda z: z / (z - s))
    return p


def test_complex_values_are_held_as_real_and_imaginary_terms(rsrr):
    p = W.diag_quadratic_complex()
    z, coef, _ = rsrr.prepared(p)
    zo = oracle.sample_points(p.region, p.N)
    # held terms: f_u for Re A_u, i f_u for Im A_u, in caller order
    want = []
    for fn in p.fns:
        f = oracle.eval_fn(fn, zo)
        want += [f, 1j * f]
    want = np.stack(want, axis=1)
    assert coef.shape == want.shape
    assert np.abs(coef - want).max() <= 1e-14 * np.abs(want).max()


def test_callback_and_taylor_terms_are_evaluated_as_defined(rsrr):
    p = callback_rational()
    z, coef, _ = rsrr.prepared(p)
    zo = oracle.sample_points(p.region, p.N)
    ref = W.diag_rational()
    for i, fn in enumerate(ref.fns):
        assert np.abs(coef[:, i] - oracle.eval_fn(fn, zo)).max() <= 1e-14 * np.abs(coef[:, i]).max()
    q = taylor_quadratic()
    z, coef, _ = rsrr.prepared(q)
    zo = oracle.sample_points(q.region, q.N)
    for i in range(3):
        want = (zo - (0.3 + 0.2j)) ** i
        assert np.abs(coef[:, 2 * i] - want).max() <= 1e-14 * max(1.0, np.abs(want).max())


def test_dense_terms_kind_prepares_points_and_coefficients(rsrr):
    q = W.dense_hidden_quadratic(n=64)
    z, coef, (kl, ku) = rsrr.prepared(q)
    zo = oracle.sample_points(q.region, q.N)
    assert np.abs(z - zo).max() <= 1e-15
    for i, fn in enumerate(q.fns):
        assert np.abs(coef[:, i] - oracle.eval_fn(fn, zo)).max() <= 1e-14 * max(1.0, np.abs(coef[:, i]).max())
    assert (kl, ku) == (0, 0)


def test_callback_returning_a_non_finite_value_is_refused(rsrr):
    p = W.diag_rational()
    p.fns[2] = W.Fn(W.F_CALLBACK, callback=lambda z: np.full(z.shape, np.nan))
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.prepared(p)
    assert e.value.status == rsrr.RSRR_EINVAL


def test_real_flag_needs_a_real_problem_at_real_points(rsrr):
    """RSRR_FLAG_REAL (real arithmetic for T(z_j) real, Sections 3.3 and 5.1)
    is accepted only where every T(z_j) is real: real values, real points,
    real f_i there; otherwise rsrr_create refuses it with EINVAL."""
    real = rsrr.default_opts(flags=rsrr.RSRR_FLAG_REAL)
    z, coef, _ = rsrr.prepared(_interval_string(), real)  # Chebyshev points on [3, 1e4]
    assert np.all(z.imag == 0) and np.all(coef.imag == 0)
    refused = [
        (W.loaded_string(N=37), real),                      # explicit real points: accepted below
        (W.rational_grid(g=20, N=16, L=4), real),           # points on an ellipse
        (W.diag_quadratic_complex(), real),                 # complex values
        (W.helmholtz_sphere(n=64, N=8, L=4), real),         # dense kind
        (_interval_string(), rsrr.default_opts(flags=rsrr.RSRR_FLAG_REAL, refine=rsrr.RSRR_REFINE_GMRES)),
    ]
    rsrr.prepared(*refused[0])
    for p, o in refused[1:]:
        with pytest.raises(rsrr.RSRRError) as e:
            rsrr.prepared(p, o)
        assert e.value.status == rsrr.RSRR_EINVAL
        assert "RSRR_FLAG_REAL" in str(e.value)


def test_real_flag_halves_the_factor_storage(rsrr):
    p = _interval_string()
    p.N, p.L = 64, 8
    for prec in (rsrr.RSRR_PREC_MIXED, rsrr.RSRR_PREC_FP64):
        c = rsrr.estimate_bytes(p, rsrr.default_opts(precision=prec))
        r = rsrr.estimate_bytes(p, rsrr.default_opts(precision=prec, flags=rsrr.RSRR_FLAG_REAL))
        assert r < c


def test_rectangle_region_is_validated(rsrr):
    """Gauss-Legendre points on a rectangle need N even and 1 <= nx <= N/2 - 1."""
    for N, nx in ((81, 27), (80, 0), (80, 40), (2, 1)):
        p = W.gun_like(gx=12, gy=10, N=N, nx=nx)
        with pytest.raises(rsrr.RSRRError) as e:
            rsrr.prepared(p)
        assert e.value.status == rsrr.RSRR_EINVAL
    z, _, _ = rsrr.prepared(W.gun_like(gx=12, gy=10, N=80, nx=39))
    assert len(z) == 80
