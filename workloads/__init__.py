"""Seeded synthetic NEP workloads, shared as *data* by the oracle and the GPU path.

This module holds problem definitions only: the coefficient matrices A_i of
T(z) = sum_i f_i(z) A_i on one shared sparse pattern, descriptors of the scalar
functions f_i (a kind code plus parameters, evaluated by each side on its own),
the region, N, L and the seeded probe matrix U.  It contains none of the
resolvent-sampling arithmetic (no sampling points, no solves, no projections).

The problem families follow the paper's NEP classes (Section 2.1: quadratic,
rational, square-root types) and its loaded-string example (Section 5.1), plus
synthetic stand-ins for its FEM workloads with the shapes of the benchmark
configurations (quadratic tridiagonal n=1000; rational 5-point grid n=g^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Scalar coefficient function kinds.  f(z) = scale * base(z; param):
#   F_ONE       base = 1
#   F_ZPOW      base = z**param            (param a non-negative integer)
#   F_RATIONAL  base = z / (z - param)
#   F_INV       base = 1 / (param - z)
#   F_SQRT      base = sqrt(z**2 - param**2)   (principal branch)
#   F_EXP       base = exp(-param * z)
#   F_TAYLOR    base = (z - shift)**power    (power a non-negative integer)
#   F_CALLBACK  base = callback(z)           (any function the caller evaluates)
F_ONE, F_ZPOW, F_RATIONAL, F_INV, F_SQRT, F_EXP, F_TAYLOR, F_CALLBACK = range(8)


@dataclass
class Fn:
    kind: int
    param: float = 0.0
    scale: complex = 1.0
    power: int = 0
    shift: complex = 0.0
    callback: object = None   # F_CALLBACK: vectorised z -> base(z)


@dataclass
class Region:
    """Ellipse phi(a) = center + a*cos(t) + i*b*sin(t), explicit sample points,
    the real interval [center - a, center + a] of the ellipse's major axis, or
    the rectangle with vertices center +- a +- i b.

    For kind == "points" the explicit points are the sampling points, and for
    kind == "interval" the N Chebyshev points of the first kind on the
    interval are; in both cases the ellipse (center, a, b) is still the
    contour used for the projected solve and for the inside test.  For
    kind == "rect" the rectangle is the contour and the region; the sampling
    points are Gauss-Legendre nodes on its sides, nx on each side parallel
    to the real axis and N/2 - nx on each of the other two.
    """
    center: complex
    a: float
    b: float
    kind: str = "ellipse"
    points: np.ndarray | None = None
    nx: int = 0


@dataclass
class Problem:
    name: str
    n: int
    row_ptr: np.ndarray          # int64 [n+1], shared CSR pattern of all A_i
    col_idx: np.ndarray          # int32 [nnz]
    values: list                 # m float64 arrays [nnz] (real coefficients)
    fns: list                    # m Fn
    region: Region
    N: int
    L: int
    U: np.ndarray                # complex128 [n, L], Fortran order
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return len(self.values)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def bandwidths(self):
        """(kl, ku) of the shared pattern."""
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d = self.col_idx.astype(np.int64) - rows
        return int(max(0, -d.min())), int(max(0, d.max()))


# ----------------------------------------------------------------------------
# helpers that build data (patterns, probes); no method arithmetic
# ----------------------------------------------------------------------------

def probe(n: int, L: int, seed: int) -> np.ndarray:
    """U with entries (g1 + i g2)/sqrt(2), g ~ N(0,1), PCG64 seeded."""
    rng = np.random.default_rng(seed)
    g1 = rng.standard_normal((n, L))
    g2 = rng.standard_normal((n, L))
    return np.asfortranarray((g1 + 1j * g2) / np.sqrt(2.0))


def _shared_csr(n: int, mats: list):
    """Union pattern (sorted columns per row) of dense or coo-like matrices.

    `mats` are dicts {(i, j): value}; returns row_ptr, col_idx, values list.
    """
    keys = set()
    for mt in mats:
        keys.update(mt.keys())
    keys = sorted(keys)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for (i, _j) in keys:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    col_idx = np.array([j for (_i, j) in keys], dtype=np.int32)
    values = [np.array([mt.get(k, 0.0) for k in keys], dtype=np.float64) for mt in mats]
    return row_ptr, col_idx, values


def _csr_from_dense_band(dense_list: list, kl: int, ku: int):
    """Shared CSR holding every entry inside the (kl, ku) band (zeros kept);
    real or complex values as the matrices are."""
    n = dense_list[0].shape[0]
    rows, cols = [], []
    for i in range(n):
        lo, hi = max(0, i - kl), min(n - 1, i + ku)
        rows.extend([i] * (hi - lo + 1))
        cols.extend(range(lo, hi + 1))
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    values = [np.ascontiguousarray(D[rows, cols], dtype=np.complex128 if np.iscomplexobj(D) else np.float64)
              for D in dense_list]
    return row_ptr, cols.astype(np.int32), values


def _tridiag(n, lo, d, up, last=None):
    mt = {}
    for i in range(n):
        mt[(i, i)] = d
        if i > 0:
            mt[(i, i - 1)] = lo
        if i < n - 1:
            mt[(i, i + 1)] = up
    if last is not None:
        mt[(n - 1, n - 1)] = last
    return mt


# ----------------------------------------------------------------------------
# benchmark-shaped workloads
# ----------------------------------------------------------------------------

def quadratic_tridiag(n: int = 1000, N: int = 32, L: int = 8,
                      center: complex = 50.0, radius: float = 40.0,
                      seed_c: int = 1000, seed_u: int = 1001,
                      c_scale: float | None = None, name: str = "c0") -> Problem:
    """T(z) = K + z C + z^2 M, K = n*tridiag(-1,2,-1), M = tridiag(1,4,1)/(6n),
    C = diag(u), u ~ U[0, 0.1] (seeded).  With c_scale given, C = c_scale*M
    instead (proportional damping: closed-form spectrum)."""
    K = {k: v * n for k, v in _tridiag(n, -1.0, 2.0, -1.0).items()}
    M = {k: v / (6.0 * n) for k, v in _tridiag(n, 1.0, 4.0, 1.0).items()}
    if c_scale is None:
        u = np.random.default_rng(seed_c).uniform(0.0, 0.1, n)
        C = {(i, i): float(u[i]) for i in range(n)}
    else:
        C = {k: c_scale * v for k, v in M.items()}
    row_ptr, col_idx, values = _shared_csr(n, [K, C, M])
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1), Fn(F_ZPOW, 2)]
    return Problem(name, n, row_ptr, col_idx, values, fns,
                   Region(complex(center), radius, radius), N, L, probe(n, L, seed_u),
                   meta=dict(seed_c=seed_c, seed_u=seed_u, c_scale=c_scale))


def rational_grid(g: int = 200, N: int = 64, L: int = 32, sigma: float = 300.0,
                  center: complex = 100.0, a: float = 80.0, b: float = 20.0,
                  frac_e: float = 0.01, e_value: float = 1.0,
                  seed_e: int = 2000, seed_u: int = 2001, name: str = "c1") -> Problem:
    """T(z) = K - z M + (z/(z - sigma)) E on a g x g 5-point grid (natural
    row-major ordering, half-bandwidth g).  K = (g+1)^2 * (4 on the diagonal,
    -1 for each grid neighbour), M = I, E = diag with round(frac_e*n) entries
    equal to e_value at seeded positions (frac_e = 0 gives E = 0)."""
    n = g * g
    idx = np.arange(n)
    gi, gj = idx // g, idx % g
    s = float((g + 1) ** 2)
    rows = [idx]
    cols = [idx]
    kval = [np.full(n, 4.0 * s)]
    for di, dj in ((-1, 0), (0, -1), (0, 1), (1, 0)):
        ok = (gi + di >= 0) & (gi + di < g) & (gj + dj >= 0) & (gj + dj < g)
        rows.append(idx[ok])
        cols.append(((gi + di) * g + (gj + dj))[ok])
        kval.append(np.full(int(ok.sum()), -s))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    kval = np.concatenate(kval)
    order = np.lexsort((cols, rows))
    rows, cols, kval = rows[order], cols[order], kval[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    diag = rows == cols
    mval = np.where(diag, 1.0, 0.0)
    ne = int(round(frac_e * n))
    epos = np.random.default_rng(seed_e).choice(n, size=ne, replace=False)
    emask = np.zeros(n, dtype=bool)
    emask[epos] = True
    evals = np.where(diag & emask[rows], e_value, 0.0)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1, -1.0), Fn(F_RATIONAL, sigma)]
    return Problem(name, n, row_ptr, cols.astype(np.int32), [kval, mval, evals], fns,
                   Region(complex(center), a, b), N, L, probe(n, L, seed_u),
                   meta=dict(g=g, sigma=sigma, seed_e=seed_e, seed_u=seed_u,
                             ne=ne, e_value=e_value))


def loaded_string(n: int = 400, N: int = 100, L: int = 1, kn_last: float = 1.0,
                  seed_u: int = 7001, name: str = "string") -> Problem:
    """Loaded string of Section 5.1: T(z) = K_s + z/(z-1) e_n e_n^T - z M.
    K_s = n*tridiag(-1,2,-1) with K_s[n-1,n-1] = n*kn_last, M = tridiag(1,4,1)/(6n)
    with M[n-1,n-1] = 2/(6n).  Sampling points: N Chebyshev points of the first
    kind in [3, 1e4]; contour for the projected problem: ellipse centre 5001.5,
    a = 4998.5, b = 0.1a (Section 5.2)."""
    K = {k: v * n for k, v in _tridiag(n, -1.0, 2.0, -1.0, last=kn_last).items()}
    M = {k: v / (6.0 * n) for k, v in _tridiag(n, 1.0, 4.0, 1.0, last=2.0).items()}
    E = {(n - 1, n - 1): 1.0}
    row_ptr, col_idx, values = _shared_csr(n, [K, E, M])
    fns = [Fn(F_ONE), Fn(F_RATIONAL, 1.0), Fn(F_ZPOW, 1, -1.0)]
    lo, hi = 3.0, 1.0e4
    i = np.arange(N)
    x = np.cos((2 * i + 1) * np.pi / (2 * N))
    pts = (0.5 * (hi + lo) + 0.5 * (hi - lo) * x).astype(np.complex128)
    reg = Region(complex(5001.5), 4998.5, 0.1 * 4998.5, kind="points", points=pts)
    return Problem(name, n, row_ptr, col_idx, values, fns, reg, N, L,
                   probe(n, L, seed_u), meta=dict(kn_last=kn_last, interval=(lo, hi)))


# ----------------------------------------------------------------------------
# closed-form test families: diagonal NEPs hidden by an orthogonal similarity
# ----------------------------------------------------------------------------

def givens_layers(n: int, layers: int, seed: int) -> np.ndarray:
    """Dense orthogonal G = product of `layers` layers of adjacent-pair Givens
    rotations with seeded angles.  G has half-bandwidths <= `layers`, so
    G^T D G has half-bandwidth <= 2*layers for diagonal D, and the same
    eigenvalues."""
    rng = np.random.default_rng(seed)
    G = np.eye(n)
    for lay in range(layers):
        start = lay % 2
        for p in range(start, n - 1, 2):
            th = rng.uniform(0.2, 1.3)
            c, s = np.cos(th), np.sin(th)
            rp, rq = G[p].copy(), G[p + 1].copy()
            G[p] = c * rp - s * rq
            G[p + 1] = s * rp + c * rq
    return G


def hidden_diagonal(diags: list, fns: list, region: Region, N: int, L: int,
                    layers: int = 3, seed: int = 5, seed_u: int = 6,
                    name: str = "hidden") -> Problem:
    """T(z) = G1^T diag(sum_i f_i(z) d_i) G2 with two different orthogonal G1,
    G2 from givens_layers (seeds `seed` and `seed`+100): a banded,
    non-symmetric NEP with det T(z) = +-det(diag(...)), so its eigenvalues are
    those of the n decoupled scalar problems sum_i f_i(z) d_i[r] = 0."""
    n = len(diags[0])
    G1 = givens_layers(n, layers, seed)
    G2 = givens_layers(n, layers, seed + 100)
    dt = np.complex128 if any(np.iscomplexobj(d) for d in diags) else np.float64
    dense = [G1.T @ np.diag(np.asarray(d, dtype=dt)) @ G2 for d in diags]
    w = 2 * layers
    row_ptr, col_idx, values = _csr_from_dense_band(dense, w, w)
    return Problem(name, n, row_ptr, col_idx, values, fns, region, N, L,
                   probe(n, L, seed_u), meta=dict(diags=[np.asarray(d) for d in diags],
                                                   layers=layers, g_seed=seed))


def diag_quadratic(n: int = 240, seed: int = 11, N: int = 32, L: int = 4,
                   layers: int = 3) -> Problem:
    """Decoupled quadratics k_r + z c_r + z^2 m_r, roots re +- i im with
    re ~ U(-6, 6), im ~ U(0.05, 8); a few percent of them lie in the region."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-6.0, 6.0, n)
    im = rng.uniform(0.05, 8.0, n)
    m = rng.uniform(0.5, 2.0, n)
    c = -2.0 * re * m
    k = m * (re ** 2 + im ** 2)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1), Fn(F_ZPOW, 2)]
    return hidden_diagonal([k, c, m], fns, Region(0.6j - 0.2, 1.0, 0.8), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_quadratic")


def diag_rational(n: int = 240, seed: int = 21, N: int = 32, L: int = 4,
                  sigma: float = 5.0, layers: int = 3) -> Problem:
    """Decoupled k_r - z m_r + (z/(z - sigma)) e_r (real roots)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.2, 40.0, n)
    m = rng.uniform(0.8, 1.2, n)
    e = rng.uniform(0.0, 0.5, n)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1, -1.0), Fn(F_RATIONAL, sigma)]
    return hidden_diagonal([k, m, e], fns, Region(2.0 + 0.0j, 1.5, 0.5), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_rational")


def diag_delay(n: int = 200, seed: int = 31, N: int = 48, L: int = 4,
               tau: float = 1.0, layers: int = 2) -> Problem:
    """Decoupled delay problems z - a_r - b_r exp(-tau z), a_r ~ U(-1, 8),
    b_r ~ U(0.05, 0.3): only the principal-branch roots of a minority of rows
    fall in the region."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 8.0, n)
    b = rng.uniform(0.05, 0.3, n)
    fns = [Fn(F_ZPOW, 1), Fn(F_ONE, 0.0, -1.0), Fn(F_EXP, tau, -1.0)]
    return hidden_diagonal([np.ones(n), a, b], fns, Region(0.5 + 0.0j, 0.6, 0.5), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_delay")


def diag_sqrt(n: int = 240, seed: int = 51, N: int = 32, L: int = 4, kappa: float = 1.0,
              layers: int = 3) -> Problem:
    """Decoupled k_r - z m_r + e_r sqrt(z^2 - kappa^2) (principal branch; the
    square-root coupling of Section 2.1), k_r ~ U(1.5, 40): one real root per
    row, near k_r / m_r.  The region (centre 5, semi-axes 1.5 / 0.5) stays away
    from the branch cuts (real |z| < kappa and the imaginary axis)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(1.5, 40.0, n)
    m = rng.uniform(0.8, 1.2, n)
    e = rng.uniform(0.05, 0.5, n)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1, -1.0), Fn(F_SQRT, kappa)]
    return hidden_diagonal([k, m, e], fns, Region(5.0 + 0.0j, 1.5, 0.5), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_sqrt")


def diag_inv(n: int = 240, seed: int = 61, N: int = 32, L: int = 4, sigma: float = 5.0,
             layers: int = 3) -> Problem:
    """Decoupled k_r - z m_r + e_r / (sigma - z) (the 1/(sigma - z) form of
    Section 2.1), real roots."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.2, 40.0, n)
    m = rng.uniform(0.8, 1.2, n)
    e = rng.uniform(0.05, 0.5, n)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1, -1.0), Fn(F_INV, sigma)]
    return hidden_diagonal([k, m, e], fns, Region(2.0 + 0.0j, 1.5, 0.5), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_inv")


def diag_quadratic_complex(n: int = 240, seed: int = 71, N: int = 32, L: int = 4,
                           layers: int = 3) -> Problem:
    """Decoupled quadratics k_r + z c_r + z^2 m_r with complex k, c, m (roots
    placed as in diag_quadratic, then all three coefficients multiplied by a
    seeded unit phase per row): a banded NEP with complex coefficient values."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-6.0, 6.0, n)
    im = rng.uniform(0.05, 8.0, n)
    m = rng.uniform(0.5, 2.0, n)
    c = -2.0 * re * m
    k = m * (re ** 2 + im ** 2)
    ph = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, n))
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1), Fn(F_ZPOW, 2)]
    return hidden_diagonal([k * ph, c * ph, m * ph], fns, Region(0.6j - 0.2, 1.0, 0.8), N, L,
                           layers=layers, seed=seed + 1, seed_u=seed + 2, name="diag_quadratic_complex")


def random_banded(n: int = 300, kl: int = 7, ku: int = 7, m: int = 3, seed: int = 41,
                  N: int = 8, L: int = 5) -> Problem:
    """Random real band matrices (every band entry present) with quadratic f;
    used for solve-level parity (no spectral content assumed)."""
    rng = np.random.default_rng(seed)
    dense = []
    for t in range(m):
        D = rng.standard_normal((n, n))
        D = np.triu(np.tril(D, ku), -kl)
        if t == 0:
            D += np.diag(np.full(n, 2.0 * (kl + ku)))
        dense.append(D)
    row_ptr, col_idx, values = _csr_from_dense_band(dense, kl, ku)
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1), Fn(F_ZPOW, 2)][:m]
    return Problem("random_banded", n, row_ptr, col_idx, values, fns,
                   Region(0.3 + 0.2j, 0.5, 0.4), N, L, probe(n, L, seed + 1))


# Benchmark configurations by name.
def config(name: str, **kw) -> Problem:
    if name == "c0":
        return quadratic_tridiag(**kw)
    if name == "c0b":
        kw.setdefault("center", -25.0 + 50.0j)
        return quadratic_tridiag(name="c0b", **kw)
    if name == "c1":
        return rational_grid(**kw)
    raise KeyError(name)


# ----------------------------------------------------------------------------
# dense BEM-like workload: single-layer Helmholtz kernel on a sphere
# ----------------------------------------------------------------------------

@dataclass
class DenseProblem:
    """T(z)_ij = exp(i z r_ij) / (4 pi r_ij) for i != j, T_ii = diag, with
    r_ij the distances between `points` (the BEM kernel of Section 2.1,
    Nystrom form with uniform weights)."""
    name: str
    n: int
    points: np.ndarray   # float64 [n, 3]
    diag: float
    region: Region
    N: int
    L: int
    U: np.ndarray        # complex128 [n, L], Fortran order
    meta: dict = field(default_factory=dict)


def fibonacci_sphere(n: int, seed: int) -> np.ndarray:
    """Quasi-uniform points on the unit sphere: Fibonacci lattice turned by a
    seeded random rotation (QR of a Gaussian matrix, sign-fixed)."""
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    theta = np.pi * (1.0 + 5.0 ** 0.5) * i
    P = np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)
    Qr, R = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    Qr = Qr * np.sign(np.diag(R))
    return np.ascontiguousarray(P @ Qr.T)


def mean_nn_distance(P: np.ndarray) -> float:
    """Mean nearest-neighbour distance of a point cloud (blockwise, O(n^2))."""
    n = len(P)
    best = np.full(n, np.inf)
    for s in range(0, n, 1024):
        d = np.linalg.norm(P[s:s + 1024, None, :] - P[None, :, :], axis=2)
        d[np.arange(d.shape[0]), np.arange(s, s + d.shape[0])] = np.inf
        best[s:s + 1024] = d.min(axis=1)
    return float(best.mean())


def helmholtz_sphere(n: int = 4096, N: int = 32, L: int = 64, center: complex = 3.0,
                     radius: float = 1.0, seed: int = 3000, seed_u: int = 3001,
                     name: str = "c2") -> DenseProblem:
    """Dense BEM-like NEP on the unit sphere: n points (Fibonacci lattice,
    seeded rotation), diagonal 1/(2h) with h the mean nearest-neighbour
    distance, circle region (centre 3, radius 1 for the benchmark shape)."""
    P = fibonacci_sphere(n, seed)
    h = mean_nn_distance(P)
    return DenseProblem(name, n, P, 1.0 / (2.0 * h), Region(complex(center), radius, radius), N, L,
                        probe(n, L, seed_u), meta=dict(h=h, seed=seed, seed_u=seed_u))


# ----------------------------------------------------------------------------
# request stream for the serving measurement: requests from the three
# benchmark families with randomised regions and sizes
# ----------------------------------------------------------------------------

def serving_stream(count: int = 48, seed: int = 5000):
    """`count` requests, family uniform over {quadratic tridiagonal (c0
    shape), rational grid (c1 shape), dense sphere kernel (c2 shape)}, sizes
    and regions drawn from `seed`.  Returns a list of (family, problem).
    Sizes are scaled down from the full configs so that a stream of tens of
    requests runs in seconds: grid side 40..100, dense n 128..512."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = ("quadratic", "grid", "dense")[int(rng.integers(0, 3))]
        s_u = seed + 1 + i
        if fam == "quadratic":
            p = quadratic_tridiag(n=1000, N=32, L=8,
                                  center=complex(-25.0, float(rng.uniform(40.0, 60.0))),
                                  radius=40.0, seed_u=s_u, name="c0_req")
        elif fam == "grid":
            g = int(rng.integers(40, 101))
            p = rational_grid(g=g, N=int(rng.choice([32, 64])), L=int(rng.choice([8, 16, 32])),
                              center=float(rng.uniform(70.0, 130.0)), seed_u=s_u, name="c1_req")
        else:
            n = int(rng.integers(128, 513))
            p = helmholtz_sphere(n=n, N=32, L=int(rng.choice([8, 16])),
                                 center=complex(float(rng.uniform(2.9, 3.1)), 0.0),
                                 seed_u=s_u, name="c2_req")
        out.append((fam, p))
    return out


def batch_uneven(count: int = 256, seed: int = 4000, dense_n=(256, 2048), grid_g=(100, 316),
                 N=(16, 64), L=(8, 32)):
    """The batched uneven workload: `count` problems, half dense sphere kernels
    with n uniform in dense_n, half rational grids with side g uniform in
    grid_g, N uniform in N and L uniform in L, in a seeded shuffled order.
    Returns a list of (family, problem)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nN = int(rng.integers(N[0], N[1] + 1))
        nL = int(rng.integers(L[0], L[1] + 1))
        if i % 2 == 0:
            n = int(rng.integers(dense_n[0], dense_n[1] + 1))
            out.append(("dense", helmholtz_sphere(n=n, N=nN, L=nL, seed=seed + 1 + i,
                                                  seed_u=seed + 10001 + i, name="c3_dense")))
        else:
            g = int(rng.integers(grid_g[0], grid_g[1] + 1))
            out.append(("grid", rational_grid(g=g, N=nN, L=nL, seed_e=seed + 1 + i,
                                              seed_u=seed + 10001 + i, name="c3_grid")))
    order = rng.permutation(count)
    return [out[k] for k in order]


# ----------------------------------------------------------------------------
# general dense terms: T(z) = sum_i f_i(z) A_i with caller-supplied dense A_i
# ----------------------------------------------------------------------------

@dataclass
class DenseTermsProblem:
    """T(z) = sum_i f_i(z) A_i with dense complex A_i (n x n)."""
    name: str
    n: int
    As: list             # m complex128 [n, n]
    fns: list            # m Fn
    region: Region
    N: int
    L: int
    U: np.ndarray        # complex128 [n, L], Fortran order
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return len(self.As)


def random_unitary(n: int, seed: int) -> np.ndarray:
    """Haar-like unitary: QR of a complex Gaussian matrix with the phases of
    R's diagonal moved into Q."""
    rng = np.random.default_rng(seed)
    Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    Qm, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Qm * (d / np.abs(d))


def dense_hidden_quadratic(n: int = 200, seed: int = 81, N: int = 32, L: int = 4) -> DenseTermsProblem:
    """Decoupled quadratics k_r + z c_r + z^2 m_r (as diag_quadratic) hidden by
    one seeded unitary W: A_i = W diag(d_i) W^H, dense and complex; the
    eigenvalues are the scalar roots."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-6.0, 6.0, n)
    im = rng.uniform(0.05, 8.0, n)
    m = rng.uniform(0.5, 2.0, n)
    c = -2.0 * re * m
    k = m * (re ** 2 + im ** 2)
    Wm = random_unitary(n, seed + 1)
    As = [np.asfortranarray((Wm * d[None, :]) @ Wm.conj().T) for d in (k, c, m)]
    fns = [Fn(F_ONE), Fn(F_ZPOW, 1), Fn(F_ZPOW, 2)]
    return DenseTermsProblem("dense_hidden_quadratic", n, As, fns, Region(0.6j - 0.2, 1.0, 0.8), N, L,
                             probe(n, L, seed + 2), meta=dict(diags=[k, c, m], seed=seed))


# ----------------------------------------------------------------------------
# gun-type NEP: square-root couplings on a 2-D grid, rectangular region
# ----------------------------------------------------------------------------

def gun_like(gx: int = 100, gy: int = 100, N: int = 80, L: int = 2, nx: int = 27,
             alpha: float = 2405.0, beta: float = 3295.0, w1: float = 1.0e4,
             w2: float = 1.0e4, kappa2: float = 108.8774, seed_u: int = 9001,
             name: str = "gun_like") -> Problem:
    """T(z) = K - z^2 M + i sqrt(z^2 - kappa_1^2) W_1 + i sqrt(z^2 - kappa_2^2) W_2
    (the radio-frequency gun form of Section 5.4, kappa_1 = 0, kappa_2 =
    108.8774), synthetic: K is the anisotropic 5-point stiffness of a gx x gy
    grid with Dirichlet sides (natural row-major ordering, half-bandwidth gx),
    sx (2 - shifts along x) + sy (2 - shifts along y) with sx = alpha (gx+1)^2
    / pi^2, sy = beta (gy+1)^2 / pi^2, so that the undamped z^2 are about
    alpha i^2 + beta j^2; M = I; W_1 = w1 on the grid line x = 0, W_2 = w2 on
    the line x = gx - 1 (the two ports, diagonal).  The damped eigenvalues lie
    just above the real axis (imaginary parts up to about 3), so the
    rectangle is [215, 330] x [-10, 40], its vertical sides in gaps of the
    spectrum (fifteen eigenvalues inside, none within 6 of the contour), with
    Gauss-Legendre sampling points, nx on each horizontal side (27 and 13 for
    N = 80, the paper's rule)."""
    n = gx * gy
    idx = np.arange(n)
    gi, gj = idx // gx, idx % gx          # row (y) and column (x) of the grid node
    sx = alpha * (gx + 1) ** 2 / np.pi ** 2
    sy = beta * (gy + 1) ** 2 / np.pi ** 2
    K, M, W1, W2 = {}, {}, {}, {}
    for r in range(n):
        K[(r, r)] = 2.0 * sx + 2.0 * sy
        M[(r, r)] = 1.0
    for r in range(n):
        if gj[r] + 1 < gx:
            K[(r, r + 1)] = K[(r + 1, r)] = -sx
        if gi[r] + 1 < gy:
            K[(r, r + gx)] = K[(r + gx, r)] = -sy
    for r in idx[gj == 0]:
        W1[(int(r), int(r))] = w1
    for r in idx[gj == gx - 1]:
        W2[(int(r), int(r))] = w2
    row_ptr, col_idx, values = _shared_csr(n, [K, M, W1, W2])
    fns = [Fn(F_ONE), Fn(F_ZPOW, 2, -1.0), Fn(F_SQRT, 0.0, 1j), Fn(F_SQRT, kappa2, 1j)]
    reg = Region(272.5 + 15.0j, 57.5, 25.0, kind="rect", nx=nx)
    return Problem(name, n, row_ptr, col_idx, values, fns, reg, N, L, probe(n, L, seed_u),
                   meta=dict(gx=gx, gy=gy, alpha=alpha, beta=beta, w1=w1, w2=w2, kappa2=kappa2))
