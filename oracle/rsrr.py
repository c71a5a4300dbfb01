"""Plain FP64 CPU oracle of resolvent sampling + Rayleigh-Ritz (RSRR).

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  It shares no code with the CUDA path
and never reads anything the CUDA path produced.

Every function follows a passage of Xiao, Zhang, Huang, Sakurai, "Solving
large-scale nonlinear eigenvalue problems by rational interpolation approach
and resolvent sampling based Rayleigh-Ritz method" (2016), cited in its
docstring.  Library primitives (banded/dense LAPACK solves, SVD, eig) serve as
single steps; nothing is blocked, fused or reordered beyond the paper's
algorithm.

Parity status per function:
  sample_points, quad_weights ........ pinned (ellipse equation, Cauchy integral)
  eval_fn, assemble .................. pinned (decoupled closed forms)
  resolvent_samples .................. pinned (decoupled closed forms, residual)
  truncated_basis, project, ss_full .. pinned (closed-form spectra, inertia counts,
                                       companion linearisation, Lambert W, the
                                       loaded-string example of Section 5.2)
  rsrr ............................... pinned (as above)
  backward_error_inf, residual,
  backward_error_inf_dense,
  residual_dense ..................... pinned (hand-computed values on a 3 x 3
                                       non-symmetric T and the two-point kernel,
                                       tests/golden/checker_norms.json; the
                                       Rigal-Gaches minimal perturbation; planted
                                       mutations of each fail a pin)
  assemble_dense, taylor_coefficients,
  resolvent_samples_dense, rsrr_dense  pinned (two-point problem with closed-form
                                       eigenvalues k pi / r + i im and eigenvectors;
                                       Taylor series against the kernel matrix;
                                       argument-principle counts)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from workloads import (F_ONE, F_ZPOW, F_RATIONAL, F_INV, F_SQRT, F_EXP, F_TAYLOR, F_CALLBACK,
                       Problem, Region)


# ---------------------------------------------------------------------------
# Step 1 of RSRR: sampling points (Section 5.1, ellipse contour and N-point
# trapezoid rule; the RIA allows explicit points, Section 3.3)
# ---------------------------------------------------------------------------

def sample_points(region: Region, N: int) -> np.ndarray:
    """z_j = phi(alpha_j), alpha_j = 2 pi (j + 1/2)/N on the ellipse
    phi(alpha) = gamma + a cos(alpha) + i b sin(alpha) (Section 5.1, ellipse
    contour and trapezoid nodes), the region's explicit points, the
    Chebyshev points of the first kind x_i = cos((2i + 1) pi / 2N) (Eq. 42)
    mapped to the interval [gamma - a, gamma + a] (Section 3.3, real points
    for an interval of interest), or Gauss-Legendre nodes on the sides of a
    rectangle (Section 5.4; explicit points with a rectangular contour for
    the second stage of two-stage sampling)."""
    if region.kind == "points" or (region.kind == "rect" and region.points is not None):
        return np.asarray(region.points, dtype=np.complex128).copy()
    if region.kind == "interval":
        i = np.arange(N)
        return region.center + region.a * np.cos((2 * i + 1) * np.pi / (2 * N)) + 0j
    if region.kind == "rect":
        return rect_rule(region, rect_counts(region, N))[0]
    j = np.arange(N)
    alpha = 2.0 * np.pi * (j + 0.5) / N
    return region.center + region.a * np.cos(alpha) + 1j * region.b * np.sin(alpha)


# ---------------------------------------------------------------------------
# Rectangular contour (Section 5.4: Gauss-Legendre nodes on the four sides,
# composite Gauss quadrature for the contour integrals of SS-FULL)
# ---------------------------------------------------------------------------

def gauss_legendre(n: int):
    """Nodes x_k and weights w_k of the n-point Gauss-Legendre rule on
    [-1, 1] (numpy's leggauss as the library primitive)."""
    return np.polynomial.legendre.leggauss(n)


def rect_sides(region: Region) -> list:
    """The four sides (start, end) counterclockwise from the lower-left
    vertex center - a - i b."""
    c, a, b = complex(region.center), region.a, region.b
    v = [c - a - 1j * b, c + a - 1j * b, c + a + 1j * b, c - a + 1j * b]
    return [(v[s], v[(s + 1) % 4]) for s in range(4)]


def rect_counts(region: Region, N: int) -> list:
    """Sampling points per side: nx on the two sides parallel to the real
    axis, N/2 - nx on the other two (27 and 13 for N = 80 in Section 5.4)."""
    ny = N // 2 - region.nx
    return [region.nx, ny, region.nx, ny]


def rect_rule(region: Region, counts: list):
    """Gauss-Legendre nodes on each side (counts[s] of them on side s,
    increasing along the side's direction) and the contour weights
    omega = dz / (2 pi): for a side from p to q, z = (p + q)/2 + (q - p) x/2,
    dz = (q - p) w / 2 -- the same normalisation as the trapezoid weights
    (1/N) phi'(alpha) of the ellipse (a change of 1/i, common to all)."""
    zs, ws = [], []
    for (p, q), c in zip(rect_sides(region), counts):
        x, w = gauss_legendre(int(c))
        zs.append(0.5 * (p + q) + 0.5 * (q - p) * x)
        ws.append(0.5 * (q - p) * w / (2.0 * np.pi))
    return np.concatenate(zs), np.concatenate(ws)


RECT_PANEL = 10  # nodes of one Gauss-Legendre panel of the composite rule


def contour_quadrature(region: Region, NQ: int):
    """Nodes and weights omega_q of the contour integrals of SS-FULL: the
    NQ-point trapezoid rule on the ellipse (Eq. 58), or on the rectangle
    composite Gauss quadrature (Section 5.4): side s of length len_s is cut
    into P_s = max(1, round(NQ len_s / (10 perimeter))) equal panels, each
    with the 10-point Gauss-Legendre rule."""
    if region.kind != "rect":
        zq = sample_points(Region(region.center, region.a, region.b), NQ)
        return zq, quad_weights(region, NQ)
    per = 4.0 * (region.a + region.b)
    x, w = gauss_legendre(RECT_PANEL)
    zs, ws = [], []
    for p, q in rect_sides(region):
        P = max(1, int(round(NQ * abs(q - p) / (RECT_PANEL * per))))
        for t in range(P):
            a0, a1 = p + (q - p) * t / P, p + (q - p) * (t + 1) / P
            zs.append(0.5 * (a0 + a1) + 0.5 * (a1 - a0) * x)
            ws.append(0.5 * (a1 - a0) * w / (2.0 * np.pi))
    return np.concatenate(zs), np.concatenate(ws)


def quad_weights(region: Region, NQ: int) -> np.ndarray:
    """omega_j = (1/N) dphi/dalpha at alpha_j (Section 5.1 trapezoid rule)."""
    j = np.arange(NQ)
    alpha = 2.0 * np.pi * (j + 0.5) / NQ
    return (-region.a * np.sin(alpha) + 1j * region.b * np.cos(alpha)) / NQ


def inside(region: Region, z) -> np.ndarray:
    """Strict interior of the ellipse ((x-gr)/a)^2 + ((y-gi)/b)^2 < 1, or of
    the rectangle |x - gr| < a, |y - gi| < b."""
    z = np.asarray(z)
    x = (z.real - complex(region.center).real) / region.a
    y = (z.imag - complex(region.center).imag) / region.b
    if region.kind == "rect":
        return (np.abs(x) < 1.0) & (np.abs(y) < 1.0)
    return x * x + y * y < 1.0


# ---------------------------------------------------------------------------
# The NEP T(z) = sum_i f_i(z) A_i (Eq. 1 and the families of Section 2.1)
# ---------------------------------------------------------------------------

def eval_fn(fn, z):
    """Scalar coefficient f_i(z) = scale * base(z) for the families of
    Section 2.1 (polynomial, rational z/(z - sigma) and 1/(sigma - z),
    square root sqrt(z^2 - kappa^2)) plus exp(-tau z) for delay problems."""
    z = np.asarray(z, dtype=np.complex128)
    if fn.kind == F_ONE:
        base = np.ones_like(z)
    elif fn.kind == F_ZPOW:
        base = z ** int(fn.param)
    elif fn.kind == F_RATIONAL:
        base = z / (z - fn.param)
    elif fn.kind == F_INV:
        base = 1.0 / (fn.param - z)
    elif fn.kind == F_SQRT:
        base = np.sqrt(z * z - fn.param * fn.param)
    elif fn.kind == F_EXP:
        base = np.exp(-fn.param * z)
    elif fn.kind == F_TAYLOR:
        base = (z - complex(fn.shift)) ** int(fn.power)
    elif fn.kind == F_CALLBACK:
        base = np.asarray(fn.callback(np.atleast_1d(z)), dtype=np.complex128).reshape(z.shape)
    else:
        raise ValueError(f"unknown function kind {fn.kind}")
    return complex(fn.scale) * base


def coeff_matrix(prob: Problem, i: int):
    """A_i as a scipy CSR matrix on the shared pattern."""
    import scipy.sparse as sp
    return sp.csr_matrix((prob.values[i], prob.col_idx, prob.row_ptr), shape=(prob.n, prob.n))


def assemble(prob: Problem, z: complex):
    """T(z) = sum_i f_i(z) A_i (Eq. 1 with the form of Section 2.1)."""
    vals = np.zeros(prob.nnz, dtype=np.complex128)
    for fn, v in zip(prob.fns, prob.values):
        vals += eval_fn(fn, z) * v
    import scipy.sparse as sp
    return sp.csr_matrix((vals, prob.col_idx, prob.row_ptr), shape=(prob.n, prob.n))


def _to_band(T, kl: int, ku: int) -> np.ndarray:
    """LAPACK general band layout ab[ku + i - j, j] = T[i, j]."""
    n = T.shape[0]
    ab = np.zeros((kl + ku + 1, n), dtype=np.complex128)
    coo = T.tocoo()
    ab[ku + coo.row - coo.col, coo.col] = coo.data
    return ab


# ---------------------------------------------------------------------------
# Step 2 of RSRR: the resolvent samples X_j = T(z_j)^{-1} U (Section 4.3)
# ---------------------------------------------------------------------------

def resolvent_samples(prob: Problem, z: np.ndarray, U: np.ndarray | None = None) -> list:
    """X_j = T(z_j)^{-1} U for each sampling point (Section 4.3, step 2),
    by a banded LU solve with partial pivoting (LAPACK gbsv) per point."""
    if U is None:
        U = prob.U
    kl, ku = prob.bandwidths()
    out = []
    for zj in z:
        ab = _to_band(assemble(prob, zj), kl, ku)
        out.append(sla.solve_banded((kl, ku), ab, U, check_finite=False))
    return out


def backward_error_inf(prob: Problem, z: complex, X: np.ndarray, U: np.ndarray | None = None):
    """Per-column normwise backward error
    eta = ||U - T(z) X||_inf / (||T(z)||_inf ||X||_inf + ||U||_inf)."""
    if U is None:
        U = prob.U
    T = assemble(prob, z)
    R = U - T @ X
    tn = np.abs(T).sum(axis=1).max()
    num = np.abs(R).max(axis=0)
    den = tn * np.abs(X).max(axis=0) + np.abs(U).max(axis=0)
    return num / den


# ---------------------------------------------------------------------------
# Step 3 of RSRR: S, column normalisation, truncated SVD (Eq. 51, Section 4.2
# last paragraph, Section 4.3 step 3)
# ---------------------------------------------------------------------------

def sample_matrix(samples: list) -> np.ndarray:
    """S = [T(z_0)^{-1}U, ..., T(z_{N-1})^{-1}U] (Eq. 51 in Section 4.2)."""
    return np.concatenate(samples, axis=1)


def normalize_columns(S: np.ndarray) -> np.ndarray:
    """Scale every column of S to unit 2-norm before the SVD (Section 4.2)."""
    return S / np.linalg.norm(S, axis=0, keepdims=True)


def truncated_basis(S: np.ndarray, delta: float = 1e-14):
    """S ~ Q Sigma V^H keeping the k singular values > delta*sigma_1
    (Section 4.3 step 3; delta = 1e-14 as in the paper)."""
    Qf, sig, _ = np.linalg.svd(S, full_matrices=False)
    k = int(np.sum(sig > delta * sig[0]))
    return Qf[:, :k], sig, k


# ---------------------------------------------------------------------------
# Step 4 of RSRR: projection T_Q(z) = Q^H T(z) Q (Eq. 45, Section 4)
# ---------------------------------------------------------------------------

def project(prob: Problem, Q: np.ndarray) -> list:
    """P_i = Q^H A_i Q so that T_Q(z) = sum_i f_i(z) P_i."""
    return [Q.conj().T @ (coeff_matrix(prob, i) @ Q) for i in range(prob.m)]


def ss_full(P: list, fns: list, region: Region, NQ: int = 500, KQ: int = 2,
            tol_gap: float = 1e3):
    """SS-FULL: the SS-RI algorithm of Section 3.3 with U = I (F = T_Q^{-1}),
    quadrature nodes on the contour: the trapezoid rule on the ellipse
    (Section 5.1) or composite Gauss on the rectangle (Section 5.4).

    Moments A_alpha = sum_q omega_q ((z_q - gamma)/rho)^alpha F(z_q), alpha <
    2 KQ (the scaled-moment reading: a fixed change of basis of z that keeps
    the pencil's eigenvalues, applied against overflow), block Hankel H, H^<
    (Eq. 33), truncated SVD of H with the count fixed by the largest gap
    sigma_j/sigma_{j+1} (gap strategy, tol_gap = 1e3), A = V0^H H^< W0
    Sigma0^{-1} (Eq. 38), eigenpairs of A, and g = M W0 Sigma0^{-1} b
    (Eq. 41) with M = [A_0 ... A_{KQ-1}] since U = I.

    Returns (lam, G, info): eigenvalues of the projected NEP, the projected
    eigenvectors as columns of G, and {"nbar", "gmax", "sv"}.
    """
    k = P[0].shape[0]
    zq, wq = contour_quadrature(region, NQ)
    gamma = region.center
    rho = max(region.a, region.b)
    Amom = [np.zeros((k, k), dtype=np.complex128) for _ in range(2 * KQ)]
    I = np.eye(k, dtype=np.complex128)
    for z, w in zip(zq, wq):
        TQ = sum(eval_fn(fn, z) * Pi for fn, Pi in zip(fns, P))
        F = np.linalg.solve(TQ, I)
        s = (z - gamma) / rho
        for al in range(2 * KQ):
            Amom[al] += w * s ** al * F
    H = np.block([[Amom[i + j] for j in range(KQ)] for i in range(KQ)])
    Hs = np.block([[Amom[i + j + 1] for j in range(KQ)] for i in range(KQ)])
    V, sv, Wh = np.linalg.svd(H)
    ratios = sv[:-1] / np.maximum(sv[1:], np.finfo(float).tiny)
    nbar = int(np.argmax(ratios)) + 1
    gmax = float(ratios[nbar - 1])
    V0 = V[:, :nbar]
    W0 = Wh.conj().T[:, :nbar]
    S0inv = np.diag(1.0 / sv[:nbar])
    A = V0.conj().T @ Hs @ W0 @ S0inv
    lam_s, B = np.linalg.eig(A)
    lam = gamma + rho * lam_s
    Mmat = np.concatenate(Amom[:KQ], axis=1)
    G = Mmat @ W0 @ S0inv @ B
    return lam, G, dict(nbar=nbar, gmax=gmax, sv=sv)


# ---------------------------------------------------------------------------
# Residual measure (Section 5.4, E(v, lambda) with the 1-norms of the A_i)
# ---------------------------------------------------------------------------

def residual(prob: Problem, lam: complex, v: np.ndarray) -> float:
    """rho(lam, v) = ||T(lam) v||_2 / ((sum_i |f_i(lam)| ||A_i||_1) ||v||_2),
    the normalised relative residual of Section 5.4."""
    T = assemble(prob, lam)
    scale = 0.0
    for i, fn in enumerate(prob.fns):
        a1 = np.abs(coeff_matrix(prob, i)).sum(axis=0).max()
        scale += abs(eval_fn(fn, lam)) * a1
    return float(np.linalg.norm(T @ v) / (scale * np.linalg.norm(v)))


def plain_residual(prob: Problem, lam: complex, v: np.ndarray) -> float:
    """||T(lam) v||_2 / ||v||_2 (Section 3.3, gap-strategy remark)."""
    return float(np.linalg.norm(assemble(prob, lam) @ v) / np.linalg.norm(v))


# ---------------------------------------------------------------------------
# The whole method (Section 4.3, steps 1-5)
# ---------------------------------------------------------------------------

def rsrr(prob: Problem, delta: float = 1e-14, NQ: int = 500, KQ: int = 2,
         tol_gap: float = 1e3, U: np.ndarray | None = None, res_tol: float = 1e-6):
    """RSRR: points and probes (step 1), X_j = T(z_j)^{-1}U (step 2), S with
    normalised columns and truncated SVD basis Q (step 3), T_Q = Q^H T Q solved
    by SS-FULL (step 4), v = Q g (step 5).

    Acceptance (readings): only pairs strictly inside the contour are kept (the
    method asks for the n_C pairs inside), and, following the advice of the
    gap-strategy paragraph of Section 3.3 to check residuals, a pair is kept
    only if its normalised residual is <= res_tol."""
    z = sample_points(prob.region, prob.N)
    X = resolvent_samples(prob, z, U)
    S = normalize_columns(sample_matrix(X))
    Q, sig, k = truncated_basis(S, delta)
    P = project(prob, Q)
    lam, G, info = ss_full(P, prob.fns, prob.region, NQ, KQ, tol_gap)
    V = Q @ G
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    keep = inside(prob.region, lam)
    lam, V = lam[keep], V[:, keep]
    res = np.array([residual(prob, l, V[:, c]) for c, l in enumerate(lam)])
    ok = res <= res_tol
    lam, V, res = lam[ok], V[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    lam, V, res = lam[order], V[:, order], res[order]
    return dict(lam=lam, V=V, res=res, k=k, sigma=sig, info=info, z=z, X=X, P=P, Q=Q)


# ---------------------------------------------------------------------------
# Independent counting tools used as pins (no RSRR arithmetic)
# ---------------------------------------------------------------------------

def negative_inertia(prob: Problem, x: float) -> int:
    """nu(T(x)): number of negative eigenvalues of the real symmetric T(x)
    (dense symmetric eigenvalues; small problems only)."""
    T = assemble(prob, x).toarray().real
    return int(np.sum(np.linalg.eigvalsh(T) < 0.0))


_INERTIA_LIB = None


def _inertia_lib():
    """The plain-C band LDL^T of oracle/band_inertia.c, compiled on first use
    (gcc, into oracle/_band_inertia.so) and loaded with ctypes."""
    global _INERTIA_LIB
    if _INERTIA_LIB is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src = os.path.join(here, "band_inertia.c")
        lib = os.path.join(here, "_band_inertia.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".{os.getpid()}.tmp"
            subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src], check=True)
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        L.band_ldlt_negcount.restype = ctypes.c_int
        L.band_ldlt_negcount.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        _INERTIA_LIB = L
    return _INERTIA_LIB


def negative_inertia_band(prob: Problem, x: float) -> int:
    """nu(T(x)) by Sylvester's law of inertia: the number of negative pivots of
    the symmetric band LDL^T of the real symmetric T(x) (oracle/band_inertia.c),
    usable at full size (n = 40000, half-bandwidth 200).  Raises if a pivot is
    exactly zero."""
    T = assemble(prob, x).tocoo()
    if np.abs(T.data.imag).max(initial=0.0) != 0.0:
        raise ValueError("T(x) is not real")
    low = T.row >= T.col
    bw = int((T.row - T.col).max(initial=0))
    ab = np.zeros((prob.n, bw + 1), dtype=np.float64)   # row j = column j of the band
    ab[T.col[low], (T.row - T.col)[low]] = T.data.real[low]
    ab = np.ascontiguousarray(ab)
    neg = _inertia_lib().band_ldlt_negcount(prob.n, bw, ab.ctypes.data, bw + 1)
    if neg < 0:
        raise ZeroDivisionError(f"zero pivot in the LDL^T of T({x})")
    return int(neg)


def bisect_real_eigenvalues(prob: Problem, lo: float, hi: float, rtol: float = 1e-13,
                            count_fn=None) -> np.ndarray:
    """Every eigenvalue of a real symmetric NEP with T'(x) negative definite in
    (lo, hi), by bisection on the inertia count: #eigenvalues in (a, b) =
    nu(T(b)) - nu(T(a)).  Intervals are split until each holds one eigenvalue
    (or one multiple eigenvalue), which is then bisected to rtol."""
    nu = count_fn or (lambda x: negative_inertia_band(prob, x))
    out = []
    stack = [(lo, hi, nu(lo), nu(hi))]
    while stack:
        a, b, na, nb = stack.pop()
        c = nb - na
        if c <= 0:
            continue
        if b - a <= rtol * max(abs(a), abs(b)):
            out += [0.5 * (a + b)] * c
            continue
        mid = 0.5 * (a + b)
        nm = nu(mid)
        if c == 1 or nm in (na, nb):
            # one eigenvalue (or a cluster not split yet) on one side of mid
            stack.append((a, mid, na, nm) if nm > na else (mid, b, nm, nb))
            if nm != na and nm != nb:
                stack.append((mid, b, nm, nb))
        else:
            stack.append((a, mid, na, nm))
            stack.append((mid, b, nm, nb))
    return np.sort(np.array(out, dtype=np.float64))


def contour_path(region: Region, t: np.ndarray) -> np.ndarray:
    """The closed contour at parameters t in [0, 1], counterclockwise: the
    ellipse phi(2 pi t), or the rectangle's perimeter at arc length
    t * perimeter from the lower-left vertex."""
    t = np.asarray(t, dtype=np.float64)
    if region.kind != "rect":
        al = 2.0 * np.pi * t
        return region.center + region.a * np.cos(al) + 1j * region.b * np.sin(al)
    sides = rect_sides(region)
    lens = np.array([abs(q - p) for p, q in sides])
    cum = np.concatenate([[0.0], np.cumsum(lens)]) / lens.sum()
    out = np.empty(t.shape, dtype=np.complex128)
    for s, (p, q) in enumerate(sides):
        sel = (t >= cum[s]) & ((t < cum[s + 1]) if s < 3 else (t <= cum[4]))
        out[sel] = p + (q - p) * (t[sel] - cum[s]) / (cum[s + 1] - cum[s])
    return out


def phase_det_band(prob: Problem, z: complex) -> float:
    """arg det T(z) from the banded LU with partial pivoting (LAPACK zgbtrf as
    the library primitive): det = (-1)^(row swaps) prod u_ii."""
    from scipy.linalg.lapack import zgbtrf
    kl, ku = prob.bandwidths()
    T = assemble(prob, z).tocoo()
    ab = np.zeros((2 * kl + ku + 1, prob.n), dtype=np.complex128)
    ab[kl + ku + T.row - T.col, T.col] = T.data
    lu, piv, info = zgbtrf(ab, kl, ku)
    d = lu[kl + ku, :]
    swaps = int(np.count_nonzero(piv != np.arange(prob.n)))
    return float(np.angle(np.prod(d / np.abs(d))) + np.pi * (swaps % 2))


def argument_principle_count(prob: Problem, region: Region, npts: int = 4096,
                             band: bool = False) -> int:
    """Number of zeros of det T inside the contour: the winding number of
    det T along the closed contour (contour_path), with the phase unwrapped and
    the contour refined until every step changes the argument by < pi/4.
    band=True takes the phase from the banded LU (large n)."""
    def logdet(z):
        if band:
            return phase_det_band(prob, z)
        T = assemble(prob, z).toarray()
        sgn, _ = np.linalg.slogdet(T)
        return np.angle(sgn)

    alpha = np.linspace(0.0, 1.0, npts + 1)
    while True:
        zz = contour_path(region, alpha)
        ph = np.array([logdet(z) for z in zz])
        d = np.angle(np.exp(1j * np.diff(ph)))
        if np.all(np.abs(d) < np.pi / 4) or len(alpha) > 1 << 16:
            break
        alpha = np.sort(np.concatenate([alpha, 0.5 * (alpha[1:] + alpha[:-1])]))
    return int(round(d.sum() / (2.0 * np.pi)))


def companion_eigvals(prob: Problem) -> np.ndarray:
    """All eigenvalues of a quadratic NEP T(z) = B0 + z B1 + z^2 B2 (B_i the
    scaled coefficient matrices) from its first companion linearisation
    [[0, I], [-B0, -B1]] w = z [[I, 0], [0, B2]] w, solved densely (QZ).
    Brute force used to pin the RSRR count and eigenvalues of quadratic
    problems (linearisation of polynomial problems is the standard route the
    paper's Section 1 reviews)."""
    B = [None, None, None]
    for i, fn in enumerate(prob.fns):
        if fn.kind == F_ONE:
            p = 0
        elif fn.kind == F_ZPOW and int(fn.param) in (1, 2):
            p = int(fn.param)
        else:
            raise ValueError("companion_eigvals needs a quadratic NEP")
        Ai = complex(fn.scale) * coeff_matrix(prob, i).toarray()
        B[p] = Ai if B[p] is None else B[p] + Ai
    n = prob.n
    B = [np.zeros((n, n)) if b is None else b for b in B]
    Z, I = np.zeros((n, n)), np.eye(n)
    A = np.block([[Z, I], [-B[0], -B[1]]])
    Bm = np.block([[I, Z], [Z, B[2]]])
    return sla.eigvals(A, Bm)


# ---------------------------------------------------------------------------
# Dense BEM-like problems (Section 2.1, Nystrom single-layer kernel)
# ---------------------------------------------------------------------------

def distances(prob) -> np.ndarray:
    P = prob.points
    return np.linalg.norm(P[:, None, :] - P[None, :, :], axis=2)


def assemble_dense(prob, z: complex, R: np.ndarray | None = None) -> np.ndarray:
    """T(z)_ij = exp(i z r_ij)/(4 pi r_ij) for i != j, T_ii = diag."""
    if R is None:
        R = distances(prob)
    n = prob.n
    off = ~np.eye(n, dtype=bool)
    T = np.empty((n, n), dtype=np.complex128)
    T[off] = np.exp(1j * z * R[off]) / (4.0 * np.pi * R[off])
    T[~off] = prob.diag
    return T


def resolvent_samples_dense(prob, z: np.ndarray, U: np.ndarray | None = None) -> list:
    """X_j = T(z_j)^{-1} U by dense LU with partial pivoting (LAPACK gesv)."""
    if U is None:
        U = prob.U
    R = distances(prob)
    return [np.linalg.solve(assemble_dense(prob, zj, R), U) for zj in z]


def taylor_terms(prob, R: np.ndarray | None = None) -> int:
    """Smallest P with (r_max rho)^P / P! < 1e-17, rho = max(a, b): the
    remainder bound of the Taylor series of exp(i z r) about the centre."""
    if R is None:
        R = distances(prob)
    x = R.max() * max(prob.region.a, prob.region.b)
    P, term = 0, 1.0
    while term >= 1e-17:
        P += 1
        term *= x / P
    return P


def taylor_coefficients(prob, R: np.ndarray | None = None, P: int | None = None) -> list:
    """A_p with T(z) = sum_{p<P} (z - c)^p A_p: A_p(i,j) = e^{i c r}(i r)^p /
    (p! 4 pi r) off the diagonal, A_0 diagonal = diag, A_p diagonal = 0 (p > 0).
    The Taylor series of exp(i z r) about the region centre c: the
    interpolation of T that makes T_Q = Q^H T Q computable (Section 6 uses
    a Chebyshev interpolant for the same purpose)."""
    if R is None:
        R = distances(prob)
    if P is None:
        P = taylor_terms(prob, R)
    c = prob.region.center
    n = prob.n
    off = ~np.eye(n, dtype=bool)
    base = np.zeros((n, n), dtype=np.complex128)
    base[off] = np.exp(1j * c * R[off]) / (4.0 * np.pi * R[off])
    out = []
    term = base.copy()
    for p in range(P):
        A = term.copy()
        if p == 0:
            A[~off] = prob.diag
        out.append(A)
        term = term * (1j * R) / (p + 1)
    return out


def residual_dense(prob, lam: complex, v: np.ndarray, R: np.ndarray | None = None) -> float:
    """||T(lam) v||_2 / (||T(lam)||_1 ||v||_2), the 1-norm computed directly."""
    T = assemble_dense(prob, lam, R)
    return float(np.linalg.norm(T @ v) / (np.abs(T).sum(axis=0).max() * np.linalg.norm(v)))


def backward_error_inf_dense(prob, z: complex, X: np.ndarray, U: np.ndarray | None = None):
    """Per-column eta = ||U - T X||_inf / (||T||_inf ||X||_inf + ||U||_inf)."""
    if U is None:
        U = prob.U
    T = assemble_dense(prob, z)
    Rr = U - T @ X
    tn = np.abs(T).sum(axis=1).max()
    return np.abs(Rr).max(axis=0) / (tn * np.abs(X).max(axis=0) + np.abs(U).max(axis=0))


def rsrr_dense(prob, delta: float = 1e-14, NQ: int = 500, KQ: int = 2, tol_gap: float = 1e3,
               U: np.ndarray | None = None, res_tol: float = 1e-6):
    """RSRR (Section 4.3) for the dense kernel problem: samples by dense
    solves, the truncated SVD basis of the normalised S, projection of the
    Taylor coefficients P_p = Q^H A_p Q, SS-FULL on T_Q(z) = sum_p (z-c)^p P_p,
    v = Q g, acceptance as in rsrr()."""
    from workloads import Fn
    R = distances(prob)
    z = sample_points(prob.region, prob.N)
    X = resolvent_samples_dense(prob, z, U)
    S = normalize_columns(sample_matrix(X))
    Q, sig, k = truncated_basis(S, delta)
    A = taylor_coefficients(prob, R)
    P = [Q.conj().T @ (Ap @ Q) for Ap in A]
    c = prob.region.center
    fns = [ShiftPow(p, c) for p in range(len(A))]
    lam, G, info = ss_full(P, fns, prob.region, NQ, KQ, tol_gap)
    V = Q @ G
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    keep = inside(prob.region, lam)
    lam, V = lam[keep], V[:, keep]
    res = np.array([residual_dense(prob, l, V[:, j], R) for j, l in enumerate(lam)])
    ok = res <= res_tol
    lam, V, res = lam[ok], V[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    return dict(lam=lam[order], V=V[:, order], res=res[order], k=k, sigma=sig, info=info,
                z=z, X=X, P=P, Q=Q, terms=len(A))


class ShiftPow:
    """f(z) = (z - c)^p, the scalar functions of the Taylor-expanded T."""
    def __init__(self, p: int, c: complex):
        self.p, self.c = p, c


_eval_fn_base = eval_fn


def eval_fn(fn, z):  # noqa: F811  (extends the families with the Taylor powers)
    if isinstance(fn, ShiftPow):
        return (np.asarray(z, dtype=np.complex128) - fn.c) ** fn.p
    return _eval_fn_base(fn, z)


def argument_principle_count_dense(prob, npts: int = 2048) -> int:
    """Zeros of det T inside the region by the winding number of det T(z):
    the phase of det T along the contour, sampled at npts points and refined
    segment by segment (midpoints inserted only where a step of the phase is
    at least pi/4) until every step is below pi/4; the winding number is the
    sum of the steps over 2 pi."""
    R = distances(prob)
    reg = prob.region

    def phase(al):
        z = reg.center + reg.a * np.cos(al) + 1j * reg.b * np.sin(al)
        s, _ = np.linalg.slogdet(assemble_dense(prob, z, R))
        return np.angle(s)

    alpha = list(np.linspace(0.0, 2.0 * np.pi, npts + 1))
    ph = [phase(a) for a in alpha]
    total = 0.0
    stack = [(alpha[i], alpha[i + 1], ph[i], ph[i + 1], 0) for i in range(npts)]
    while stack:
        a, b, pa, pb, depth = stack.pop()
        d = float(np.angle(np.exp(1j * (pb - pa))))
        if abs(d) < np.pi / 4 or depth >= 20:
            total += d
            continue
        m = 0.5 * (a + b)
        pm = phase(m)
        stack.append((m, b, pm, pb, depth + 1))
        stack.append((a, m, pa, pm, depth + 1))
    return int(round(total / (2.0 * np.pi)))


# ---------------------------------------------------------------------------
# General dense terms T(z) = sum_i f_i(z) A_i (Eq. 1 with dense A_i; the
# "black-box" BEM matrices of Section 2.1 with a separated z-dependence)
# ---------------------------------------------------------------------------

def assemble_terms(prob, z: complex) -> np.ndarray:
    """T(z) = sum_i f_i(z) A_i, dense."""
    T = np.zeros((prob.n, prob.n), dtype=np.complex128)
    for fn, A in zip(prob.fns, prob.As):
        T += complex(eval_fn(fn, z)) * A
    return T


def resolvent_samples_terms(prob, z: np.ndarray, U: np.ndarray | None = None) -> list:
    """X_j = T(z_j)^{-1} U by dense LU with partial pivoting (LAPACK gesv)."""
    if U is None:
        U = prob.U
    return [np.linalg.solve(assemble_terms(prob, zj), U) for zj in z]


def backward_error_inf_terms(prob, z: complex, X: np.ndarray, U: np.ndarray | None = None):
    """Per-column eta = ||U - T X||_inf / (||T||_inf ||X||_inf + ||U||_inf)."""
    if U is None:
        U = prob.U
    T = assemble_terms(prob, z)
    Rr = U - T @ X
    tn = np.abs(T).sum(axis=1).max()
    return np.abs(Rr).max(axis=0) / (tn * np.abs(X).max(axis=0) + np.abs(U).max(axis=0))


def residual_terms(prob, lam: complex, v: np.ndarray) -> float:
    """||T(lam) v||_2 / ((sum_i |f_i(lam)| ||A_i||_1) ||v||_2), the normalised
    residual of Section 5.4 with the 1-norms of the dense A_i."""
    scale = sum(abs(complex(eval_fn(fn, lam))) * np.abs(A).sum(axis=0).max()
                for fn, A in zip(prob.fns, prob.As))
    return float(np.linalg.norm(assemble_terms(prob, lam) @ v) / (scale * np.linalg.norm(v)))


def rsrr_terms(prob, delta: float = 1e-14, NQ: int = 500, KQ: int = 2, tol_gap: float = 1e3,
               U: np.ndarray | None = None, res_tol: float = 1e-6):
    """RSRR (Section 4.3) for dense terms: samples by dense solves, truncated
    SVD basis of the normalised S, P_i = Q^H A_i Q, SS-FULL on T_Q, v = Q g,
    acceptance as in rsrr()."""
    z = sample_points(prob.region, prob.N)
    X = resolvent_samples_terms(prob, z, U)
    S = normalize_columns(sample_matrix(X))
    Q, sig, k = truncated_basis(S, delta)
    P = [Q.conj().T @ (A @ Q) for A in prob.As]
    lam, G, info = ss_full(P, prob.fns, prob.region, NQ, KQ, tol_gap)
    V = Q @ G
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    keep = inside(prob.region, lam)
    lam, V = lam[keep], V[:, keep]
    res = np.array([residual_terms(prob, l, V[:, j]) for j, l in enumerate(lam)])
    ok = res <= res_tol
    lam, V, res = lam[ok], V[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    return dict(lam=lam[order], V=V[:, order], res=res[order], k=k, sigma=sig, info=info,
                z=z, X=X, P=P, Q=Q)


# ---------------------------------------------------------------------------
# The comparison methods of Sections 3 and 4.1: SS-RI (moments of
# F(z) = U^H T(z)^{-1} U, Hankel pencil) and SSRR-M (Rayleigh-Ritz on the
# moment matrix M instead of S).  Both use the sampled X_j = T(z_j)^{-1} U.
# ---------------------------------------------------------------------------

def interpolation_weights(region: Region, z: np.ndarray) -> np.ndarray:
    """Weights omega_i of the moments (up to a common factor, which changes
    neither the pencil's eigenvalues nor span(M), Section 3.3 item 3):
    trapezoid nodes on the ellipse -> the quadrature weights (1/N) phi'(alpha_i)
    of Eq. 58 (the contour-integral special case); Chebyshev points of an
    interval -> (-1)^i sin((2i + 1) pi / 2N) (Eq. 43); explicit points -> the
    barycentric weights 1 / prod_{j != i} (z_i - z_j) of Eq. 19, every factor
    scaled by the reciprocal capacity (here 2 / rho of the region's scale rho)
    and formed through logarithms against under- and overflow."""
    N = len(z)
    if region.kind == "ellipse":
        return quad_weights(region, N)
    if region.kind == "rect" and region.points is None:  # Gauss-Legendre nodes: dz / (2 pi)
        return rect_rule(region, rect_counts(region, N))[1]
    if region.kind == "interval":
        i = np.arange(N)
        return (-1.0) ** i * np.sin((2 * i + 1) * np.pi / (2 * N)) + 0j
    rho = max(region.a, region.b)
    s = (np.asarray(z) - region.center) * (2.0 / rho)
    logw = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        d = s[i] - np.delete(s, i)
        logw[i] = -np.sum(np.log(d))
    logw -= logw.real.max()
    return np.exp(logw)


def moment_matrix(X: list, z: np.ndarray, w: np.ndarray, region: Region, K: int) -> np.ndarray:
    """M = [M_0 ... M_{K-1}], M_alpha = sum_i omega_i s_i^alpha X_i (Eq. 40 and
    Eq. 48) with the scaled powers s_i = (z_i - gamma)/rho (a fixed change of
    basis of the polynomials of degree < K: span(M) is unchanged)."""
    rho = max(region.a, region.b)
    s = (np.asarray(z) - region.center) / rho
    return np.concatenate([sum(w[i] * s[i] ** al * X[i] for i in range(len(X))) for al in range(K)],
                          axis=1)


def ss_ri(prob: Problem, K: int, U: np.ndarray | None = None, tol_gap: float = 1e3,
          res_tol: float = 1e-6):
    """SS-RI (Section 3.3, steps 1-6): F(z_i) = U^H X_i (Eq. 14), moments
    A_alpha = sum_i omega_i s_i^alpha F(z_i) (Eq. 18, scaled powers), Hankel H
    and H^< (Eq. 33), truncated SVD of H with the count from the largest gap
    (Eq. 37, Eq. 44), A = V0^H H^< W0 Sigma0^{-1} (Eq. 38), its eigenpairs,
    lambda = gamma + rho lambda' and v = M W0 Sigma0^{-1} b (Eq. 41) with
    M = [M_0 ... M_{K-1}] (Eq. 39-40); acceptance as in rsrr()."""
    if U is None:
        U = prob.U
    region = prob.region
    z = sample_points(region, prob.N)
    X = resolvent_samples(prob, z, U)
    w = interpolation_weights(region, z)
    rho = max(region.a, region.b)
    s = (z - region.center) / rho
    F = [U.conj().T @ Xi for Xi in X]
    A = [sum(w[i] * s[i] ** al * F[i] for i in range(len(F))) for al in range(2 * K)]
    H = np.block([[A[i + j] for j in range(K)] for i in range(K)])
    Hs = np.block([[A[i + j + 1] for j in range(K)] for i in range(K)])
    V, sv, Wh = np.linalg.svd(H)
    ratios = sv[:-1] / np.maximum(sv[1:], np.finfo(float).tiny)
    nbar = int(np.argmax(ratios)) + 1
    V0, W0 = V[:, :nbar], Wh.conj().T[:, :nbar]
    S0inv = np.diag(1.0 / sv[:nbar])
    Am = V0.conj().T @ Hs @ W0 @ S0inv
    lam_s, B = np.linalg.eig(Am)
    lam = region.center + rho * lam_s
    M = moment_matrix(X, z, w, region, K)
    Vv = M @ (W0 @ S0inv @ B)
    Vv = Vv / np.linalg.norm(Vv, axis=0, keepdims=True)
    keep = inside(region, lam)
    lam, Vv = lam[keep], Vv[:, keep]
    res = np.array([residual(prob, l, Vv[:, c]) for c, l in enumerate(lam)])
    ok = res <= res_tol
    lam, Vv, res = lam[ok], Vv[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    return dict(lam=lam[order], V=Vv[:, order], res=res[order], nbar=nbar, sv=sv)


def ssrr_m(prob: Problem, K: int, delta: float = 1e-14, NQ: int = 500, KQ: int = 2,
           tol_gap: float = 1e3, U: np.ndarray | None = None, res_tol: float = 1e-6):
    """SSRR-M (Section 4.1 and the last paragraphs of Section 4.3): RSRR with
    the moment matrix M (Eq. 48) in place of the sampling matrix S: truncated
    SVD basis of M (normalised columns), projection, SS-FULL, v = Q g."""
    z = sample_points(prob.region, prob.N)
    X = resolvent_samples(prob, z, U)
    w = interpolation_weights(prob.region, z)
    M = normalize_columns(moment_matrix(X, z, w, prob.region, K))
    Q, sig, k = truncated_basis(M, delta)
    P = project(prob, Q)
    lam, G, info = ss_full(P, prob.fns, prob.region, NQ, KQ, tol_gap)
    V = Q @ G
    V = V / np.linalg.norm(V, axis=0, keepdims=True)
    keep = inside(prob.region, lam)
    lam, V = lam[keep], V[:, keep]
    res = np.array([residual(prob, l, V[:, c]) for c, l in enumerate(lam)])
    ok = res <= res_tol
    lam, V, res = lam[ok], V[:, ok], res[ok]
    order = np.lexsort((np.angle(lam), np.abs(lam)))
    return dict(lam=lam[order], V=V[:, order], res=res[order], k=k, sigma=sig, info=info)
