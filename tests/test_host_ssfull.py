"""CPU tests of the library's host SS-FULL finish (csrc/ssfull_host.cpp: block
Hankel matrices of the moments, truncated SVD by column-pivoted QR + Jacobi,
singular-value gap, the small eigenproblem and the lifted eigenvectors;
Section 3.3 with U = I).  The source is compiled here with g++ behind a
one-function C harness and fed moments with a closed form: for
T(z) = V diag(z - mu_i) V^{-1}, the contour moments of T^{-1} are
c * V diag(s_i^alpha [mu_i inside]) V^{-1}, s_i = (mu_i - gamma) / rho, for any
common factor c.  The eigenvalues must be the mu_i inside the ellipse and the
eigenvectors the matching columns of V."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1605_07951_gb300", "csrc")

HARNESS = r"""
#include <complex>
#include <vector>
#include "ssfull_host.h"
extern "C" int ssf_finish(const double *mom, int k, int KQ, double gr, double gi, double rho,
                          int cap, double *lam, double *G, int *nbar, double *gmax) {
    using cplx = std::complex<double>;
    std::vector<std::vector<cplx>> A(2 * KQ, std::vector<cplx>((size_t)k * k));
    for (int a = 0; a < 2 * KQ; ++a)
        for (size_t e = 0; e < (size_t)k * k; ++e)
            A[a][e] = cplx(mom[2 * ((size_t)a * k * k + e)], mom[2 * ((size_t)a * k * k + e) + 1]);
    std::vector<cplx> l, g;
    int nb = 0;
    double gm = 0.0;
    const int st = rsrr::ss_full_finish(A, k, KQ, cplx(gr, gi), rho, 2, l, g, nb, gm);
    if (st != 0) return st;
    *nbar = nb;
    *gmax = gm;
    if (nb > cap) return -2;
    for (int j = 0; j < nb; ++j) { lam[2 * j] = l[j].real(); lam[2 * j + 1] = l[j].imag(); }
    for (size_t e = 0; e < (size_t)k * nb; ++e) { G[2 * e] = g[e].real(); G[2 * e + 1] = g[e].imag(); }
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("ssfull")
    h = d / "harness.cpp"
    h.write_text(HARNESS)
    so = d / "libssf.so"
    # the same floating-point rules the library build uses for this file
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-fcx-fortran-rules", "-I", SRC,
                    str(h), os.path.join(SRC, "ssfull_host.cpp"), "-o", str(so), "-pthread"],
                   check=True, capture_output=True, text=True)
    L = C.CDLL(str(so))
    L.ssf_finish.restype = C.c_int
    L.ssf_finish.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                             C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int),
                             C.POINTER(C.c_double)]
    return L


def closed_form_moments(V, mu, gamma, rho, a, b, KQ, c=1j):
    inside = ((mu.real - gamma.real) / a) ** 2 + ((mu.imag - gamma.imag) / b) ** 2 < 1.0
    s = (mu - gamma) / rho
    Vi = np.linalg.inv(V)
    mom = np.stack([c * (V * np.where(inside, s ** al, 0.0)) @ Vi for al in range(2 * KQ)])
    return mom, inside


def finish(lib, mom, KQ, gamma, rho):
    k = mom.shape[1]
    buf = np.ascontiguousarray(np.stack([m.T for m in mom]))  # column major per moment
    cap = KQ * k
    lam = np.zeros(cap, dtype=np.complex128)
    G = np.zeros((cap, k), dtype=np.complex128)
    nbar, gmax = C.c_int(0), C.c_double(0.0)
    st = lib.ssf_finish(buf.ctypes.data, k, KQ, gamma.real, gamma.imag, rho, cap, lam.ctypes.data,
                        G.ctypes.data, C.byref(nbar), C.byref(gmax))
    assert st == 0
    n = nbar.value
    return lam[:n], G[:n].T, gmax.value


@pytest.mark.parametrize("k,KQ,seed", [(6, 2, 0), (10, 2, 1), (12, 3, 2), (5, 1, 3)])
def test_eigenvalues_and_vectors_from_closed_form_moments(lib, k, KQ, seed):
    rng = np.random.default_rng(seed)
    gamma, a, b = complex(1.0, 0.5), 2.0, 1.0
    rho = max(a, b)
    # about half of the mu inside the ellipse, the rest well outside
    t = rng.uniform(0, 2 * np.pi, k)
    rad = np.where(np.arange(k) % 2 == 0, rng.uniform(0.1, 0.8, k), rng.uniform(1.5, 3.0, k))
    mu = gamma + rad * (a * np.cos(t) + 1j * b * np.sin(t))
    V = rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k)) + 3 * np.eye(k)
    mom, inside = closed_form_moments(V, mu, gamma, rho, a, b, KQ)
    lam, G, gmax = finish(lib, mom, KQ, gamma, rho)
    want = mu[inside]
    assert len(lam) == len(want) == inside.sum()
    assert gmax > 1e10  # exact moments: the gap is at the rounding level
    for j, l in enumerate(lam):
        i = int(np.argmin(np.abs(want - l)))
        assert abs(want[i] - l) <= 1e-12 * max(1.0, abs(want[i]))
        # lifted eigenvector parallel to the matching column of V
        v = V[:, np.flatnonzero(inside)[i]]
        g = G[:, j]
        cosang = abs(np.vdot(v, g)) / (np.linalg.norm(v) * np.linalg.norm(g))
        assert cosang >= 1 - 1e-12


def test_common_factor_of_the_moments_does_not_matter(lib):
    rng = np.random.default_rng(7)
    k, KQ = 8, 2
    gamma, a, b = complex(0.0, 0.0), 1.0, 1.0
    mu = np.concatenate([0.5 * np.exp(2j * np.pi * rng.random(3)), 2.5 * np.exp(2j * np.pi * rng.random(5))])
    V = np.eye(k) + 0.3 * (rng.normal(size=(k, k)) + 1j * rng.normal(size=(k, k)))
    out = []
    for c in (1.0, 1j, -3.5 + 2j):
        mom, inside = closed_form_moments(V, mu, gamma, 1.0, a, b, KQ, c)
        lam, _, _ = finish(lib, mom, KQ, gamma, 1.0)
        out.append(np.sort_complex(lam))
    assert len(out[0]) == 3
    assert np.abs(out[0] - out[1]).max() <= 1e-13 and np.abs(out[0] - out[2]).max() <= 1e-13
