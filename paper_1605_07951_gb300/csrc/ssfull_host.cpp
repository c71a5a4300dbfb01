// SS-FULL on the projected NEP T_Q(z) = sum_i f_i(z) P_i (k x k), in FP64 on
// the host: the SS-RI algorithm of Section 2.3 with U = I (F = T_Q^{-1}),
// quadrature nodes and weights of the trapezoid rule on the ellipse
// (Section 4.1), moments scaled by ((z - gamma)/rho)^alpha, block Hankel
// matrices H and H^<, truncated SVD of H with the count given by the largest
// singular-value gap (tol_gap test), A = V0^H H^< W0 Sigma0^{-1}, and the
// eigenpairs of A lifted by g = M W0 Sigma0^{-1} b with M = [A_0 .. A_{K-1}].
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <functional>
#include <thread>
#include <vector>

#include "ssfull_host.h"

namespace rsrr {

using cplx = std::complex<double>;

namespace {

struct Mat {
    int r = 0, c = 0;
    std::vector<cplx> a;  // column major
    Mat() = default;
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_) {}
    cplx &operator()(int i, int j) { return a[(size_t)j * r + i]; }
    const cplx &operator()(int i, int j) const { return a[(size_t)j * r + i]; }
};

void parallel_for(int count, int threads, const std::function<void(int, int)> &fn) {
    // fn(index, worker); worker w takes indices w, w + threads, ... so that
    // per-worker partial sums (and their rounding) do not depend on timing
    threads = std::max(1, std::min(threads, count));
    if (threads == 1) {
        for (int i = 0; i < count; ++i) fn(i, 0);
        return;
    }
    std::vector<std::thread> pool;
    for (int w = 0; w < threads; ++w)
        pool.emplace_back([&, w]() {
            for (int i = w; i < count; i += threads) fn(i, w);
        });
    for (auto &t : pool) t.join();
}

// In-place LU with partial pivoting (max modulus, first index on ties) and
// F = T^{-1} by solving T F = I.  Returns false for an exactly zero pivot.
bool invert(Mat &T, Mat &F, std::vector<int> &piv) {
    const int k = T.r;
    piv.resize(k);
    for (int j = 0; j < k; ++j) {
        int p = j;
        double best = std::abs(T(j, j));
        for (int i = j + 1; i < k; ++i) {
            const double v = std::abs(T(i, j));
            if (v > best) { best = v; p = i; }
        }
        piv[j] = p;
        if (best == 0.0) return false;
        if (p != j)
            for (int c = 0; c < k; ++c) std::swap(T(j, c), T(p, c));
        const cplx inv = 1.0 / T(j, j);
        for (int i = j + 1; i < k; ++i) T(i, j) *= inv;
        for (int c = j + 1; c < k; ++c) {
            const cplx u = T(j, c);
            if (u == cplx(0.0)) continue;
            cplx *col = &T(0, c);
            const cplx *l = &T(0, j);
            for (int i = j + 1; i < k; ++i) col[i] -= l[i] * u;
        }
    }
    F = Mat(k, k);
    for (int j = 0; j < k; ++j) F(j, j) = 1.0;
    for (int j = 0; j < k; ++j)
        if (piv[j] != j)
            for (int c = 0; c < k; ++c) std::swap(F(j, c), F(piv[j], c));
    for (int c = 0; c < k; ++c) {
        cplx *x = &F(0, c);
        for (int j = 0; j < k; ++j) {  // L y = b
            const cplx y = x[j];
            if (y == cplx(0.0)) continue;
            const cplx *l = &T(0, j);
            for (int i = j + 1; i < k; ++i) x[i] -= l[i] * y;
        }
        for (int j = k - 1; j >= 0; --j) {  // U x = y
            x[j] /= T(j, j);
            const cplx y = x[j];
            const cplx *u = &T(0, j);
            for (int i = 0; i < j; ++i) x[i] -= u[i] * y;
        }
    }
    return true;
}

// One-sided Jacobi SVD (Hestenes): A (r x c, r >= c not required) = U S W^H.
// Columns are orthogonalised pairwise in a round-robin order (pairs of one
// round are independent and run in parallel).  Singular values descending.
void svd_jacobi(const Mat &A0, Mat &U, std::vector<double> &S, Mat &W, int threads) {
    Mat A = A0;
    const int r = A.r, c = A.c;
    W = Mat(c, c);
    for (int j = 0; j < c; ++j) W(j, j) = 1.0;
    const int cp = c + (c & 1);
    for (int sweep = 0; sweep < 60; ++sweep) {
        std::atomic<int> rotated(0);
        for (int round = 0; round < cp - 1; ++round) {
            parallel_for(cp / 2, threads, [&](int a, int) {
                int p, q;
                if (a == 0) { p = cp - 1; q = round; }
                else { p = (round + a) % (cp - 1); q = (round - a + (cp - 1)) % (cp - 1); }
                if (p > q) std::swap(p, q);
                if (q >= c) return;
                double al = 0.0, be = 0.0;
                cplx ga = 0.0;
                const cplx *x = &A(0, p), *y = &A(0, q);
                for (int i = 0; i < r; ++i) {
                    al += std::norm(x[i]);
                    be += std::norm(y[i]);
                    ga += std::conj(x[i]) * y[i];
                }
                const double ag = std::abs(ga);
                if (ag <= 1e-15 * std::sqrt(al * be) || ag == 0.0) return;
                rotated++;
                const double tau = (be - al) / (2.0 * ag);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                const cplx e = ga / ag;  // e^{i phi}
                const cplx se = sn * e, sec = sn * std::conj(e);
                cplx *xm = &A(0, p), *ym = &A(0, q);
                for (int i = 0; i < r; ++i) {
                    const cplx xi = xm[i], yi = ym[i];
                    xm[i] = cs * xi - sec * yi;
                    ym[i] = se * xi + cs * yi;
                }
                cplx *wp = &W(0, p), *wq = &W(0, q);
                for (int i = 0; i < c; ++i) {
                    const cplx xi = wp[i], yi = wq[i];
                    wp[i] = cs * xi - sec * yi;
                    wq[i] = se * xi + cs * yi;
                }
            });
        }
        if (rotated.load() == 0) break;
    }
    std::vector<double> nrm(c);
    for (int j = 0; j < c; ++j) {
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += std::norm(A(i, j));
        nrm[j] = std::sqrt(s);
    }
    std::vector<int> ord(c);
    for (int j = 0; j < c; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
    U = Mat(r, c);
    Mat Ws(c, c);
    S.resize(c);
    for (int jj = 0; jj < c; ++jj) {
        const int j = ord[jj];
        S[jj] = nrm[j];
        for (int i = 0; i < r; ++i) U(i, jj) = nrm[j] > 0 ? A(i, j) / nrm[j] : cplx(0.0);
        for (int i = 0; i < c; ++i) Ws(i, jj) = W(i, j);
    }
    W = Ws;
}

// Eigenvalues and eigenvectors of a general complex matrix: Householder
// reduction to Hessenberg form, shifted QR iteration (Wilkinson shifts,
// Givens rotations) to the Schur form T = Z^H A Z, eigenvectors of T by back
// substitution, mapped back by Z.
void eig_general(const Mat &A0, std::vector<cplx> &lam, Mat &V) {
    const int n = A0.r;
    Mat H = A0, Z(n, n);
    for (int i = 0; i < n; ++i) Z(i, i) = 1.0;
    // Hessenberg reduction
    for (int k = 0; k + 2 < n + 0 && k < n - 2; ++k) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; ++i) alpha += std::norm(H(i, k));
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        std::vector<cplx> v(n, 0.0);
        const cplx x0 = H(k + 1, k);
        const cplx ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cplx(1.0);
        v[k + 1] = x0 + ph * alpha;
        for (int i = k + 2; i < n; ++i) v[i] = H(i, k);
        double vn = 0.0;
        for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        // H <- (I - 2 v v^H / vn) H (I - 2 v v^H / vn)
        for (int j = 0; j < n; ++j) {
            cplx s = 0.0;
            for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * H(i, j);
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; ++i) H(i, j) -= v[i] * s;
        }
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int j = k + 1; j < n; ++j) s += H(i, j) * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; ++j) H(i, j) -= s * std::conj(v[j]);
        }
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int j = k + 1; j < n; ++j) s += Z(i, j) * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; ++j) Z(i, j) -= s * std::conj(v[j]);
        }
        for (int i = k + 2; i < n; ++i) H(i, k) = 0.0;
    }
    // shifted QR
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0;
    while (hi > 0 && iter < 100 * n) {
        int lo = hi;
        while (lo > 0) {
            const double s = std::abs(H(lo, lo)) + std::abs(H(lo - 1, lo - 1));
            if (std::abs(H(lo, lo - 1)) <= eps * (s > 0 ? s : 1.0)) {
                H(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) { --hi; iter = 0; continue; }
        ++iter;
        // Wilkinson shift from the trailing 2x2
        const cplx a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
        const cplx tr = a + d, det = a * d - b * c;
        const cplx disc = std::sqrt(tr * tr - 4.0 * det);
        const cplx l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
        cplx mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 10) mu = d + cplx(std::abs(H(hi, hi - 1)), 0.0);  // exceptional shift
        // QR step on the active window via Givens rotations
        std::vector<double> gc(hi - lo);
        std::vector<cplx> gs(hi - lo);
        for (int i = lo; i <= hi; ++i) H(i, i) -= mu;
        for (int k = lo; k < hi; ++k) {
            const cplx x = H(k, k), y = H(k + 1, k);
            const double r = std::hypot(std::abs(x), std::abs(y));
            double cs;
            cplx sn;
            if (r == 0.0) { cs = 1.0; sn = 0.0; }
            else if (std::abs(x) == 0.0) { cs = 0.0; sn = std::conj(y) / std::abs(y); }
            else {
                cs = std::abs(x) / r;
                sn = (x / std::abs(x)) * std::conj(y) / r;
            }
            gc[k - lo] = cs;
            gs[k - lo] = sn;
            // rows k, k+1 : [c, s; -conj(s), c]
            for (int j = k; j < n; ++j) {
                const cplx t1 = H(k, j), t2 = H(k + 1, j);
                H(k, j) = cs * t1 + sn * t2;
                H(k + 1, j) = -std::conj(sn) * t1 + cs * t2;
            }
        }
        for (int k = lo; k < hi; ++k) {
            const double cs = gc[k - lo];
            const cplx sn = gs[k - lo];
            // columns k, k+1 : multiply by G^H = [c, -s; conj(s), c]
            for (int i = 0; i <= std::min(hi, k + 2 > hi ? hi : k + 2); ++i) {
                const cplx t1 = H(i, k), t2 = H(i, k + 1);
                H(i, k) = cs * t1 + std::conj(sn) * t2;
                H(i, k + 1) = -sn * t1 + cs * t2;
            }
            for (int i = 0; i < lo; ++i) {}  // rows above lo already covered by i from 0
            for (int i = 0; i < n; ++i) {
                const cplx t1 = Z(i, k), t2 = Z(i, k + 1);
                Z(i, k) = cs * t1 + std::conj(sn) * t2;
                Z(i, k + 1) = -sn * t1 + cs * t2;
            }
        }
        for (int i = lo; i <= hi; ++i) H(i, i) += mu;
    }
    lam.resize(n);
    for (int i = 0; i < n; ++i) lam[i] = H(i, i);
    // eigenvectors of the triangular T = H
    Mat X(n, n);
    double tnorm = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) tnorm = std::max(tnorm, std::abs(H(i, j)));
    const double small = std::max(tnorm * eps, 1e-300);
    for (int k = 0; k < n; ++k) {
        X(k, k) = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            cplx s = 0.0;
            for (int j = i + 1; j <= k; ++j) s += H(i, j) * X(j, k);
            cplx den = H(i, i) - lam[k];
            if (std::abs(den) < small) den = small;
            X(i, k) = -s / den;
        }
    }
    V = Mat(n, n);
    for (int k = 0; k < n; ++k) {
        double nv = 0.0;
        for (int i = 0; i < n; ++i) {
            cplx s = 0.0;
            for (int j = 0; j <= k; ++j) s += Z(i, j) * X(j, k);
            V(i, k) = s;
            nv += std::norm(s);
        }
        nv = std::sqrt(nv);
        for (int i = 0; i < n; ++i) V(i, k) /= nv;
    }
}

}  // namespace

int ss_full_host(const std::vector<std::vector<cplx>> &P, int k,
                 const std::function<cplx(int, cplx)> &f, int m, cplx gamma, double a, double b,
                 int NQ, int KQ, int threads, std::vector<cplx> &lam, std::vector<cplx> &G,
                 int &nbar, double &gmax) {
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    const double rho = std::max(a, b);
    const int nmom = 2 * KQ;
    std::vector<std::vector<Mat>> part(threads, std::vector<Mat>(nmom, Mat(k, k)));
    std::atomic<int> singular(0);
    parallel_for(NQ, threads, [&](int q, int w) {
        const double al = 2.0 * M_PI * (q + 0.5) / NQ;
        const cplx z = gamma + cplx(a * std::cos(al), b * std::sin(al));
        const cplx wq = cplx(-a * std::sin(al), b * std::cos(al)) / (double)NQ;
        Mat T(k, k);
        for (int i = 0; i < m; ++i) {
            const cplx fi = f(i, z);
            const std::vector<cplx> &Pi = P[i];
            for (size_t e = 0; e < T.a.size(); ++e) T.a[e] += fi * Pi[e];
        }
        Mat F;
        std::vector<int> piv;
        if (!invert(T, F, piv)) { singular++; return; }
        const cplx s = (z - gamma) / rho;
        cplx c = wq;
        for (int al2 = 0; al2 < nmom; ++al2) {
            std::vector<cplx> &acc = part[w][al2].a;
            for (size_t e = 0; e < acc.size(); ++e) acc[e] += c * F.a[e];
            c *= s;
        }
    });
    if (singular.load() > 0) return -1;
    std::vector<Mat> Am(nmom, Mat(k, k));
    for (int al2 = 0; al2 < nmom; ++al2)
        for (int w = 0; w < threads; ++w)
            for (size_t e = 0; e < Am[al2].a.size(); ++e) Am[al2].a[e] += part[w][al2].a[e];
    const int dim = KQ * k;
    Mat H(dim, dim), Hs(dim, dim);
    for (int bi = 0; bi < KQ; ++bi)
        for (int bj = 0; bj < KQ; ++bj)
            for (int j = 0; j < k; ++j)
                for (int i = 0; i < k; ++i) {
                    H(bi * k + i, bj * k + j) = Am[bi + bj](i, j);
                    Hs(bi * k + i, bj * k + j) = Am[bi + bj + 1](i, j);
                }
    Mat Us, Ws;
    std::vector<double> sv;
    svd_jacobi(H, Us, sv, Ws, threads);
    nbar = 1;
    gmax = 0.0;
    for (int j = 0; j + 1 < dim; ++j) {
        const double r = sv[j] / std::max(sv[j + 1], 1e-300);
        if (r > gmax) { gmax = r; nbar = j + 1; }
    }
    if (dim == 1) { nbar = 1; gmax = 0.0; }
    // A = V0^H H^< W0 Sigma0^{-1}
    Mat HW(dim, nbar);
    for (int j = 0; j < nbar; ++j)
        for (int l = 0; l < dim; ++l) {
            const cplx w = Ws(l, j) / sv[j];
            if (w == cplx(0.0)) continue;
            for (int i = 0; i < dim; ++i) HW(i, j) += Hs(i, l) * w;
        }
    Mat A(nbar, nbar);
    for (int j = 0; j < nbar; ++j)
        for (int i = 0; i < nbar; ++i) {
            cplx s = 0.0;
            for (int l = 0; l < dim; ++l) s += std::conj(Us(l, i)) * HW(l, j);
            A(i, j) = s;
        }
    std::vector<cplx> ls;
    Mat B;
    eig_general(A, ls, B);
    lam.resize(nbar);
    for (int j = 0; j < nbar; ++j) lam[j] = gamma + rho * ls[j];
    // g = M W0 Sigma0^{-1} b, M = [A_0 ... A_{KQ-1}] (k x dim)
    Mat WB(dim, nbar);
    for (int j = 0; j < nbar; ++j)
        for (int l = 0; l < nbar; ++l) {
            const cplx bl = B(l, j) / sv[l];
            for (int i = 0; i < dim; ++i) WB(i, j) += Ws(i, l) * bl;
        }
    G.assign((size_t)k * nbar, 0.0);
    for (int j = 0; j < nbar; ++j)
        for (int bi = 0; bi < KQ; ++bi)
            for (int l = 0; l < k; ++l) {
                const cplx w = WB(bi * k + l, j);
                if (w == cplx(0.0)) continue;
                const Mat &Mb = Am[bi];
                for (int i = 0; i < k; ++i) G[(size_t)j * k + i] += Mb(i, l) * w;
            }
    return 0;
}

}  // namespace rsrr
