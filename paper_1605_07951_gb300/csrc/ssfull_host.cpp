// SS-FULL on the projected NEP T_Q(z) = sum_i f_i(z) P_i (k x k), in FP64 on
// the host, from the moments A_alpha = sum_q w_q ((z_q - gamma)/rho)^alpha
// T_Q(z_q)^{-1} (computed on the GPU, ssfull_dev.cu): the SS-RI algorithm of
// Section 3.3 with U = I, block Hankel matrices H and H^<, truncated SVD of H
// with the count given by the largest singular-value gap (tol_gap test),
// A = V0^H H^< W0 Sigma0^{-1}, and the eigenpairs of A lifted by
// g = M W0 Sigma0^{-1} b with M = [A_0 .. A_{K-1}].
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

// Truncated SVD A = U S W^H of A (r x c) through a column-pivoted Householder
// QR: A P = Q R, stopped once every remaining column norm is <= rel_tol times
// the largest column norm of A (those directions lie at the rounding level of
// the moments); then one-sided Jacobi on the t columns of R^H (the rows of a
// pivoted R are graded and nearly orthogonal, so few sweeps are needed):
// R^H J = X S, hence A = (Q J) S (P X)^H.  U is r x t, W is c x t, S has t
// values (descending); `tail` is the largest remaining column norm, an upper
// bound of the next singular value up to a factor sqrt(c).
void svd_qr_jacobi(const Mat &A0, Mat &U, std::vector<double> &S, double &tail, Mat &W,
                   int threads, double rel_tol) {
    Mat A = A0;
    const int r = A.r, c = A.c;
    std::vector<int> perm(c);
    std::vector<double> nrm2(c);
    for (int j = 0; j < c; ++j) {
        perm[j] = j;
        double s = 0.0;
        for (int i = 0; i < r; ++i) s += std::norm(A(i, j));
        nrm2[j] = s;
    }
    std::vector<std::vector<cplx>> refl;  // Householder vectors v (rows s..r-1), |v| = sqrt(2)
    std::vector<cplx> diag;
    double first = -1.0;
    tail = 0.0;
    int t = 0;
    for (int s = 0; s < std::min(r, c); ++s) {
        int p = s;
        for (int j = s + 1; j < c; ++j)
            if (nrm2[j] > nrm2[p]) p = j;
        const double np = std::sqrt(std::max(nrm2[p], 0.0));
        if (first < 0.0) first = np;
        if (np <= rel_tol * first || np == 0.0) { tail = np; break; }
        if (p != s) {
            for (int i = 0; i < r; ++i) std::swap(A(i, s), A(i, p));
            std::swap(nrm2[s], nrm2[p]);
            std::swap(perm[s], perm[p]);
        }
        // reflector mapping A(s:, s) to alpha e_1, alpha = -e^{i arg x0} |x|
        double xn = 0.0;
        for (int i = s; i < r; ++i) xn += std::norm(A(i, s));
        xn = std::sqrt(xn);
        const cplx x0 = A(s, s);
        const cplx ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplx(1.0);
        const cplx alpha = -ph * xn;
        std::vector<cplx> v(r - s);
        v[0] = x0 - alpha;
        for (int i = s + 1; i < r; ++i) v[i - s] = A(i, s);
        double vn = 0.0;
        for (const cplx &e : v) vn += std::norm(e);
        vn = std::sqrt(vn);
        if (vn > 0.0)
            for (cplx &e : v) e *= std::sqrt(2.0) / vn;  // H = I - v v^H
        // trailing columns: A(s:, j) -= v (v^H A(s:, j)), column norms recomputed
        parallel_for(c - s - 1, threads, [&](int jj, int) {
            const int j = s + 1 + jj;
            cplx w = 0.0;
            for (int i = s; i < r; ++i) w += std::conj(v[i - s]) * A(i, j);
            double nn = 0.0;
            for (int i = s; i < r; ++i) {
                A(i, j) -= v[i - s] * w;
                if (i > s) nn += std::norm(A(i, j));
            }
            nrm2[j] = nn;
        });
        refl.push_back(std::move(v));
        diag.push_back(alpha);
        t = s + 1;
    }
    if (t == 0) {
        U = Mat(r, 0);
        W = Mat(c, 0);
        S.clear();
        return;
    }
    // B = R^H (c x t): B(j, i) = conj(R(i, j)), R upper trapezoidal
    Mat B(c, t);
    for (int i = 0; i < t; ++i) {
        B(i, i) = std::conj(diag[i]);
        for (int j = i + 1; j < c; ++j) B(j, i) = std::conj(A(i, j));
    }
    Mat J(t, t);
    for (int j = 0; j < t; ++j) J(j, j) = 1.0;
    const int tp = t + (t & 1);
    for (int sweep = 0; sweep < 60; ++sweep) {
        std::atomic<int> rotated(0);
        for (int round = 0; round < tp - 1; ++round) {
            auto pair = [&](int a, int) {
                int p, q;
                if (a == 0) { p = tp - 1; q = round; }
                else { p = (round + a) % (tp - 1); q = (round - a + (tp - 1)) % (tp - 1); }
                if (p > q) std::swap(p, q);
                if (q >= t) return;
                double al = 0.0, be = 0.0;
                cplx ga = 0.0;
                const cplx *x = &B(0, p), *y = &B(0, q);
                for (int i = 0; i < c; ++i) {
                    al += std::norm(x[i]);
                    be += std::norm(y[i]);
                    ga += std::conj(x[i]) * y[i];
                }
                const double ag = std::abs(ga);
                if (ag <= 1e-15 * std::sqrt(al * be) || ag == 0.0) return;
                rotated++;
                const double tau = (be - al) / (2.0 * ag);
                const double tt = (tau >= 0 ? 1.0 : -1.0) / (std::abs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + tt * tt), sn = tt * cs;
                const cplx e = ga / ag;
                const cplx se = sn * e, sec = sn * std::conj(e);
                cplx *xm = &B(0, p), *ym = &B(0, q);
                for (int i = 0; i < c; ++i) {
                    const cplx xi = xm[i], yi = ym[i];
                    xm[i] = cs * xi - sec * yi;
                    ym[i] = se * xi + cs * yi;
                }
                cplx *jp = &J(0, p), *jq = &J(0, q);
                for (int i = 0; i < t; ++i) {
                    const cplx xi = jp[i], yi = jq[i];
                    jp[i] = cs * xi - sec * yi;
                    jq[i] = se * xi + cs * yi;
                }
            };
            // small rounds run inline: a thread start costs more than the work
            if ((int64_t)c * t < 200000) {
                for (int a = 0; a < tp / 2; ++a) pair(a, 0);
            } else {
                parallel_for(tp / 2, threads, pair);
            }
        }
        if (rotated.load() == 0) break;
    }
    std::vector<double> sv(t);
    for (int j = 0; j < t; ++j) {
        double s = 0.0;
        for (int i = 0; i < c; ++i) s += std::norm(B(i, j));
        sv[j] = std::sqrt(s);
    }
    std::vector<int> ord(t);
    for (int j = 0; j < t; ++j) ord[j] = j;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
    S.resize(t);
    // W = P X with X = B J / S;  U = Q [J; 0]
    W = Mat(c, t);
    U = Mat(r, t);
    for (int jj = 0; jj < t; ++jj) {
        const int j = ord[jj];
        S[jj] = sv[j];
        for (int i = 0; i < c; ++i) W(perm[i], jj) = sv[j] > 0 ? B(i, j) / sv[j] : cplx(0.0);
        for (int i = 0; i < t; ++i) U(i, jj) = J(i, j);
    }
    parallel_for(t, threads, [&](int jj, int) {
        cplx *u = &U(0, jj);
        for (int s = t - 1; s >= 0; --s) {
            const std::vector<cplx> &v = refl[s];
            cplx w = 0.0;
            for (int i = s; i < r; ++i) w += std::conj(v[i - s]) * u[i];
            for (int i = s; i < r; ++i) u[i] -= v[i - s] * w;
        }
    });
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

int ss_full_finish(const std::vector<std::vector<cplx>> &Amom, int k, int KQ, cplx gamma, double rho,
                   int threads, std::vector<cplx> &lam, std::vector<cplx> &G, int &nbar, double &gmax,
                   std::vector<cplx> *WBout) {
    if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
    std::vector<Mat> Am(2 * KQ, Mat(k, k));
    for (int al2 = 0; al2 < 2 * KQ; ++al2) Am[al2].a = Amom[al2];
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
    double tail = 0.0;
    svd_qr_jacobi(H, Us, sv, tail, Ws, threads, 1e-15);
    const int t = (int)sv.size();
    if (t == 0) return -1;
    // gap test over the resolved singular values and the bound of the rest
    std::vector<double> gs(sv);
    if (t < dim) gs.push_back(tail);
    nbar = 1;
    gmax = 0.0;
    for (int j = 0; j + 1 < (int)gs.size(); ++j) {
        const double r = gs[j] / std::max(gs[j + 1], 1e-300);
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
    if (WBout) {
        WBout->assign((size_t)dim * nbar, 0.0);
        for (int j = 0; j < nbar; ++j)
            for (int i = 0; i < dim; ++i) (*WBout)[(size_t)j * dim + i] = WB(i, j);
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
