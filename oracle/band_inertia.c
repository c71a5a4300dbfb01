/*
 * Sylvester inertia of a real symmetric band matrix (test infrastructure of
 * the FP64 oracle; nothing of the product links or calls it).
 *
 * T(x) of a real NEP is real symmetric for real x.  Its LDL^T factorisation
 * without pivoting, T = L D L^T (a congruence), has as many negative pivots
 * d_k as T has negative eigenvalues (Sylvester's law of inertia).  When T'(x)
 * is negative definite, the number of eigenvalues of the NEP in (a, b) is
 * nu(T(b)) - nu(T(a)), and bisection on nu pins every eigenvalue: the count
 * and eigenvalue pins of the grid rational problem and the loaded string
 * (all eigenvalues real, Section 5.1).
 *
 * Plain symmetric band elimination: column k gives the pivot d_k = A(k,k) and
 * the multipliers l_i = A(k+i,k) / d_k, and the trailing band is updated by
 * A(k+i, k+j) -= l_j A(k+i, k) for 1 <= j <= i <= bw.
 *
 *   n     order
 *   bw    half-bandwidth (A(i,j) = 0 for |i - j| > bw)
 *   ab    lower band storage, column major: A(j+d, j) at ab[d + j*ldab],
 *         0 <= d <= bw; overwritten by the factorisation
 *   ldab  >= bw + 1
 * Returns the number of negative pivots, or -1 if a pivot is exactly zero
 * (x is then an eigenvalue of a leading block and the count is undefined).
 */
int band_ldlt_negcount(int n, int bw, double *ab, int ldab) {
    int neg = 0;
    for (int k = 0; k < n; ++k) {
        const double d = ab[(long)k * ldab];
        if (d == 0.0) return -1;
        if (d < 0.0) ++neg;
        const int m = bw < n - 1 - k ? bw : n - 1 - k;
        const double *col = ab + (long)k * ldab + 1; /* A(k+1 .. k+m, k) */
        for (int j = 0; j < m; ++j) {
            const double lj = col[j] / d;
            double *cj = ab + (long)(k + 1 + j) * ldab; /* cj[i - j] = A(k+1+i, k+1+j) */
            for (int i = j; i < m; ++i) cj[i - j] -= lj * col[i];
        }
    }
    return neg;
}
