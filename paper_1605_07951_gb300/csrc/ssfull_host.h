// Host FP64 SS-FULL for the projected NEP (see ssfull_host.cpp).
#pragma once
#include <complex>
#include <functional>
#include <vector>

namespace rsrr {

// P: m matrices k x k (column major).  f(i, z) = f_i(z).  Ellipse gamma, a, b.
// Outputs: lam (nbar eigenvalues of the projected NEP), G (k x nbar, column
// major; projected eigenvectors), nbar and the gap gmax.  Returns 0, or -1
// if T_Q is exactly singular at a quadrature node.
int ss_full_host(const std::vector<std::vector<std::complex<double>>> &P, int k,
                 const std::function<std::complex<double>(int, std::complex<double>)> &f, int m,
                 std::complex<double> gamma, double a, double b, int NQ, int KQ, int threads,
                 std::vector<std::complex<double>> &lam, std::vector<std::complex<double>> &G,
                 int &nbar, double &gmax);

}  // namespace rsrr
