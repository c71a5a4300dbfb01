// Host FP64 SS-FULL for the projected NEP (see ssfull_host.cpp).
#pragma once
#include <complex>
#include <functional>
#include <vector>

namespace rsrr {

// Amom: the 2 KQ moments A_alpha (k x k, column major) of T_Q^{-1} on the
// ellipse (centre gamma, rho = max(a, b) scaling).  Outputs: lam (nbar
// eigenvalues of the projected NEP), G (k x nbar, column major; projected
// eigenvectors), nbar and the gap gmax.  Returns 0, or -1 if the moments
// vanish.
// With WB set, it also receives W0 Sigma0^{-1} B (KQ k x nbar, column major),
// the coefficients of the eigenvectors in the block moments (SS-RI, Eq. 41).
int ss_full_finish(const std::vector<std::vector<std::complex<double>>> &Amom, int k, int KQ,
                   std::complex<double> gamma, double rho, int threads,
                   std::vector<std::complex<double>> &lam, std::vector<std::complex<double>> &G,
                   int &nbar, double &gmax, std::vector<std::complex<double>> *WB = nullptr);

}  // namespace rsrr
