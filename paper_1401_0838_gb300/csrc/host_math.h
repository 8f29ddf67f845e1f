// Host FP64 helpers of the library (coefficients, stencils, growth fit).
#pragma once
#include <vector>

namespace picgb {
double field_multiplier(int scheme, double alpha, double s);
int correction_coeffs(int scheme, double alpha, double pe[5], double pb[5]);
void psi_stencil(const double a[5], double taps[9]);
std::vector<double> convolve(const std::vector<double>& a, const std::vector<double>& b);
std::vector<double> filter_taps(int nbin, int ncomp, double a);
int growth_fit(const double* t, const double* w, int n, double* g, int* i0, int* i1);
// Psi_B(D)^-1 on a periodic line as first-order recursions: with r_i the roots of Psi_B(xi),
// D - r = (1/(4 lam)) (1 - lam S)(1 - lam S^-1), lam + 1/lam = 2 - 4 r, |lam| < 1 (S: shift by one
// cell). Writes the lam_i (re, im pairs) and the real factor prod(4 lam_i) / b_deg; PIC_E_SINGULAR
// when Psi_B vanishes on [0, 1] (no inverse), PIC_E_ARG when Psi_B is identically zero.
int psi_inverse_factors(const double pb[5], double lam_re[4], double lam_im[4], int* nf, double* scale);
}  // namespace picgb
