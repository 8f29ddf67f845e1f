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
}  // namespace picgb
