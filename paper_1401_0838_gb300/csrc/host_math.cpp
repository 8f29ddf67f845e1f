// Host-side FP64 math of the library: the correction coefficients (Sec. 2, Eq. 3-5 and the
// (4,4) rational interpolation), the 9-tap Psi(D_z) stencils, the filter taps (Sec. 3 Eq. 6,
// Sec. 4) and the growth-rate fit. Plain C++ with libm; no CUDA.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "../../include/pic.h"
#include "host_math.h"

namespace picgb {

// Eq. 3-5 at s = k_z dz / 2, alpha = c dt / dz: sin(a s) cos(a s) / a times csc^2(s) s (Galerkin),
// csc(s) (Uniform) or cot(s) (momentum-conserving). All tend to 1 as s -> 0.
double field_multiplier(int scheme, double alpha, double s) {
  if (s <= 0.0) return 1.0;
  const double base = 0.5 * sin(2.0 * alpha * s) / alpha;
  const double sn = sin(s);
  if (scheme == PIC_GALERKIN) return base * (s / sn) / sn;
  if (scheme == PIC_UNIFORM) return base / sn;
  if (scheme == PIC_MOMENTUM) return base * cos(s) / sn;
  return NAN;
}

// Solve the 9x9 interpolation system by Householder QR (no pivoting). Returns the ratio of
// smallest to largest |R_ii| through *rcond.
static bool qr_solve9(double A[9][9], double b[9], double x[9], double* rcond) {
  const int n = 9;
  for (int k = 0; k < n; ++k) {
    double norm = 0.0;
    for (int i = k; i < n; ++i) norm += A[i][k] * A[i][k];
    norm = sqrt(norm);
    if (norm == 0.0) continue;
    const double alpha = A[k][k] > 0 ? -norm : norm;
    double v[9];
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    v[k] = A[k][k] - alpha;
    for (int i = k + 1; i < n; ++i) v[i] = A[i][k];
    double vv = 0.0;
    for (int i = k; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    for (int j = k; j < n; ++j) {
      double d = 0.0;
      for (int i = k; i < n; ++i) d += v[i] * A[i][j];
      d = 2.0 * d / vv;
      for (int i = k; i < n; ++i) A[i][j] -= d * v[i];
    }
    double d = 0.0;
    for (int i = k; i < n; ++i) d += v[i] * b[i];
    d = 2.0 * d / vv;
    for (int i = k; i < n; ++i) b[i] -= d * v[i];
  }
  double rmax = 0.0, rmin = INFINITY;
  for (int k = 0; k < n; ++k) {
    rmax = std::max(rmax, fabs(A[k][k]));
    rmin = std::min(rmin, fabs(A[k][k]));
  }
  *rcond = rmax > 0 ? rmin / rmax : 0.0;
  if (*rcond < 1e-14) return false;
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k][j] * x[j];
    x[k] = s / A[k][k];
  }
  return true;
}

int correction_coeffs(int scheme, double alpha, double pe[5], double pb[5]) {
  if (!(alpha > 0.0) || !isfinite(alpha) || scheme < PIC_GALERKIN || scheme > PIC_MOMENTUM) return PIC_E_ARG;
  double A[9][9], b[9], m[9];
  for (int j = 0; j < 9; ++j) {
    const double xi = j / 8.0;
    m[j] = field_multiplier(scheme, alpha, asin(sqrt(xi)));
    double xp[5] = {1.0, xi, xi * xi, xi * xi * xi, xi * xi * xi * xi};
    for (int q = 0; q < 5; ++q) A[j][q] = xp[q];             // a_0..a_4
    for (int q = 1; q < 5; ++q) A[j][4 + q] = -m[j] * xp[q];  // b_1..b_4
    b[j] = m[j];                                              // b_0 = 1 moved to the right
  }
  double x[9], rcond = 0.0;
  const bool ok = qr_solve9(A, b, x, &rcond);
  if (!ok) {
    // rank deficient: accept only the constant multiplier (Uniform at alpha = 1/2)
    for (int j = 0; j < 9; ++j)
      if (fabs(m[j] - 1.0) > 1e-12) return PIC_E_SINGULAR;
    for (int q = 0; q < 5; ++q) pe[q] = pb[q] = (q == 0) ? 1.0 : 0.0;
    return PIC_OK;
  }
  if (rcond < 1e-12) return PIC_E_SINGULAR;
  for (int q = 0; q < 5; ++q) pe[q] = x[q];
  pb[0] = 1.0;
  for (int q = 1; q < 5; ++q) pb[q] = x[4 + q];
  for (int t = 0; t <= 2048; ++t) {  // Psi_B must keep its sign on [0, 1]
    const double xi = t / 2048.0;
    const double v = pb[0] + xi * (pb[1] + xi * (pb[2] + xi * (pb[3] + xi * pb[4])));
    if (!(v > 0.0)) return PIC_E_SINGULAR;
  }
  return PIC_OK;
}

// Polynomial sum_n a_n D^n with D = -(1,-2,1)/4, as 9 taps for offsets -4..4 (Horner form:
// Psi = a0 + D(a1 + D(a2 + D(a3 + D a4)))).
void psi_stencil(const double a[5], double taps[9]) {
  double cur[9] = {0, 0, 0, 0, a[4], 0, 0, 0, 0};
  for (int q = 3; q >= 0; --q) {
    double nx[9];
    for (int t = 0; t < 9; ++t) {
      const double l = t > 0 ? cur[t - 1] : 0.0, r = t < 8 ? cur[t + 1] : 0.0;
      nx[t] = 0.5 * cur[t] - 0.25 * (l + r);
    }
    nx[4] += a[q];
    memcpy(cur, nx, sizeof cur);
  }
  memcpy(taps, cur, sizeof cur);
}

std::vector<double> convolve(const std::vector<double>& a, const std::vector<double>& b) {
  std::vector<double> c(a.size() + b.size() - 1, 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) c[i + j] += a[i] * b[j];
  return c;
}

// nbin bilinear passes (1,2,1)/4 and ncomp compensation passes (-(a-1)/2, a, -(a-1)/2).
std::vector<double> filter_taps(int nbin, int ncomp, double a) {
  std::vector<double> t{1.0};
  for (int i = 0; i < nbin; ++i) t = convolve(t, {0.25, 0.5, 0.25});
  for (int i = 0; i < ncomp; ++i) t = convolve(t, {-(a - 1.0) / 2.0, a, -(a - 1.0) / 2.0});
  return t;
}

static double lsq_slope(const double* t, const double* y, int n) {
  double tm = 0, ym = 0;
  for (int i = 0; i < n; ++i) {
    tm += t[i];
    ym += y[i];
  }
  tm /= n;
  ym /= n;
  double num = 0, den = 0;
  for (int i = 0; i < n; ++i) {
    num += (t[i] - tm) * (y[i] - ym);
    den += (t[i] - tm) * (t[i] - tm);
  }
  return num / den;
}

int growth_fit(const double* t_in, const double* w_in, int n_in, double* g, int* i0o, int* i1o) {
  for (int i = 0; i < n_in; ++i)
    if (!isfinite(t_in[i]) || (i > 0 && !(t_in[i] > t_in[i - 1]))) return PIC_E_ARG;  // times must increase
  std::vector<double> t, lnw, lg;
  std::vector<int> src;  // index of each kept sample in the caller's arrays
  for (int i = 0; i < n_in; ++i)
    if (w_in[i] > 0 && isfinite(w_in[i])) {
      t.push_back(t_in[i]);
      lnw.push_back(log(w_in[i]));
      lg.push_back(log10(w_in[i]));
      src.push_back(i);
    }
  const int n = (int)t.size();
  if (n < 5) return PIC_E_ARG;
  const int head = std::max(3, n / 10);
  std::vector<double> h(lg.begin(), lg.begin() + head);
  std::sort(h.begin(), h.end());
  const double floor_l = (head % 2) ? h[head / 2] : 0.5 * (h[head / 2 - 1] + h[head / 2]);
  const double sat = *std::max_element(lg.begin(), lg.end());
  const double lo = floor_l + 2.0, hi = sat - 1.0;
  int a = n;
  for (int i = 0; i < n; ++i)
    if (lg[i] >= lo) {
      a = i;
      break;
    }
  int b = a;
  while (b < n - 1 && lg[b] < hi) ++b;
  if (hi > lo && a < n && b - a + 1 >= 5) {
    *g = 0.5 * lsq_slope(&t[a], &lnw[a], b - a + 1);
    if (i0o) *i0o = src[a];
    if (i1o) *i1o = src[b];
    return PIC_OK;
  }
  const int m = std::max(5, n / 5);
  double best = -INFINITY;
  int bi = 0;
  for (int s = std::min(head, n - m); s + m <= n; ++s) {
    const double sl = lsq_slope(&t[s], &lnw[s], m);
    if (sl > best) {
      best = sl;
      bi = s;
    }
  }
  *g = 0.5 * best;
  if (i0o) *i0o = src[bi];
  if (i1o) *i1o = src[bi + m - 1];
  return PIC_OK;
}


int psi_inverse_factors(const double pb[5], double lam_re[4], double lam_im[4], int* nf, double* scale) {
  using cd = std::complex<double>;
  int deg = 4;
  while (deg > 0 && pb[deg] == 0.0) --deg;
  if (deg == 0) {
    if (pb[0] == 0.0) return PIC_E_ARG;
    *nf = 0;
    *scale = 1.0 / pb[0];
    return PIC_OK;
  }
  // roots of the monic polynomial by simultaneous (Durand-Kerner) iteration, then Newton polish
  cd c[5];
  for (int n = 0; n <= deg; ++n) c[n] = cd(pb[n] / pb[deg], 0.0);
  auto P = [&](cd x) {
    cd r = c[deg];
    for (int n = deg - 1; n >= 0; --n) r = r * x + c[n];
    return r;
  };
  auto dP = [&](cd x) {
    cd r = double(deg) * c[deg];
    for (int n = deg - 1; n >= 1; --n) r = r * x + double(n) * c[n];
    return r;
  };
  cd z[4];
  const cd seed(0.4, 0.9);
  for (int i = 0; i < deg; ++i) z[i] = std::pow(seed, i) * 2.0;
  for (int it = 0; it < 500; ++it) {
    double move = 0.0;
    for (int i = 0; i < deg; ++i) {
      cd den(1.0, 0.0);
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (z[i] - z[j]);
      const cd dz = P(z[i]) / den;
      z[i] -= dz;
      move = std::max(move, std::abs(dz));
    }
    if (move < 1e-15) break;
  }
  for (int i = 0; i < deg; ++i)
    for (int it = 0; it < 3; ++it) {
      const cd d = dP(z[i]);
      if (std::abs(d) > 0) z[i] -= P(z[i]) / d;
    }
  // a real root on [0, 1], or Psi_B changing sign there: no inverse
  for (int i = 0; i < deg; ++i)
    if (std::abs(z[i].imag()) < 1e-9 * (1.0 + std::abs(z[i])) && z[i].real() >= -1e-12 && z[i].real() <= 1.0 + 1e-12)
      return PIC_E_SINGULAR;
  for (int k = 0; k <= 64; ++k) {
    const double xi = k / 64.0;
    double v = 0.0, p = 1.0;
    for (int n = 0; n <= 4; ++n) {
      v += pb[n] * p;
      p *= xi;
    }
    if (!(v > 0.0) && !(v < 0.0)) return PIC_E_SINGULAR;
    if (k > 0 && (v > 0.0) != (pb[0] > 0.0)) return PIC_E_SINGULAR;
  }
  cd prod(1.0 / pb[deg], 0.0);
  for (int i = 0; i < deg; ++i) {
    const cd a = 0.5 - z[i];  // D - r = a - (S + S^-1) / 4
    const cd root = std::sqrt(4.0 * a * a - 1.0);
    cd lam = 2.0 * a - root;
    if (std::abs(lam) >= 1.0) lam = 2.0 * a + root;
    lam_re[i] = lam.real();
    lam_im[i] = lam.imag();
    prod *= 4.0 * lam;
  }
  *nf = deg;
  *scale = prod.real();
  return PIC_OK;
}

}  // namespace picgb
