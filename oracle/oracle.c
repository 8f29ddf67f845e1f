/*
 * FP64 CPU oracle for the stabilised FDTD-Esirkepov PIC time step of
 * Godfrey & Vay, "Suppressing the Numerical Cherenkov Instability in FDTD PIC
 * Codes" (arXiv 1401.0838).
 *
 * THIS IS TEST INFRASTRUCTURE. Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load it. The CUDA library never links,
 * includes or calls anything in this directory, and this file includes nothing
 * from the CUDA library: the two share no code, headers or constants.
 *
 * Style: plain, slow and literal. Every pass is applied on its own (no fusion),
 * there are no tiles, particles are visited one at a time, FP64 throughout,
 * libm for sin/cos/asin/log/exp, compiled with -ffp-contract=off.
 *
 * Units: c = eps0 = mu0 = 1, particle mass m = 1, charge q = +-1. Positions are
 * stored in grid units (x/dx), momenta as u = gamma*v. Fields live on the
 * standard Yee staggering (periodic in every direction):
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)
 *   Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k)
 * and array element [(k*ny+j)*nx+i] holds the component at the position above.
 * A 2D x-z run is the y-invariant case ny = 1, dy = 1.
 *
 * Parity pins for every function here are in tests/test_oracle_*.py. The
 * readings taken where the paper is silent are listed in the file header of
 * each section below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GALERKIN 0
#define ORC_UNIFORM 1
#define ORC_MOMENTUM 2

#define ORC_OK 0
#define ORC_E_SINGULAR (-1)
#define ORC_E_ARG (-2)

/* ------------------------------------------------------------------------ */
/* Parameters, fields and particles (the oracle's own types)                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int ndim;               /* 2 or 3 */
  int nx, ny, nz;         /* ny = 1 in 2D */
  double dx, dy, dz, dt;  /* dy = 1 in 2D */
  int scheme;             /* gather: 0 Galerkin, 1 Uniform */
  double psi_e[9];        /* 9-tap z-stencil of Psi_E(D_z), taps for offsets -4..4 */
  double psi_b[9];        /* 9-tap z-stencil of Psi_B(D_z) */
  int f_nbin;             /* bilinear passes per direction, per side */
  int f_ncomp;            /* compensation passes per direction, per side */
  double f_alpha;         /* compensation centre weight (3 in the paper's filter) */
  int f_targets;          /* bit 0: filter J; bit 1: filter the gather copies */
  int order;              /* particle shape order: 1 (linear) or 3 (cubic) */
  int corr_mode;          /* 0: Psi_E on Ex, Ey and Psi_B on the others; 1: Psi_E / Psi_B on Ex, Ey only */
  double psi_b_coef[5];   /* Psi_B polynomial coefficients (powers of xi), used by corr_mode 1 */
  int solver;             /* 0: Yee; 1: Cole-Karkkainen curl of E in the B update (2D x-z only) */
  double ck_beta_x;       /* CK: transverse (z) averaging weight of the x differences */
  double ck_beta_z;       /* CK: transverse (x) averaging weight of the z differences (Fig. 1: 1/8) */
} orc_params;

typedef struct {
  double *ex, *ey, *ez, *bx, *by, *bz, *jx, *jy, *jz;
} orc_fields;

typedef struct {
  long n;
  double *x, *y, *z;    /* grid units, in [0, n) after every step; y unused in 2D */
  double *ux, *uy, *uz; /* u = gamma v */
  double *w;            /* number weight of the macro-particle */
  double *q;            /* charge, -1 or +1 (mass 1) */
} orc_particles;

static long idx3(const orc_params* p, int i, int j, int k) {
  return ((long)k * p->ny + j) * p->nx + i;
}
static int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}
static double wrapf(double x, double n) {
  double r = fmod(x, n);
  if (r < 0) r += n;
  if (r >= n) r -= n;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, Eq. 3-5: field multipliers; s = k_z dz / 2, alpha = c dt / dz.     */
/* k_z dt / 2 = alpha s and dz/dt = 1/alpha (c = 1).                          */
/* The multiplier speed is c (tuned for infinite gamma, Sec. 3).             */
/* ------------------------------------------------------------------------ */
double orc_multiplier(int scheme, double alpha, double s) {
  if (s == 0.0) return 1.0; /* limit s -> 0 of every form */
  double sc = sin(alpha * s) * cos(alpha * s) / alpha;
  switch (scheme) {
    case ORC_GALERKIN: /* Eq. 3: ... csc^2(s) * s */
      return sc * s / (sin(s) * sin(s));
    case ORC_UNIFORM: /* Eq. 4: ... csc(s) */
      return sc / sin(s);
    case ORC_MOMENTUM: /* Eq. 5: ... cot(s) */
      return sc * cos(s) / sin(s);
    default:
      return NAN;
  }
}

/* Value of the polynomial sum_n c[n] xi^n, n = 0..4. */
static double poly4(const double c[5], double xi) {
  double r = 0.0, p = 1.0;
  for (int n = 0; n < 5; ++n) {
    r += c[n] * p;
    p *= xi;
  }
  return r;
}

/*
 * Sec. 2: (4,4) rational interpolation of the multiplier in xi = sin^2(s) on
 * the nine nodes xi_j = j/8. Unknowns a0..a4 (Psi_E) and b1..b4 (Psi_B, with
 * b0 = 1); the interpolation conditions Psi_E(xi_j) = M_j Psi_B(xi_j) are the
 * linear system sum_n a_n xi^n - M_j sum_{n>=1} b_n xi^n = M_j, solved here by
 * Gaussian elimination with partial pivoting.
 * Degenerate case (reading): if the system is singular, the constant
 * interpolant Psi_E = Psi_B = 1 is returned when it reproduces every node
 * (Uniform at alpha = 1/2, where the multiplier is identically 1); any other
 * singular case, or a Psi_B with a zero on [0,1], returns ORC_E_SINGULAR.
 */
int orc_rational_coeffs(int scheme, double alpha, double psi_e[5], double psi_b[5]) {
  double A[9][10];
  double m[9];
  double amax = 0.0;
  for (int j = 0; j < 9; ++j) {
    double xi = j / 8.0;
    double s = asin(sqrt(xi));
    m[j] = orc_multiplier(scheme, alpha, s);
    double p = 1.0;
    for (int n = 0; n <= 4; ++n) {
      A[j][n] = p;
      if (n >= 1) A[j][4 + n] = -m[j] * p;
      p *= xi;
    }
    A[j][9] = m[j];
    for (int c = 0; c < 9; ++c) amax = fmax(amax, fabs(A[j][c]));
  }
  int singular = 0;
  for (int c = 0; c < 9; ++c) {
    int piv = c;
    for (int r = c + 1; r < 9; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (fabs(A[piv][c]) <= 1e-12 * amax) {
      singular = 1;
      break;
    }
    if (piv != c)
      for (int cc = 0; cc < 10; ++cc) {
        double t = A[c][cc];
        A[c][cc] = A[piv][cc];
        A[piv][cc] = t;
      }
    for (int r = c + 1; r < 9; ++r) {
      double f = A[r][c] / A[c][c];
      for (int cc = c; cc < 10; ++cc) A[r][cc] -= f * A[c][cc];
    }
  }
  if (singular) {
    for (int j = 0; j < 9; ++j)
      if (fabs(m[j] - 1.0) > 1e-12) return ORC_E_SINGULAR;
    for (int n = 0; n < 5; ++n) psi_e[n] = psi_b[n] = (n == 0) ? 1.0 : 0.0;
    return ORC_OK;
  }
  double sol[9];
  for (int r = 8; r >= 0; --r) {
    double acc = A[r][9];
    for (int c = r + 1; c < 9; ++c) acc -= A[r][c] * sol[c];
    sol[r] = acc / A[r][r];
  }
  for (int n = 0; n < 5; ++n) psi_e[n] = sol[n];
  psi_b[0] = 1.0;
  for (int n = 1; n < 5; ++n) psi_b[n] = sol[4 + n];
  for (int t = 0; t <= 4096; ++t)
    if (poly4(psi_b, t / 4096.0) <= 0.0) return ORC_E_SINGULAR;
  return ORC_OK;
}

/*
 * Sec. 2: xi corresponds to the operator D = -(1,-2,1)/4 along z, since
 * D exp(i k z) = sin^2(k dz/2) exp(i k z). Psi(D) = sum_n a_n D^n is a 9-tap
 * symmetric stencil; taps[m+4] multiplies f[k+m]. Built by repeated
 * convolution of D with itself.
 */
void orc_psi_taps(const double a[5], double taps[9]) {
  double pw[9] = {0, 0, 0, 0, 1, 0, 0, 0, 0}; /* D^0 */
  const double d[3] = {-0.25, 0.5, -0.25};
  for (int m = 0; m < 9; ++m) taps[m] = a[0] * pw[m];
  for (int n = 1; n <= 4; ++n) {
    double nx[9] = {0};
    for (int m = 0; m < 9; ++m)
      for (int t = -1; t <= 1; ++t) {
        int mm = m + t;
        if (mm >= 0 && mm < 9) nx[mm] += pw[m] * d[t + 1];
      }
    memcpy(pw, nx, sizeof pw);
    for (int m = 0; m < 9; ++m) taps[m] += a[n] * pw[m];
  }
}

/* ------------------------------------------------------------------------ */
/* Periodic convolutions along one axis (0 = x, 1 = y, 2 = z).               */
/* ------------------------------------------------------------------------ */
void orc_conv_axis(const orc_params* p, double* f, int axis, const double* taps, int half) {
  long ncell = (long)p->nx * p->ny * p->nz;
  double* out = (double*)malloc(sizeof(double) * ncell);
  int n = axis == 0 ? p->nx : axis == 1 ? p->ny : p->nz;
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        double acc = 0.0;
        for (int m = -half; m <= half; ++m) {
          int ii = i, jj = j, kk = k;
          if (axis == 0) ii = wrap(i + m, n);
          if (axis == 1) jj = wrap(j + m, n);
          if (axis == 2) kk = wrap(k + m, n);
          acc += taps[m + half] * f[idx3(p, ii, jj, kk)];
        }
        out[idx3(p, i, j, k)] = acc;
      }
  memcpy(f, out, sizeof(double) * ncell);
  free(out);
}

/*
 * Sec. 3 (Eq. 6) and Sec. 4: the digital filter is a number of bilinear
 * (1/4, 1/2, 1/4) passes, transfer cos^2(s), and of compensation passes
 * (-(a-1)/2, a, -(a-1)/2), transfer a - (a-1) cos(2s) (= 5 - 4cos^2 s for
 * a = 3), along every direction of the grid. One bilinear and one
 * compensation pass per direction is the square root of Eq. 6.
 */
void orc_filter(const orc_params* p, double* f) {
  const double bil[3] = {0.25, 0.5, 0.25};
  const double cmp[3] = {-(p->f_alpha - 1.0) / 2.0, p->f_alpha, -(p->f_alpha - 1.0) / 2.0};
  int naxes[3] = {1, p->ndim == 3, 1};
  for (int axis = 0; axis < 3; ++axis) {
    if (!naxes[axis]) continue;
    for (int r = 0; r < p->f_nbin; ++r) orc_conv_axis(p, f, axis, bil, 1);
    for (int r = 0; r < p->f_ncomp; ++r) orc_conv_axis(p, f, axis, cmp, 1);
  }
}

/*
 * Sec. 2 (last paragraph) and Sec. 3: the copies of the fields that the
 * particles see. Psi_E is applied to the transverse E components (Ex, Ey) and
 * Psi_B to every other component (Ez, Bx, By, Bz); the 3D rule is used in 2D
 * too (reading). Then the gather-side share of the digital filter. The Yee
 * fields themselves are never modified.
 * out[0..5] receive Ex, Ey, Ez, Bx, By, Bz copies.
 */
/*
 * Sec. 2: Psi_B applied exactly, by its inverse: on a periodic line of nz
 * cells the operator Psi_B(D_z) is circulant, with eigenvalue
 * Psi_B(sin^2(pi m / nz)) on the Fourier mode m, so its inverse divides each
 * mode by that value. Written as a direct DFT along z (O(nz^2) per line).
 */
void orc_inverse_psi_z(const orc_params* p, double* f) {
  const int nz = p->nz;
  const long nxy = (long)p->nx * p->ny;
  const double two_pi = 6.283185307179586476925286766559;
  double* re = (double*)malloc(sizeof(double) * nz);
  double* im = (double*)malloc(sizeof(double) * nz);
  for (long l = 0; l < nxy; ++l) {
    for (int m = 0; m < nz; ++m) { /* forward transform, then divide by the symbol */
      double a = 0.0, b = 0.0;
      for (int k = 0; k < nz; ++k) {
        double ph = -two_pi * (double)m * (double)k / (double)nz;
        a += f[k * nxy + l] * cos(ph);
        b += f[k * nxy + l] * sin(ph);
      }
      double sn = sin(0.5 * two_pi * (double)m / (double)nz);
      double den = poly4(p->psi_b_coef, sn * sn);
      re[m] = a / den;
      im[m] = b / den;
    }
    for (int k = 0; k < nz; ++k) { /* inverse transform (the result is real) */
      double a = 0.0;
      for (int m = 0; m < nz; ++m) {
        double ph = two_pi * (double)m * (double)k / (double)nz;
        a += re[m] * cos(ph) - im[m] * sin(ph);
      }
      f[k * nxy + l] = a / (double)nz;
    }
  }
  free(re);
  free(im);
}

void orc_gather_copies(const orc_params* p, const orc_fields* F, double* out[6]) {
  long ncell = (long)p->nx * p->ny * p->nz;
  const double* src[6] = {F->ex, F->ey, F->ez, F->bx, F->by, F->bz};
  for (int c = 0; c < 6; ++c) {
    memcpy(out[c], src[c], sizeof(double) * ncell);
    if (p->corr_mode == 1) {
      /* Sec. 2 / Sec. 3 variant: the rational multiplier Psi_E / Psi_B on the transverse E copies
         only (Psi_B by exact inversion), none on the other components */
      if (c < 2) {
        orc_conv_axis(p, out[c], 2, p->psi_e, 4);
        orc_inverse_psi_z(p, out[c]);
      }
    } else {
      orc_conv_axis(p, out[c], 2, c < 2 ? p->psi_e : p->psi_b, 4);
    }
    if (p->f_targets & 2) orc_filter(p, out[c]);
  }
}

/* ------------------------------------------------------------------------ */
/* Yee solver (standard staggering, periodic)                                */
/* ------------------------------------------------------------------------ */
/* Cole-Karkkainen solver (named in Sec. 2 for Fig. 1, with beta_z = 1/8), 2D x-z reading: the
   B update uses a curl of E in which the forward difference along z is averaged over the x
   neighbours i-1, i, i+1 with weights (beta_z, 1 - 2 beta_z, beta_z), and the forward difference
   along x over the z neighbours with (beta_x, 1 - 2 beta_x, beta_x). The E update stays Yee's, so
   Gauss's law and the Esirkepov charge conservation are those of Yee. Both are written out literally
   below: one averaged difference per call. */
static double ck_dz(const orc_params* p, const double* f, int i, int k) {
  const int kp = wrap(k + 1, p->nz);
  double s = 0.0;
  for (int a = -1; a <= 1; ++a) {
    const int ia = wrap(i + a, p->nx);
    const double w = a == 0 ? 1.0 - 2.0 * p->ck_beta_z : p->ck_beta_z;
    s += w * (f[idx3(p, ia, 0, kp)] - f[idx3(p, ia, 0, k)]);
  }
  return s / p->dz;
}

static double ck_dx(const orc_params* p, const double* f, int i, int k) {
  const int ip = wrap(i + 1, p->nx);
  double s = 0.0;
  for (int b = -1; b <= 1; ++b) {
    const int kb = wrap(k + b, p->nz);
    const double w = b == 0 ? 1.0 - 2.0 * p->ck_beta_x : p->ck_beta_x;
    s += w * (f[idx3(p, ip, 0, kb)] - f[idx3(p, i, 0, kb)]);
  }
  return s / p->dx;
}

/* B -= h curl_CK E (2D: the y differences vanish) */
static void orc_ck_b(const orc_params* p, orc_fields* F, double h) {
  for (int k = 0; k < p->nz; ++k)
    for (int i = 0; i < p->nx; ++i) {
      const long c = idx3(p, i, 0, k);
      const double cex = -ck_dz(p, F->ey, i, k);
      const double cey = ck_dz(p, F->ex, i, k) - ck_dx(p, F->ez, i, k);
      const double cez = ck_dx(p, F->ey, i, k);
      F->bx[c] -= h * cex;
      F->by[c] -= h * cey;
      F->bz[c] -= h * cez;
    }
}

/* B -= h curl E */
void orc_yee_b(const orc_params* p, orc_fields* F, double h) {
  if (p->solver == 1) {
    orc_ck_b(p, F, h);
    return;
  }
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        int ip = wrap(i + 1, p->nx), jp = wrap(j + 1, p->ny), kp = wrap(k + 1, p->nz);
        long c = idx3(p, i, j, k);
        double cex = (F->ez[idx3(p, i, jp, k)] - F->ez[c]) / p->dy - (F->ey[idx3(p, i, j, kp)] - F->ey[c]) / p->dz;
        double cey = (F->ex[idx3(p, i, j, kp)] - F->ex[c]) / p->dz - (F->ez[idx3(p, ip, j, k)] - F->ez[c]) / p->dx;
        double cez = (F->ey[idx3(p, ip, j, k)] - F->ey[c]) / p->dx - (F->ex[idx3(p, i, jp, k)] - F->ex[c]) / p->dy;
        F->bx[c] -= h * cex;
        F->by[c] -= h * cey;
        F->bz[c] -= h * cez;
      }
}

/* E += h (curl B - J) */
void orc_yee_e(const orc_params* p, orc_fields* F, double h) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        int im = wrap(i - 1, p->nx), jm = wrap(j - 1, p->ny), km = wrap(k - 1, p->nz);
        long c = idx3(p, i, j, k);
        double cbx = (F->bz[c] - F->bz[idx3(p, i, jm, k)]) / p->dy - (F->by[c] - F->by[idx3(p, i, j, km)]) / p->dz;
        double cby = (F->bx[c] - F->bx[idx3(p, i, j, km)]) / p->dz - (F->bz[c] - F->bz[idx3(p, im, j, k)]) / p->dx;
        double cbz = (F->by[c] - F->by[idx3(p, im, j, k)]) / p->dx - (F->bx[c] - F->bx[idx3(p, i, jm, k)]) / p->dy;
        F->ex[c] += h * (cbx - F->jx[c]);
        F->ey[c] += h * (cby - F->jy[c]);
        F->ez[c] += h * (cbz - F->jz[c]);
      }
}

/* ------------------------------------------------------------------------ */
/* Particle shapes and field gather (Sec. 2 Eq. 3-4; Sec. 3 last paragraph)  */
/* ------------------------------------------------------------------------ */
/* Linear spline S1(d) = max(0, 1-|d|). */
static double S1(double d) {
  double a = 1.0 - fabs(d);
  return a > 0.0 ? a : 0.0;
}

/*
 * Centred cardinal B-spline of order n (n = 0..3) at t, in cell units: S0 the
 * box [-1/2, 1/2), S1 the hat, S2 the quadratic and S3 the cubic spline (each
 * the box convolved with the previous one). Sec. 3 runs with cubic shapes.
 */
static double bspline(int n, double t) {
  double a = fabs(t);
  switch (n) {
    case 0:
      return (t >= -0.5 && t < 0.5) ? 1.0 : 0.0;
    case 1:
      return S1(t);
    case 2:
      if (a <= 0.5) return 0.75 - a * a;
      if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
      return 0.0;
    case 3:
      if (a <= 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
      if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
      return 0.0;
    default:
      return NAN;
  }
}

double orc_bspline(int n, double t) { return bspline(n, t); }

/*
 * Interpolate one component at grid-unit position (x[0..2]) with stagger
 * st[axis] (0: nodes at integers, 1: nodes at half-integers) and spline order
 * ord[axis] (0..3): the ord+1 nodes of this component's lattice nearest the
 * position, weighted by the B-spline of that order.
 * Galerkin: one order lower along each direction in which the component is
 * half staggered, the particle shape order along the others (the ratio of
 * Eq. 3 to Eq. 4 is s/sin s, the ratio of the transforms of consecutive
 * B-splines). Uniform: the shape order everywhere.
 */
static double gather1(const orc_params* p, const double* F, const double x[3], const int st[3], const int ord[3]) {
  int n[3] = {p->nx, p->ny, p->nz};
  int base[3], cnt[3];
  double wt[3][4];
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && p->ndim == 2) {
      base[a] = 0;
      cnt[a] = 1;
      wt[a][0] = 1.0;
      continue;
    }
    double xs = x[a] - 0.5 * st[a]; /* coordinate in units of this component's node lattice */
    int o = ord[a];
    /* first node: floor(xs) - (o-1)/2 for odd orders, floor(xs + 1/2) - o/2 for even ones */
    base[a] = (o % 2) ? (int)floor(xs) - (o - 1) / 2 : (int)floor(xs + 0.5) - o / 2;
    cnt[a] = o + 1;
    for (int q = 0; q < cnt[a]; ++q) wt[a][q] = bspline(o, xs - (double)(base[a] + q));
  }
  double acc = 0.0;
  for (int c = 0; c < cnt[2]; ++c)
    for (int b = 0; b < cnt[1]; ++b)
      for (int a = 0; a < cnt[0]; ++a) {
        long id = idx3(p, wrap(base[0] + a, n[0]), wrap(base[1] + b, n[1]), wrap(base[2] + c, n[2]));
        acc += wt[0][a] * wt[1][b] * wt[2][c] * F[id];
      }
  return acc;
}

/* Stagger of Ex, Ey, Ez, Bx, By, Bz along x, y, z. */
static const int STAG[6][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

/*
 * Momentum-conserving scheme (the one Eq. 5 belongs to): a component averaged
 * from its Yee location to the node (i, j, k), i.e. over the two neighbours
 * along each direction in which it is half staggered.
 */
static double node_average(const orc_params* p, const double* F, int c, int i, int j, int k) {
  int n[3] = {p->nx, p->ny, p->nz};
  int lo[3] = {i, j, k};
  int m[3];
  for (int a = 0; a < 3; ++a) m[a] = STAG[c][a] ? 2 : 1;
  double acc = 0.0;
  for (int dc = 0; dc < m[2]; ++dc)
    for (int db = 0; db < m[1]; ++db)
      for (int da = 0; da < m[0]; ++da)
        acc += F[idx3(p, wrap(lo[0] - da, n[0]), wrap(lo[1] - db, n[1]), wrap(lo[2] - dc, n[2]))];
  return acc / (double)(m[0] * m[1] * m[2]);
}

static double gather_momentum(const orc_params* p, const double* F, int c, const double x[3]) {
  int n[3] = {p->nx, p->ny, p->nz};
  int o = p->order;
  int base[3], cnt[3];
  double wt[3][4];
  for (int a = 0; a < 3; ++a) {
    if (a == 1 && p->ndim == 2) {
      base[a] = 0;
      cnt[a] = 1;
      wt[a][0] = 1.0;
      continue;
    }
    base[a] = (int)floor(x[a]) - (o - 1) / 2;
    cnt[a] = o + 1;
    for (int q = 0; q < cnt[a]; ++q) wt[a][q] = bspline(o, x[a] - (double)(base[a] + q));
  }
  double acc = 0.0;
  for (int cc = 0; cc < cnt[2]; ++cc)
    for (int b = 0; b < cnt[1]; ++b)
      for (int a = 0; a < cnt[0]; ++a)
        acc += wt[0][a] * wt[1][b] * wt[2][cc] *
               node_average(p, F, c, wrap(base[0] + a, n[0]), wrap(base[1] + b, n[1]), wrap(base[2] + cc, n[2]));
  return acc;
}

/* Gather the six components from field arrays G[6] at particle position. */
void orc_gather_point(const orc_params* p, double* const G[6], double x, double y, double z, double out[6]) {
  double pos[3] = {x, y, z};
  for (int c = 0; c < 6; ++c) {
    if (p->scheme == ORC_MOMENTUM) {
      out[c] = gather_momentum(p, G[c], c, pos);
      continue;
    }
    int ord[3];
    for (int a = 0; a < 3; ++a) ord[a] = (p->scheme == ORC_GALERKIN) ? p->order - STAG[c][a] : p->order;
    out[c] = gather1(p, G[c], pos, STAG[c], ord);
  }
}

void orc_gather(const orc_params* p, double* const G[6], const double* x, const double* y, const double* z, long n,
                double* out6[6]) {
  for (long i = 0; i < n; ++i) {
    double o[6];
    orc_gather_point(p, G, x[i], p->ndim == 3 ? y[i] : 0.0, z[i], o);
    for (int c = 0; c < 6; ++c) out6[c][i] = o[c];
  }
}

/* ------------------------------------------------------------------------ */
/* Relativistic Boris push (Boris 1970; the paper does not state its pusher) */
/* ------------------------------------------------------------------------ */
void orc_boris(double q, double dt, const double E[3], const double B[3], double u[3]) {
  double h = 0.5 * q * dt; /* q dt / (2 m), m = 1 */
  double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
  double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double t[3] = {h * B[0] / g, h * B[1] / g, h * B[2] / g};
  double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + tt), 2.0 * t[1] / (1.0 + tt), 2.0 * t[2] / (1.0 + tt)};
  double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]), um[1] + (um[2] * t[0] - um[0] * t[2]),
                  um[2] + (um[0] * t[1] - um[1] * t[0])};
  double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]), um[1] + (up[2] * s[0] - up[0] * s[2]),
                   um[2] + (up[0] * s[1] - up[1] * s[0])};
  for (int a = 0; a < 3; ++a) u[a] = upl[a] + h * E[a];
}

void orc_boris_many(const double* q, double dt, double* const E3[3], double* const B3[3], double* ux, double* uy,
                    double* uz, long n) {
  for (long i = 0; i < n; ++i) {
    double E[3] = {E3[0][i], E3[1][i], E3[2][i]}, B[3] = {B3[0][i], B3[1][i], B3[2][i]};
    double u[3] = {ux[i], uy[i], uz[i]};
    orc_boris(q[i], dt, E, B, u);
    ux[i] = u[0];
    uy[i] = u[1];
    uz[i] = u[2];
  }
}

/* ------------------------------------------------------------------------ */
/* Esirkepov current deposition (Esirkepov 2001; cited in Sec. 2)            */
/* ------------------------------------------------------------------------ */
/*
 * Charge density at node (i,j,k): rho = sum q w S1 S1 (S1) / dV, dV = dx dy dz.
 * The weights W satisfy S1(x1)S1(z1) - S1(x0)S1(z0) = Wx + Wz (2D) and the
 * currents follow from discrete continuity,
 *   J_a(node + 1/2 e_a) - J_a(node - 1/2 e_a) = -(q w d_a / (dV dt)) W_a(node),
 * summed from a node left of the footprint where J = 0.
 * The move is given as start position r0 (grid units) and displacement dr
 * (|dr| < 1 cell); shapes are evaluated relative to the start cell
 * floor(r0), and each shape change dS = S1(n - r0 - dr) - S1(n - r0) is formed
 * from the displacement: where both arguments lie on the same linear piece of
 * S1 it equals the slope times -dr exactly, so that a move far below one cell
 * (the transverse drift of a cold relativistic beam) keeps full relative
 * precision. Across a kink of S1 the two shape values are subtracted.
 */
#define FP 6 /* footprint window: nodes -2..3 relative to the start cell */

/* piece of S1 containing a: 0 (a <= -1), 1 (-1 < a <= 0), 2 (0 < a < 1), 3 (a >= 1) */
static int s1_piece(double a) { return a <= -1.0 ? 0 : a <= 0.0 ? 1 : a < 1.0 ? 2 : 3; }

static double s1_change(double a0, double d) {
  double a1 = a0 - d;
  int p = s1_piece(a0);
  if (p == s1_piece(a1)) {
    double slope = p == 1 ? 1.0 : p == 2 ? -1.0 : 0.0;
    return slope * (-d);
  }
  return S1(a1) - S1(a0);
}

/*
 * Cubic spline: its polynomial pieces are (-2,-1], (-1,0], (0,1], (1,2); on one
 * piece P(a0 - d) - P(a0) = -d P'(a0) + d^2/2 P''(a0) - d^3/6 P'''(a0) exactly
 * (the Taylor series of a cubic ends there), which keeps full relative
 * precision for small moves; across a knot the two values are subtracted.
 */
static int s3_piece(double t) {
  return t <= -2.0 ? 0 : t <= -1.0 ? 1 : t <= 0.0 ? 2 : t <= 1.0 ? 3 : t < 2.0 ? 4 : 5;
}

static double s3_change(double a0, double d) {
  double a1 = a0 - d;
  int p = s3_piece(a0);
  if (p != s3_piece(a1)) return bspline(3, a1) - bspline(3, a0);
  double d1, d2, d3; /* P', P'', P''' at a0 */
  switch (p) {
    case 1:
      d1 = 0.5 * (2.0 + a0) * (2.0 + a0);
      d2 = 2.0 + a0;
      d3 = 1.0;
      break;
    case 2:
      d1 = -2.0 * a0 - 1.5 * a0 * a0;
      d2 = -2.0 - 3.0 * a0;
      d3 = -3.0;
      break;
    case 3:
      d1 = -2.0 * a0 + 1.5 * a0 * a0;
      d2 = -2.0 + 3.0 * a0;
      d3 = 3.0;
      break;
    case 4:
      d1 = -0.5 * (2.0 - a0) * (2.0 - a0);
      d2 = 2.0 - a0;
      d3 = -1.0;
      break;
    default:
      return 0.0; /* outside the support on both sides */
  }
  return -d * d1 + 0.5 * d * d * d2 - d * d * d * d3 / 6.0;
}

/* S0 and dS of the particle shape (order 1 or 3) on the window nodes lo+a, a = 0..FP-1, for one direction */
static void shape_window(int order, double r0, double dr, int* lo, double S0[FP], double dS[FP]) {
  double c = floor(r0);
  double o = r0 - c;
  *lo = (int)c - 2;
  for (int a = 0; a < FP; ++a) {
    double node = a - 2; /* relative to the start cell */
    if (order == 3) {
      S0[a] = bspline(3, node - o);
      dS[a] = s3_change(node - o, dr);
    } else {
      S0[a] = S1(node - o);
      dS[a] = s1_change(node - o, dr);
    }
  }
}

void orc_deposit_2d(const orc_params* p, orc_fields* F, double x0, double z0, double ddx, double ddz, double vy,
                    double qw) {
  double dV = p->dx * p->dy * p->dz;
  int ia, ka;
  double S0x[FP], dSx[FP], S0z[FP], dSz[FP];
  shape_window(p->order, x0, ddx, &ia, S0x, dSx);
  shape_window(p->order, z0, ddz, &ka, S0z, dSz);
  double cx = -qw * p->dx / (dV * p->dt);
  double cz = -qw * p->dz / (dV * p->dt);
  double cy = qw * vy / dV;
  for (int b = 0; b < FP; ++b) { /* Jx(i+1/2, k): running sum over i */
    double acc = 0.0;
    for (int a = 0; a < FP; ++a) {
      acc += dSx[a] * (S0z[b] + 0.5 * dSz[b]);
      if (acc != 0.0) F->jx[idx3(p, wrap(ia + a, p->nx), 0, wrap(ka + b, p->nz))] += cx * acc;
    }
  }
  for (int a = 0; a < FP; ++a) { /* Jz(i, k+1/2): running sum over k */
    double acc = 0.0;
    for (int b = 0; b < FP; ++b) {
      acc += dSz[b] * (S0x[a] + 0.5 * dSx[a]);
      if (acc != 0.0) F->jz[idx3(p, wrap(ia + a, p->nx), 0, wrap(ka + b, p->nz))] += cz * acc;
    }
  }
  for (int b = 0; b < FP; ++b) /* Jy(i, k): out-of-plane weight */
    for (int a = 0; a < FP; ++a) {
      double wy = S0x[a] * S0z[b] + 0.5 * dSx[a] * S0z[b] + 0.5 * S0x[a] * dSz[b] + dSx[a] * dSz[b] / 3.0;
      if (wy != 0.0) F->jy[idx3(p, wrap(ia + a, p->nx), 0, wrap(ka + b, p->nz))] += cy * wy;
    }
}

void orc_deposit_3d(const orc_params* p, orc_fields* F, const double r0[3], const double dr[3], double qw) {
  double dV = p->dx * p->dy * p->dz;
  int n[3] = {p->nx, p->ny, p->nz};
  double d[3] = {p->dx, p->dy, p->dz};
  int lo[3];
  double S0[3][FP], dS[3][FP];
  for (int ax = 0; ax < 3; ++ax) shape_window(p->order, r0[ax], dr[ax], &lo[ax], S0[ax], dS[ax]);
  double* J[3] = {F->jx, F->jy, F->jz};
  for (int ax = 0; ax < 3; ++ax) {
    int b1 = (ax + 1) % 3, b2 = (ax + 2) % 3; /* the two transverse axes */
    double c = -qw * d[ax] / (dV * p->dt);
    for (int t2 = 0; t2 < FP; ++t2)
      for (int t1 = 0; t1 < FP; ++t1) {
        /* transverse factor of W_ax: S0 S0 + dS S0/2 + S0 dS/2 + dS dS/3 */
        double tr = S0[b1][t1] * S0[b2][t2] + 0.5 * dS[b1][t1] * S0[b2][t2] + 0.5 * S0[b1][t1] * dS[b2][t2] +
                    dS[b1][t1] * dS[b2][t2] / 3.0;
        double acc = 0.0;
        for (int a = 0; a < FP; ++a) {
          acc += dS[ax][a] * tr;
          if (acc == 0.0) continue;
          int node[3];
          node[ax] = lo[ax] + a;
          node[b1] = lo[b1] + t1;
          node[b2] = lo[b2] + t2;
          J[ax][idx3(p, wrap(node[0], n[0]), wrap(node[1], n[1]), wrap(node[2], n[2]))] += c * acc;
        }
      }
  }
}

/* Node charge density with S1 shapes (used by the continuity and Gauss checks). */
void orc_rho(const orc_params* p, const orc_particles* P, double* rho) {
  long ncell = (long)p->nx * p->ny * p->nz;
  double dV = p->dx * p->dy * p->dz;
  memset(rho, 0, sizeof(double) * ncell);
  for (long m = 0; m < P->n; ++m) {
    double r[3] = {P->x[m], p->ndim == 3 ? P->y[m] : 0.0, P->z[m]};
    int n[3] = {p->nx, p->ny, p->nz};
    int b[3];
    double wt[3][4];
    const int o = p->order, nn = o + 1; /* the shape's o+1 nodes per direction */
    for (int a = 0; a < 3; ++a) {
      double fl = floor(r[a]);
      b[a] = (int)fl - (o - 1) / 2;
      for (int q = 0; q < nn; ++q) wt[a][q] = bspline(o, r[a] - (double)(b[a] + q));
    }
    int cy = p->ndim == 3 ? nn : 1;
    for (int c = 0; c < nn; ++c)
      for (int bb = 0; bb < cy; ++bb)
        for (int a = 0; a < nn; ++a) {
          double wy = p->ndim == 3 ? wt[1][bb] : 1.0;
          rho[idx3(p, wrap(b[0] + a, n[0]), wrap(b[1] + bb, n[1]), wrap(b[2] + c, n[2]))] +=
              P->q[m] * P->w[m] * wt[0][a] * wy * wt[2][c] / dV;
        }
  }
}

/* ------------------------------------------------------------------------ */
/* One full time step, in the order the paper's loop implies                 */
/* ------------------------------------------------------------------------ */
/*
 * State in: x^n, u^{n-1/2}, E^n, B^n. State out: x^{n+1}, u^{n+1/2}, E^{n+1},
 * B^{n+1}. J holds J^{n+1/2} (filtered) on return. B is advanced in two half
 * steps around the E update, so that the particles see B at integer time (the
 * cos(k_z dt/2) factor of Eq. 3-5).
 */
void orc_step(const orc_params* p, orc_fields* F, orc_particles* P) {
  long ncell = (long)p->nx * p->ny * p->nz;
  double* G[6];
  for (int c = 0; c < 6; ++c) G[c] = (double*)malloc(sizeof(double) * ncell);
  /* 1. corrected and filtered copies of the fields seen by the particles */
  orc_gather_copies(p, F, G);
  memset(F->jx, 0, sizeof(double) * ncell);
  memset(F->jy, 0, sizeof(double) * ncell);
  memset(F->jz, 0, sizeof(double) * ncell);
  double nn[3] = {p->nx, p->ny, p->nz};
  for (long m = 0; m < P->n; ++m) {
    double x0 = P->x[m], y0 = p->ndim == 3 ? P->y[m] : 0.0, z0 = P->z[m];
    /* 2. gather at x^n */
    double f[6];
    orc_gather_point(p, G, x0, y0, z0, f);
    /* 3. Boris u^{n-1/2} -> u^{n+1/2} */
    double u[3] = {P->ux[m], P->uy[m], P->uz[m]};
    orc_boris(P->q[m], p->dt, f, f + 3, u);
    P->ux[m] = u[0];
    P->uy[m] = u[1];
    P->uz[m] = u[2];
    /* 4. move: displacement in grid units */
    double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double ddx = p->dt * u[0] / gam / p->dx;
    double ddy = p->dt * u[1] / gam / p->dy;
    double ddz = p->dt * u[2] / gam / p->dz;
    double x1 = x0 + ddx, y1 = y0 + ddy, z1 = z0 + ddz;
    /* 5. Esirkepov deposition of J^{n+1/2} */
    double qw = P->q[m] * P->w[m];
    if (p->ndim == 2) {
      orc_deposit_2d(p, F, x0, z0, ddx, ddz, u[1] / gam, qw);
    } else {
      double r0[3] = {x0, y0, z0}, dr[3] = {ddx, ddy, ddz};
      orc_deposit_3d(p, F, r0, dr, qw);
    }
    P->x[m] = wrapf(x1, nn[0]);
    if (p->ndim == 3) P->y[m] = wrapf(y1, nn[1]);
    P->z[m] = wrapf(z1, nn[2]);
  }
  /* 6. current filter */
  if (p->f_targets & 1) {
    orc_filter(p, F->jx);
    orc_filter(p, F->jy);
    orc_filter(p, F->jz);
  }
  /* 7. Yee: B half step, E full step with J, B half step */
  orc_yee_b(p, F, 0.5 * p->dt);
  orc_yee_e(p, F, p->dt);
  orc_yee_b(p, F, 0.5 * p->dt);
  for (int c = 0; c < 6; ++c) free(G[c]);
}

void orc_run(const orc_params* p, orc_fields* F, orc_particles* P, int nsteps) {
  for (int s = 0; s < nsteps; ++s) orc_step(p, F, P);
}

/* ------------------------------------------------------------------------ */
/* Diagnostics: energies (FP64)                                              */
/* ------------------------------------------------------------------------ */
/*
 * out[0] W_E = 1/2 sum E^2 dV, out[1] W_B = 1/2 sum B^2 dV,
 * out[2] W_perp = 1/2 sum (Ex^2+Ey^2+Bx^2+By^2) dV,
 * out[3] K = sum w (gamma - 1) (m = c = 1; u is at the half step),
 * out[4] W_E + W_B + K.
 */
void orc_energy(const orc_params* p, const orc_fields* F, const orc_particles* P, double out[5]) {
  long ncell = (long)p->nx * p->ny * p->nz;
  double dV = p->dx * p->dy * p->dz;
  double we = 0, wb = 0, wp = 0, k = 0;
  for (long c = 0; c < ncell; ++c) {
    double ex2 = F->ex[c] * F->ex[c], ey2 = F->ey[c] * F->ey[c], ez2 = F->ez[c] * F->ez[c];
    double bx2 = F->bx[c] * F->bx[c], by2 = F->by[c] * F->by[c], bz2 = F->bz[c] * F->bz[c];
    we += ex2 + ey2 + ez2;
    wb += bx2 + by2 + bz2;
    wp += ex2 + ey2 + bx2 + by2;
  }
  for (long m = 0; m < P->n; ++m) {
    double u2 = P->ux[m] * P->ux[m] + P->uy[m] * P->uy[m] + P->uz[m] * P->uz[m];
    k += P->w[m] * u2 / (sqrt(1.0 + u2) + 1.0); /* gamma - 1 without cancellation */
  }
  out[0] = 0.5 * we * dV;
  out[1] = 0.5 * wb * dV;
  out[2] = 0.5 * wp * dV;
  out[3] = k;
  out[4] = out[0] + out[1] + out[3];
}

/* Divergence of E at nodes (for the Gauss-law check). */
void orc_div_e(const orc_params* p, const orc_fields* F, double* out) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        long c = idx3(p, i, j, k);
        out[c] = (F->ex[c] - F->ex[idx3(p, wrap(i - 1, p->nx), j, k)]) / p->dx +
                 (F->ey[c] - F->ey[idx3(p, i, wrap(j - 1, p->ny), k)]) / p->dy +
                 (F->ez[c] - F->ez[idx3(p, i, j, wrap(k - 1, p->nz))]) / p->dz;
      }
}

/* Divergence of B at cell centres (i+1/2, j+1/2, k+1/2). */
void orc_div_b(const orc_params* p, const orc_fields* F, double* out) {
  for (int k = 0; k < p->nz; ++k)
    for (int j = 0; j < p->ny; ++j)
      for (int i = 0; i < p->nx; ++i) {
        long c = idx3(p, i, j, k);
        out[c] = (F->bx[idx3(p, wrap(i + 1, p->nx), j, k)] - F->bx[c]) / p->dx +
                 (F->by[idx3(p, i, wrap(j + 1, p->ny), k)] - F->by[c]) / p->dy +
                 (F->bz[idx3(p, i, j, wrap(k + 1, p->nz))] - F->bz[c]) / p->dz;
      }
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the beam recipe     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* Uniform on (0,1) from 32 random bits: (r + 1/2) 2^-32, exact in FP64. */
static double u01(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

typedef struct {
  int ppc;              /* lattice points per cell per species */
  double gamma;         /* drift Lorentz factor along +z */
  double omega_p_dz;    /* total (both species) plasma frequency times dz / c */
  double jitter;        /* uniform jitter half-width, cells */
  double u_th;          /* Gaussian thermal spread of each u component */
  double sigma_perp;    /* > 0: Gaussian transverse weight profile, cells (3D) */
  uint64_t seed;
} orc_beam;

/* Lattice of ppc points per cell: counts per axis, as even as possible, z last. */
void orc_lattice_dims(int ndim, int ppc, int out[3]) {
  out[0] = out[1] = out[2] = 1;
  if (ndim == 2) {
    int best = 1;
    for (int d = 1; d * d <= ppc; ++d)
      if (ppc % d == 0) best = d;
    out[0] = best;
    out[2] = ppc / best;
  } else {
    int bx = 1, by = 1;
    double bscore = 1e30;
    for (int a = 1; a <= ppc; ++a)
      for (int b = a; a * b <= ppc; ++b) {
        if (ppc % (a * b)) continue;
        int c = ppc / (a * b);
        if (c < b) continue;
        double score = (double)(c - a);
        if (score < bscore) {
          bscore = score;
          bx = a;
          by = b;
        }
      }
    out[0] = bx;
    out[1] = by;
    out[2] = ppc / (bx * by);
  }
}

/*
 * Beam initial state (the synthetic stand-in for the paper's drifting beam):
 * per cell and lattice point one electron (q = -1) and one positron (q = +1)
 * at the same jittered position (so rho = 0 and E = B = 0 is a consistent
 * start), each with its own thermal draw u = (N*u_th, N*u_th, u0 + N*u_th),
 * u0 = sqrt(gamma^2 - 1). Particle id = (cell*ppc + point)*2 + species, and
 * the arrays are filled in id order. Random numbers: Philox4x32-10 with key
 * (seed lo, seed hi) and counter (point id lo, point id hi, stream, 0);
 * stream 0 gives the jitter (outputs 0, 1, 2 for x, y, z), streams 1 and 2
 * the thermal draws of species 0 and 1 by Box-Muller on outputs (0,1), (2,3).
 * Weight w = omega_p^2 dV / (2 ppc), times exp(-r_perp^2 / (2 sigma^2)) with
 * r_perp measured from the box axis (nx/2, ny/2) when sigma_perp > 0.
 */
void orc_init_beam(const orc_params* p, const orc_beam* b, orc_particles* P) {
  int L[3];
  orc_lattice_dims(p->ndim, b->ppc, L);
  double u0 = sqrt(b->gamma * b->gamma - 1.0);
  double wp = b->omega_p_dz / p->dz;
  double w0 = wp * wp * p->dx * p->dy * p->dz / (2.0 * b->ppc);
  uint32_t key[2] = {(uint32_t)(b->seed & 0xffffffffu), (uint32_t)(b->seed >> 32)};
  long ncell = (long)p->nx * p->ny * p->nz;
  const double two_pi = 6.283185307179586476925286766559;
  for (long c = 0; c < ncell; ++c) {
    int i = (int)(c % p->nx), j = (int)((c / p->nx) % p->ny), k = (int)(c / ((long)p->nx * p->ny));
    for (int l = 0; l < b->ppc; ++l) {
      int lx = l % L[0], ly = (l / L[0]) % L[1], lz = l / (L[0] * L[1]);
      uint64_t pid = (uint64_t)c * b->ppc + l;
      uint32_t ctr[4] = {(uint32_t)(pid & 0xffffffffu), (uint32_t)(pid >> 32), 0, 0};
      uint32_t r[4];
      orc_philox4x32_10(ctr, key, r);
      double x = i + (lx + 0.5) / L[0] + b->jitter * (2.0 * u01(r[0]) - 1.0);
      double y = p->ndim == 3 ? j + (ly + 0.5) / L[1] + b->jitter * (2.0 * u01(r[1]) - 1.0) : 0.0;
      double z = k + (lz + 0.5) / L[2] + b->jitter * (2.0 * u01(r[2]) - 1.0);
      x = wrapf(x, p->nx);
      if (p->ndim == 3) y = wrapf(y, p->ny);
      z = wrapf(z, p->nz);
      double w = w0;
      if (b->sigma_perp > 0) {
        double rx = x - 0.5 * p->nx, ry = p->ndim == 3 ? y - 0.5 * p->ny : 0.0;
        w = w0 * exp(-(rx * rx + ry * ry) / (2.0 * b->sigma_perp * b->sigma_perp));
      }
      for (int s = 0; s < 2; ++s) {
        long m = (long)pid * 2 + s;
        ctr[2] = (uint32_t)(1 + s);
        orc_philox4x32_10(ctr, key, r);
        double ra = sqrt(-2.0 * log(u01(r[0]))), ta = two_pi * u01(r[1]);
        double rb = sqrt(-2.0 * log(u01(r[2]))), tb = two_pi * u01(r[3]);
        P->x[m] = x;
        if (p->ndim == 3) P->y[m] = y;
        P->z[m] = z;
        P->ux[m] = b->u_th * ra * cos(ta);
        P->uy[m] = b->u_th * ra * sin(ta);
        P->uz[m] = u0 + b->u_th * rb * cos(tb);
        P->w[m] = w;
        P->q[m] = s == 0 ? -1.0 : 1.0;
      }
    }
  }
}
