/*
 * feast_oracle.c -- plain, slow, FP64 CPU oracle for banded FEAST spectrum
 * slicing (arXiv 2012.00506, "A Parallel Direct Eigensolver for Sequences of
 * Hermitian Eigenvalue Problems with No Tridiagonalization").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every routine works in complex128 (real symmetric input is carried with zero
 * imaginary parts), except the inertia count which has separate real and
 * complex versions so that each matches its GPU counterpart operation by
 * operation.  Compile with -ffp-contract=off (no fused multiply-add).
 *
 * Storage: the Hermitian band B (order n, semi-bandwidth b) is the LAPACK lower
 * compact band, column-major: B(i,j), j <= i <= j+b, at ab[(i-j) + j*ldab].
 * Dense n x m blocks are column-major with leading dimension n.
 *
 * Parts and the passages they follow:
 *   or_inertia_*       Sylvester inertia through a pivot-free LDL^T / LDL^H of
 *                      B - sigma I (Section 3.2 "Validation and Other Details":
 *                      counts from the inertia of D - b_i I; Section 3.1).
 *   or_gauss_legendre  Gauss-Legendre rule (Section 2.2, eq. (9)-(10): the
 *                      projector is discretised by Gauss quadrature).
 *   or_contour_rule    nodes/weights on the upper half of an ellipse around
 *                      the slice; r(x) = 2 Re sum_j w_j/(z_j - x) (eq. (8)-(9)).
 *   or_band_lu/solve   shifted band LU with partial pivoting inside the band
 *                      and the solves (z_j I - B) X = Y of eq. (10).
 *   or_cholqr          Q <- Q R^{-1} with Q^H Q = R^H R (orthonormal basis for
 *                      the Rayleigh-Ritz step, Section 2.2).
 *   or_jacobi_eig      cyclic Jacobi eigensolver for the small projected
 *                      matrix A_q (Section 2.2, A_q W_q = W_q Lambda_q).
 *   or_feast_slice     Algorithm 1 (the FEAST loop) on one slice.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double re, im;
} zc;

static inline zc zmk(double re, double im) {
  zc r;
  r.re = re;
  r.im = im;
  return r;
}
static inline zc zadd(zc a, zc b) { return zmk(a.re + b.re, a.im + b.im); }
static inline zc zsub(zc a, zc b) { return zmk(a.re - b.re, a.im - b.im); }
static inline zc zmul(zc a, zc b) {
  return zmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
/* a * conj(b) */
static inline zc zmulc(zc a, zc b) {
  return zmk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
static inline zc zconj(zc a) { return zmk(a.re, -a.im); }
static inline zc zscale(zc a, double s) { return zmk(a.re * s, a.im * s); }
static inline double zabs1(zc a) { return fabs(a.re) + fabs(a.im); }
static inline double zabs(zc a) { return hypot(a.re, a.im); }
static inline double zabs2(zc a) { return a.re * a.re + a.im * a.im; }
/* a / b with Smith's scaling */
static inline zc zdiv(zc a, zc b) {
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, den = b.re + b.im * r;
    return zmk((a.re + a.im * r) / den, (a.im - a.re * r) / den);
  } else {
    double r = b.re / b.im, den = b.re * r + b.im;
    return zmk((a.re * r + a.im) / den, (a.im * r - a.re) / den);
  }
}

/* B(i,j) of the Hermitian band stored as complex lower band. */
static zc band_get(const zc* ab, int64_t ldab, int64_t b, int64_t i, int64_t j) {
  if (i >= j) {
    if (i - j > b) return zmk(0.0, 0.0);
    return ab[(i - j) + j * ldab];
  }
  if (j - i > b) return zmk(0.0, 0.0);
  return zconj(ab[(j - i) + i * ldab]);
}

/* ------------------------------------------------------------------------ */
/* Inertia.  Pivot-free right-looking LDL^T (real) / LDL^H (complex) of      */
/* B - sigma I on a working copy of the band.  The number of negative        */
/* pivots equals the number of eigenvalues below sigma (Sylvester).  A pivot */
/* that is exactly zero is replaced by -pivmin, pivmin = DBL_MIN *           */
/* max(1, amax^2), amax = max over stored entries of max(|Re|, |Im|).        */
/* ------------------------------------------------------------------------ */

double or_pivmin_real(int64_t n, int64_t b, const double* ab, int64_t ldab) {
  double amax = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t d = 0; d <= b && j + d < n; ++d) {
      double v = fabs(ab[d + j * ldab]);
      if (v > amax) amax = v;
    }
  double s = amax * amax;
  return DBL_MIN * (s > 1.0 ? s : 1.0);
}

double or_pivmin_complex(int64_t n, int64_t b, const double* abz, int64_t ldab) {
  const zc* ab = (const zc*)abz;
  double amax = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t d = 0; d <= b && j + d < n; ++d) {
      zc v = ab[d + j * ldab];
      double a = fabs(v.re), c = fabs(v.im);
      if (a > amax) amax = a;
      if (c > amax) amax = c;
    }
  double s = amax * amax;
  return DBL_MIN * (s > 1.0 ? s : 1.0);
}

/* W(i,j) for j <= i <= j+b held in a copy of the band: w[(i-j) + j*(b+1)]. */
int64_t or_inertia_real(int64_t n, int64_t b, const double* ab, int64_t ldab,
                        double sigma, double pivmin, double* dpiv) {
  const int64_t lw = b + 1;
  double* w = (double*)calloc((size_t)(n * lw), sizeof(double));
  double* l = (double*)malloc((size_t)(lw) * sizeof(double));
  if (!w || !l) {
    free(w);
    free(l);
    return -1;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t d = 0; d <= b && j + d < n; ++d) w[d + j * lw] = ab[d + j * ldab];
  for (int64_t j = 0; j < n; ++j) w[j * lw] = w[j * lw] - sigma;

  int64_t neg = 0;
  for (int64_t k = 0; k < n; ++k) {
    double d = w[k * lw];
    if (d == 0.0) d = -pivmin;
    if (d < 0.0) ++neg;
    if (dpiv) dpiv[k] = d;
    int64_t kmax = k + b < n - 1 ? k + b : n - 1;
    for (int64_t i = k + 1; i <= kmax; ++i) l[i - k] = w[(i - k) + k * lw] / d;
    for (int64_t i = k + 1; i <= kmax; ++i)
      for (int64_t j = k + 1; j <= i; ++j) {
        double a = w[(j - k) + k * lw];
        double t = l[i - k] * a;
        w[(i - j) + j * lw] = w[(i - j) + j * lw] - t;
      }
  }
  free(w);
  free(l);
  return neg;
}

int64_t or_inertia_complex(int64_t n, int64_t b, const double* abz, int64_t ldab,
                           double sigma, double pivmin, double* dpiv) {
  const zc* ab = (const zc*)abz;
  const int64_t lw = b + 1;
  zc* w = (zc*)calloc((size_t)(n * lw), sizeof(zc));
  zc* l = (zc*)malloc((size_t)(lw) * sizeof(zc));
  if (!w || !l) {
    free(w);
    free(l);
    return -1;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t d = 0; d <= b && j + d < n; ++d) w[d + j * lw] = ab[d + j * ldab];
  for (int64_t j = 0; j < n; ++j) {
    w[j * lw].re = w[j * lw].re - sigma;
    w[j * lw].im = 0.0;
  }
  int64_t neg = 0;
  for (int64_t k = 0; k < n; ++k) {
    double d = w[k * lw].re;
    if (d == 0.0) d = -pivmin;
    if (d < 0.0) ++neg;
    if (dpiv) dpiv[k] = d;
    int64_t kmax = k + b < n - 1 ? k + b : n - 1;
    for (int64_t i = k + 1; i <= kmax; ++i) {
      zc a = w[(i - k) + k * lw];
      l[i - k].re = a.re / d;
      l[i - k].im = a.im / d;
    }
    for (int64_t i = k + 1; i <= kmax; ++i)
      for (int64_t j = k + 1; j <= i; ++j) {
        zc a = w[(j - k) + k * lw];
        zc li = l[i - k];
        /* t = l_i * conj(a_jk), each product rounded, then the sum */
        double p1 = li.re * a.re;
        double p2 = li.im * a.im;
        double tre = p1 + p2;
        if (i == j) {
          w[j * lw].re = w[j * lw].re - tre;
        } else {
          double p3 = li.im * a.re;
          double p4 = li.re * a.im;
          double tim = p3 - p4;
          zc* e = &w[(i - j) + j * lw];
          e->re = e->re - tre;
          e->im = e->im - tim;
        }
      }
  }
  free(w);
  free(l);
  return neg;
}

/* Gershgorin interval [glo, ghi] containing the spectrum. */
void or_gershgorin(int64_t n, int64_t b, const double* abz, int64_t ldab, double* glo,
                   double* ghi) {
  const zc* ab = (const zc*)abz;
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double r = 0.0;
    int64_t j0 = i - b < 0 ? 0 : i - b, j1 = i + b > n - 1 ? n - 1 : i + b;
    for (int64_t j = j0; j <= j1; ++j)
      if (j != i) {
        /* |b_ij| as sqrt(re^2 + im^2) (correctly rounded square root, no FMA), summed in */
        /* ascending column order: the interval is then a fixed function of the band's bits */
        const zc v = band_get(ab, ldab, b, i, j);
        r += sqrt(v.re * v.re + v.im * v.im);
      }
    double c = ab[i * ldab].re;
    if (c - r < lo) lo = c - r;
    if (c + r > hi) hi = c + r;
  }
  *glo = lo;
  *ghi = hi;
}

/* ------------------------------------------------------------------------ */
/* Quadrature.                                                               */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes x[0..ne) (ascending) and weights on [-1, 1]: Newton */
/* iteration on P_ne evaluated by the three-term recurrence.                */
void or_gauss_legendre(int32_t ne, double* x, double* wt) {
  for (int32_t i = 0; i < ne; ++i) {
    /* i-th root counted from the right end, standard cosine initial guess */
    double t = cos(M_PI * (i + 0.75) / (ne + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      /* pk = P_ne(t), pkm1 = P_{ne-1}(t) by the three-term recurrence */
      double pk = t, pkm1 = 1.0;
      for (int32_t k = 2; k <= ne; ++k) {
        double pk1 = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
        pkm1 = pk;
        pk = pk1;
      }
      dp = ne * (t * pk - pkm1) / (t * t - 1.0);
      double dt = pk / dp;
      t -= dt;
      if (fabs(dt) <= 1e-16 * (1.0 + fabs(t))) break;
    }
    /* derivative at the converged root for the weight */
    {
      double pk = t, pkm1 = 1.0;
      for (int32_t k = 2; k <= ne; ++k) {
        double pk1 = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
        pkm1 = pk;
        pk = pk1;
      }
      dp = ne * (t * pk - pkm1) / (t * t - 1.0);
    }
    x[ne - 1 - i] = t;
    wt[ne - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

/* Upper-half ellipse rule for the slice [lo, hi]:                          */
/*   c = (lo+hi)/2, r = (hi-lo)/2, theta_k = (pi/2)(1 - x_k),               */
/*   z_k = c + r (cos theta_k + i rho sin theta_k),                          */
/*   w_k = (omega_k r / 4) (rho cos theta_k + i sin theta_k),               */
/* so that (1/(2 pi i)) of the closed contour integral of 1/(z - x) is       */
/* approximated by r(x) = 2 Re sum_k w_k / (z_k - x).                        */
void or_contour_rule(int32_t ne, double lo, double hi, double rho, double* zout,
                     double* wout) {
  double* x = (double*)malloc(sizeof(double) * ne);
  double* om = (double*)malloc(sizeof(double) * ne);
  or_gauss_legendre(ne, x, om);
  double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
  for (int32_t k = 0; k < ne; ++k) {
    double th = 0.5 * M_PI * (1.0 - x[k]);
    double ct = cos(th), st = sin(th);
    zout[2 * k] = c + r * ct;
    zout[2 * k + 1] = r * rho * st;
    wout[2 * k] = 0.25 * om[k] * r * rho * ct;
    wout[2 * k + 1] = 0.25 * om[k] * r * st;
  }
  free(x);
  free(om);
}

/* r(x) = 2 Re sum_k w_k / (z_k - x) */
double or_filter_value(int32_t ne, const double* z, const double* w, double xv) {
  zc s = zmk(0.0, 0.0);
  for (int32_t k = 0; k < ne; ++k) {
    zc zk = zmk(z[2 * k] - xv, z[2 * k + 1]);
    s = zadd(s, zdiv(zmk(w[2 * k], w[2 * k + 1]), zk));
  }
  return 2.0 * s.re;
}

/* ------------------------------------------------------------------------ */
/* Shifted band LU with partial pivoting inside the band (LAPACK gbtrf      */
/* conventions): F(i,j), -2b <= i-j <= b, at F[(2b + i - j) + j*ldf],       */
/* ldf >= 3b+1.  Pivot = first maximum of |Re| + |Im| among rows k..k+b.    */
/* Returns 0, or k+1 if the k-th pivot is exactly zero.                      */
/* ------------------------------------------------------------------------ */
#define FE(i, j) F[(2 * b + (i) - (j)) + (j)*ldf]

int64_t or_band_lu(int64_t n, int64_t b, const double* abz, int64_t ldab, double zre,
                   double zim, double* Fz, int64_t ldf, int32_t* ipiv) {
  const zc* ab = (const zc*)abz;
  zc* F = (zc*)Fz;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < ldf; ++r) F[r + j * ldf] = zmk(0.0, 0.0);
  /* F = z I - B on the band */
  for (int64_t j = 0; j < n; ++j) {
    int64_t i0 = j - b < 0 ? 0 : j - b, i1 = j + b > n - 1 ? n - 1 : j + b;
    for (int64_t i = i0; i <= i1; ++i) {
      zc v = band_get(ab, ldab, b, i, j);
      zc e = zmk(-v.re, -v.im);
      if (i == j) e = zmk(zre - v.re, zim);
      FE(i, j) = e;
    }
  }
  int64_t info = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t kmax = k + b < n - 1 ? k + b : n - 1;
    int64_t jmax = k + 2 * b < n - 1 ? k + 2 * b : n - 1;
    int64_t p = k;
    double best = zabs1(FE(k, k));
    for (int64_t i = k + 1; i <= kmax; ++i) {
      double v = zabs1(FE(i, k));
      if (v > best) {
        best = v;
        p = i;
      }
    }
    ipiv[k] = (int32_t)p;
    if (best == 0.0) {
      if (info == 0) info = k + 1;
      continue;
    }
    if (p != k)
      for (int64_t j = k; j <= jmax; ++j) {
        zc t = FE(k, j);
        FE(k, j) = FE(p, j);
        FE(p, j) = t;
      }
    zc piv = FE(k, k);
    for (int64_t i = k + 1; i <= kmax; ++i) FE(i, k) = zdiv(FE(i, k), piv);
    for (int64_t j = k + 1; j <= jmax; ++j) {
      zc ukj = FE(k, j);
      if (ukj.re == 0.0 && ukj.im == 0.0) continue;
      for (int64_t i = k + 1; i <= kmax; ++i) FE(i, j) = zsub(FE(i, j), zmul(FE(i, k), ukj));
    }
  }
  return info;
}

/* Solve (z I - B) X = Y (trans = 0) or (z I - B)^H X = Y (trans = 1) in place  */
/* on Y (n x nrhs column-major, leading dimension ldy).                         */
void or_band_solve(int64_t n, int64_t b, const double* Fz, int64_t ldf, const int32_t* ipiv,
                   int32_t trans, int64_t nrhs, double* Yz, int64_t ldy) {
  const zc* F = (const zc*)Fz;
  zc* Y = (zc*)Yz;
  for (int64_t c = 0; c < nrhs; ++c) {
    zc* y = Y + c * ldy;
    if (trans == 0) {
      for (int64_t k = 0; k < n; ++k) {
        int64_t p = ipiv[k];
        if (p != k) {
          zc t = y[k];
          y[k] = y[p];
          y[p] = t;
        }
        int64_t kmax = k + b < n - 1 ? k + b : n - 1;
        for (int64_t i = k + 1; i <= kmax; ++i) y[i] = zsub(y[i], zmul(FE(i, k), y[k]));
      }
      for (int64_t k = n - 1; k >= 0; --k) {
        zc s = y[k];
        int64_t jmax = k + 2 * b < n - 1 ? k + 2 * b : n - 1;
        for (int64_t j = k + 1; j <= jmax; ++j) s = zsub(s, zmul(FE(k, j), y[j]));
        y[k] = zdiv(s, FE(k, k));
      }
    } else {
      /* U^H w = y */
      for (int64_t k = 0; k < n; ++k) {
        zc s = y[k];
        int64_t j0 = k - 2 * b < 0 ? 0 : k - 2 * b;
        for (int64_t j = j0; j < k; ++j) s = zsub(s, zmul(zconj(FE(j, k)), y[j]));
        y[k] = zdiv(s, zconj(FE(k, k)));
      }
      /* x = P_0^T L_0^H ... P_{n-1}^T L_{n-1}^H w */
      for (int64_t k = n - 1; k >= 0; --k) {
        int64_t kmax = k + b < n - 1 ? k + b : n - 1;
        zc s = y[k];
        for (int64_t i = k + 1; i <= kmax; ++i) s = zsub(s, zmul(zconj(FE(i, k)), y[i]));
        y[k] = s;
        int64_t p = ipiv[k];
        if (p != k) {
          zc t = y[k];
          y[k] = y[p];
          y[p] = t;
        }
      }
    }
  }
}
#undef FE

/* Y = B X for the Hermitian band (lower storage), X and Y n x m column-major. */
void or_band_matvec(int64_t n, int64_t b, const double* abz, int64_t ldab, int64_t m,
                    const double* Xz, int64_t ldx, double* Yz, int64_t ldy) {
  const zc* ab = (const zc*)abz;
  const zc* X = (const zc*)Xz;
  zc* Y = (zc*)Yz;
  for (int64_t c = 0; c < m; ++c)
    for (int64_t i = 0; i < n; ++i) {
      zc s = zmk(0.0, 0.0);
      int64_t j0 = i - b < 0 ? 0 : i - b, j1 = i + b > n - 1 ? n - 1 : i + b;
      for (int64_t j = j0; j <= j1; ++j) s = zadd(s, zmul(band_get(ab, ldab, b, i, j), X[j + c * ldx]));
      Y[i + c * ldy] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* CholQR: G = Q^H Q = R^H R (R upper, positive diagonal), Q <- Q R^{-1}.    */
/* Returns 0, or j+1 if the j-th Cholesky pivot is not positive.            */
/* R (m x m column-major) is written when non-NULL.                          */
/* ------------------------------------------------------------------------ */
int64_t or_cholqr(int64_t n, int64_t m, double* Qz, int64_t ldq, double* Rz) {
  zc* Q = (zc*)Qz;
  zc* G = (zc*)calloc((size_t)(m * m), sizeof(zc));
  zc* row = (zc*)malloc(sizeof(zc) * (size_t)m);
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i <= j; ++i) {
      zc s = zmk(0.0, 0.0);
      for (int64_t k = 0; k < n; ++k) s = zadd(s, zmulc(Q[k + j * ldq], Q[k + i * ldq]));
      /* s = sum conj(q_ki) q_kj = G(i,j) */
      G[i + j * m] = s;
      G[j + i * m] = zconj(s);
    }
  /* Cholesky G = R^H R, R upper stored in G's upper triangle */
  for (int64_t j = 0; j < m; ++j) {
    double dsum = G[j + j * m].re;
    for (int64_t k = 0; k < j; ++k) dsum -= zabs2(G[k + j * m]);
    if (!(dsum > 0.0)) {
      free(G);
      free(row);
      return j + 1;
    }
    double rjj = sqrt(dsum);
    G[j + j * m] = zmk(rjj, 0.0);
    for (int64_t i = j + 1; i < m; ++i) {
      zc s = G[j + i * m];
      for (int64_t k = 0; k < j; ++k) s = zsub(s, zmul(zconj(G[k + j * m]), G[k + i * m]));
      G[j + i * m] = zscale(s, 1.0 / rjj);
    }
  }
  /* Q <- Q R^{-1}, row by row: x R = q */
  for (int64_t r = 0; r < n; ++r) {
    for (int64_t j = 0; j < m; ++j) {
      zc s = Q[r + j * ldq];
      for (int64_t k = 0; k < j; ++k) s = zsub(s, zmul(row[k], G[k + j * m]));
      row[j] = zscale(s, 1.0 / G[j + j * m].re);
    }
    for (int64_t j = 0; j < m; ++j) Q[r + j * ldq] = row[j];
  }
  if (Rz) {
    zc* R = (zc*)Rz;
    for (int64_t j = 0; j < m; ++j)
      for (int64_t i = 0; i < m; ++i) R[i + j * m] = i <= j ? G[i + j * m] : zmk(0.0, 0.0);
  }
  free(G);
  free(row);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cyclic (row-by-row) Jacobi for a dense Hermitian m x m matrix A          */
/* (column-major, overwritten).  Each rotation zeroes A(p,q): with          */
/* A(p,q) = g u, |u| = 1, the 2x2 block equals D M D^H, D = diag(u, 1),      */
/* M = [[a_pp, g], [g, a_qq]] real; M is diagonalised by the classical       */
/* real rotation [[c, s], [-s, c]], t = sgn(th)/(|th| + sqrt(th^2+1)),       */
/* th = (a_qq - a_pp)/(2g).  J = D R on rows/cols (p, q); A <- J^H A J,       */
/* V <- V J.  Sweeps stop when off(A) <= tol * ||A||_F.                     */
/* Output: eigenvalues ascending; each eigenvector scaled so that its first */
/* largest-magnitude component is real and positive.  Returns sweeps used,  */
/* or -1 if max_sweeps was reached.                                          */
/* ------------------------------------------------------------------------ */
int32_t or_jacobi_eig(int64_t m, double* Az, double* lam, double* Vz, double tol,
                      int32_t max_sweeps) {
  zc* A = (zc*)Az;
  zc* V = (zc*)Vz;
#define AE(i, j) A[(i) + (j)*m]
#define VE(i, j) V[(i) + (j)*m]
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) VE(i, j) = zmk(i == j ? 1.0 : 0.0, 0.0);
  for (int64_t i = 0; i < m; ++i) AE(i, i).im = 0.0;
  double fro = 0.0;
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) fro += zabs2(AE(i, j));
  fro = sqrt(fro);
  int32_t sweeps = 0, converged = 0;
  for (; sweeps <= max_sweeps; ++sweeps) {
    double off = 0.0;
    for (int64_t j = 0; j < m; ++j)
      for (int64_t i = 0; i < m; ++i)
        if (i != j) off += zabs2(AE(i, j));
    off = sqrt(off);
    if (off <= tol * fro || fro == 0.0) {
      converged = 1;
      break;
    }
    if (sweeps == max_sweeps) break;
    for (int64_t p = 0; p < m - 1; ++p)
      for (int64_t q = p + 1; q < m; ++q) {
        zc apq = AE(p, q);
        double g = zabs(apq);
        if (g == 0.0) continue;
        zc u = zscale(apq, 1.0 / g);
        double app = AE(p, p).re, aqq = AE(q, q).re;
        double th = (aqq - app) / (2.0 * g);
        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* columns: A <- A J, J(:,p) = (u c at p, -s at q), J(:,q) = (u s at p, c at q) */
        zc uc = zscale(u, c), us = zscale(u, s);
        for (int64_t k = 0; k < m; ++k) {
          zc akp = AE(k, p), akq = AE(k, q);
          AE(k, p) = zsub(zmul(akp, uc), zscale(akq, s));
          AE(k, q) = zadd(zmul(akp, us), zscale(akq, c));
        }
        /* rows: A <- J^H A */
        zc ucc = zconj(uc), usc = zconj(us);
        for (int64_t k = 0; k < m; ++k) {
          zc apk = AE(p, k), aqk = AE(q, k);
          AE(p, k) = zsub(zmul(ucc, apk), zscale(aqk, s));
          AE(q, k) = zadd(zmul(usc, apk), zscale(aqk, c));
        }
        AE(p, q) = zmk(0.0, 0.0);
        AE(q, p) = zmk(0.0, 0.0);
        AE(p, p).im = 0.0;
        AE(q, q).im = 0.0;
        for (int64_t k = 0; k < m; ++k) {
          zc vkp = VE(k, p), vkq = VE(k, q);
          VE(k, p) = zsub(zmul(vkp, uc), zscale(vkq, s));
          VE(k, q) = zadd(zmul(vkp, us), zscale(vkq, c));
        }
      }
  }
  /* sort ascending (selection sort, stable for equal keys by index) */
  for (int64_t i = 0; i < m; ++i) lam[i] = AE(i, i).re;
  for (int64_t i = 0; i < m; ++i) {
    int64_t k = i;
    for (int64_t j = i + 1; j < m; ++j)
      if (lam[j] < lam[k]) k = j;
    if (k != i) {
      double t = lam[i];
      lam[i] = lam[k];
      lam[k] = t;
      for (int64_t r = 0; r < m; ++r) {
        zc tv = VE(r, i);
        VE(r, i) = VE(r, k);
        VE(r, k) = tv;
      }
    }
  }
  /* phase normalisation */
  for (int64_t j = 0; j < m; ++j) {
    int64_t kbest = 0;
    double best = -1.0;
    for (int64_t r = 0; r < m; ++r) {
      double a = zabs(VE(r, j));
      if (a > best) {
        best = a;
        kbest = r;
      }
    }
    if (best > 0.0) {
      zc ph = zscale(zconj(VE(kbest, j)), 1.0 / best);
      for (int64_t r = 0; r < m; ++r) VE(r, j) = zmul(VE(r, j), ph);
      VE(kbest, j).im = 0.0;
    }
  }
#undef AE
#undef VE
  return converged ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* FEAST on one slice [lo, hi) (Algorithm 1).                               */
/*   repeat:  Q = sum_j [ w_j (z_j I - B)^{-1} Y + conj(w_j) (conj(z_j) I - B)^{-1} Y ]
 *            (real B and real Y: Q = 2 Re sum_j w_j (z_j I - B)^{-1} Y)    */
/*            Q <- orthonormal basis of Q (CholQR, applied twice)            */
/*            A_q = Q^H B Q,  A_q W = W Lambda (Jacobi),  X = Q W            */
/*            res_i = ||B x_i - lambda_i x_i|| / (bnorm ||x_i||)             */
/*            converged when `count` (the exact inertia count of the slice)  */
/*            Ritz pairs in [lo, hi) have residual <= tol; Ritz values in    */
/*            the slice with larger residual are spurious (mixtures of       */
/*            eigenvectors from both sides) and do not count;  else Y = X.   */
/* The conjugate-node solve uses (conj(z) I - B) = (z I - B)^H.             */
/* Inputs: rule z, w (ne complex), Y0 n x m0 (complex128 column-major).     */
/* Outputs: evals[m0], evecs n x m0, res[m0]: first the converged in-slice  */
/* pairs (ascending), then every other Ritz pair (ascending).               */
/* Status: 0 converged, 1 not converged in max_iter, 3 CholQR breakdown,    */
/* 7 singular shifted system.                                                */
/* ------------------------------------------------------------------------ */
int32_t or_feast_slice(int64_t n, int64_t b, const double* abz, int64_t ldab,
                       int32_t is_real, double lo, double hi, int32_t ne, const double* zr,
                       const double* wr, int64_t m0, const double* Y0z, double tol,
                       double bnorm, int32_t max_iter, int64_t count, double* evals,
                       double* evecsz, double* res, int64_t* nfound, int32_t* iters,
                       double* hist /* max_iter entries of max in-slice residual, nullable */) {
  const zc* ab = (const zc*)abz;
  const zc* z = (const zc*)zr;
  const zc* w = (const zc*)wr;
  const int64_t ldf = 3 * b + 1;
  zc* F = (zc*)malloc(sizeof(zc) * (size_t)(ldf * n));
  int32_t* ipiv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  zc* Y = (zc*)malloc(sizeof(zc) * (size_t)(n * m0));
  zc* X = (zc*)malloc(sizeof(zc) * (size_t)(n * m0));
  zc* Q = (zc*)malloc(sizeof(zc) * (size_t)(n * m0));
  zc* BQ = (zc*)malloc(sizeof(zc) * (size_t)(n * m0));
  zc* Aq = (zc*)malloc(sizeof(zc) * (size_t)(m0 * m0));
  zc* W = (zc*)malloc(sizeof(zc) * (size_t)(m0 * m0));
  double* lam = (double*)calloc((size_t)m0, sizeof(double));
  double* rr = (double*)calloc((size_t)m0, sizeof(double));
  memcpy(Y, Y0z, sizeof(zc) * (size_t)(n * m0));
  int32_t status = 1, it = 0;
  int64_t nin = 0, nconv = 0;
  for (it = 1; it <= max_iter; ++it) {
    for (int64_t e = 0; e < n * m0; ++e) Q[e] = zmk(0.0, 0.0);
    for (int32_t j = 0; j < ne; ++j) {
      if (or_band_lu(n, b, (const double*)ab, ldab, z[j].re, z[j].im, (double*)F, ldf, ipiv)) {
        status = 7;
        goto done;
      }
      memcpy(X, Y, sizeof(zc) * (size_t)(n * m0));
      or_band_solve(n, b, (const double*)F, ldf, ipiv, 0, m0, (double*)X, n);
      if (is_real) {
        for (int64_t e = 0; e < n * m0; ++e) Q[e].re += 2.0 * zmul(w[j], X[e]).re;
      } else {
        for (int64_t e = 0; e < n * m0; ++e) Q[e] = zadd(Q[e], zmul(w[j], X[e]));
        memcpy(X, Y, sizeof(zc) * (size_t)(n * m0));
        or_band_solve(n, b, (const double*)F, ldf, ipiv, 1, m0, (double*)X, n);
        for (int64_t e = 0; e < n * m0; ++e) Q[e] = zadd(Q[e], zmul(zconj(w[j]), X[e]));
      }
    }
    if (or_cholqr(n, m0, (double*)Q, n, NULL) || or_cholqr(n, m0, (double*)Q, n, NULL)) {
      status = 3;
      goto done;
    }
    or_band_matvec(n, b, (const double*)ab, ldab, m0, (const double*)Q, n, (double*)BQ, n);
    for (int64_t j = 0; j < m0; ++j)
      for (int64_t i = 0; i < m0; ++i) {
        zc s = zmk(0.0, 0.0);
        for (int64_t k = 0; k < n; ++k) s = zadd(s, zmulc(BQ[k + j * n], Q[k + i * n]));
        Aq[i + j * m0] = s;
      }
    /* symmetrise the rounding: Aq <- (Aq + Aq^H)/2 */
    for (int64_t j = 0; j < m0; ++j)
      for (int64_t i = 0; i <= j; ++i) {
        zc a = Aq[i + j * m0], c = zconj(Aq[j + i * m0]);
        zc s = zscale(zadd(a, c), 0.5);
        Aq[i + j * m0] = s;
        Aq[j + i * m0] = zconj(s);
      }
    or_jacobi_eig(m0, (double*)Aq, lam, (double*)W, 1e-14, 60);
    /* X = Q W */
    for (int64_t j = 0; j < m0; ++j)
      for (int64_t k = 0; k < n; ++k) {
        zc s = zmk(0.0, 0.0);
        for (int64_t i = 0; i < m0; ++i) s = zadd(s, zmul(Q[k + i * n], W[i + j * m0]));
        X[k + j * n] = s;
      }
    if (is_real)
      for (int64_t e = 0; e < n * m0; ++e) X[e].im = 0.0;
    /* residuals */
    or_band_matvec(n, b, (const double*)ab, ldab, m0, (const double*)X, n, (double*)BQ, n);
    nin = 0;
    nconv = 0;
    for (int64_t j = 0; j < m0; ++j) {
      double num = 0.0, den = 0.0;
      for (int64_t k = 0; k < n; ++k) {
        zc r = zsub(BQ[k + j * n], zscale(X[k + j * n], lam[j]));
        num += zabs2(r);
        den += zabs2(X[k + j * n]);
      }
      rr[j] = sqrt(num) / (bnorm * sqrt(den));
      if (lam[j] >= lo && lam[j] < hi) {
        ++nin;
        if (rr[j] <= tol) ++nconv;
      }
    }
    /* convergence measure: the count-th smallest in-slice residual */
    double worst = INFINITY;
    if (count == 0) worst = 0.0;
    for (int64_t j = 0; j < m0 && count > 0; ++j) {
      if (!(lam[j] >= lo && lam[j] < hi)) continue;
      int64_t smaller = 0;
      for (int64_t q = 0; q < m0; ++q)
        if (lam[q] >= lo && lam[q] < hi && (rr[q] < rr[j] || (rr[q] == rr[j] && q < j))) ++smaller;
      if (smaller == count - 1) worst = rr[j];
    }
    if (hist) hist[it - 1] = worst;
    memcpy(Y, X, sizeof(zc) * (size_t)(n * m0));
    if (nconv == count) {
      status = 0;
      break;
    }
  }
  if (it > max_iter) it = max_iter;
done:
  /* order: converged in-slice pairs (ascending), then all other Ritz pairs (ascending) */
  {
    int64_t pos = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int64_t j = 0; j < m0; ++j) {
        int good = lam[j] >= lo && lam[j] < hi && rr[j] <= tol;
        if ((pass == 0) != (good != 0)) continue;
        evals[pos] = lam[j];
        res[pos] = rr[j];
        memcpy(evecsz + 2 * pos * n, Y + j * n, sizeof(zc) * (size_t)n);
        ++pos;
      }
  }
  *nfound = nconv;
  *iters = it;
  free(F);
  free(ipiv);
  free(Y);
  free(X);
  free(Q);
  free(BQ);
  free(Aq);
  free(W);
  free(lam);
  free(rr);
  return status;
}
