// slicing.cu -- host-side pieces of the slicing step: the quadrature rule of
// Section 2.2 (Gauss-Legendre nodes on the upper half of an ellipse around the
// slice, eqs. (8)-(9); the trapezoid and Zolotarev rules it cites beside them), eigenvalue enclosures by batched bisection on the GPU
// inertia kernel (slice boundaries with exact counts, Section 3.2), status
// strings and option defaults.
#include <math.h>

#include <cmath>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace pdeshep {

static thread_local char g_last_error[512] = "";
static unsigned long long g_launches = 0;

void count_launch() { __atomic_add_fetch(&g_launches, 1ull, __ATOMIC_RELAXED); }
void count_launches(long long k) { __atomic_add_fetch(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
unsigned long long launches_so_far() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

void set_last_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}
void set_last_error_msg(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

// defined in inertia.cu
size_t inertia_ws_bytes(int b, int cplx, int nsigma);
int inertia_counts(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                   const double* h_sigma, int64_t* h_neg, double* d_piv, void* work, size_t wbytes,
                   cudaStream_t st, bool* nonfinite_out);
int gershgorin_device(int64_t n, int b, int cplx, const void* band, int64_t ldab, double* d_lo,
                      double* d_hi, cudaStream_t st);
size_t gershgorin_ws_doubles();

// Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton's method
// on P_ne from the three-term recurrence P_k = ((2k-1) x P_{k-1} - (k-1) P_{k-2})/k.
void gauss_legendre(int ne, double* x, double* w) {
  for (int i = 0; i < ne; ++i) {
    double t = cos(M_PI * (i + 0.75) / (ne + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = t;  // P_{k-1}, P_k
      for (int k = 2; k <= ne; ++k) {
        double p3 = ((2.0 * k - 1.0) * t * p2 - (k - 1.0) * p1) / k;
        p1 = p2;
        p2 = p3;
      }
      dp = ne * (t * p2 - p1) / (t * t - 1.0);
      double step = p2 / dp;
      t -= step;
      if (fabs(step) <= 1e-16 * (1.0 + fabs(t))) break;
    }
    double p1 = 1.0, p2 = t;
    for (int k = 2; k <= ne; ++k) {
      double p3 = ((2.0 * k - 1.0) * t * p2 - (k - 1.0) * p1) / k;
      p1 = p2;
      p2 = p3;
    }
    dp = ne * (t * p2 - p1) / (t * t - 1.0);
    x[ne - 1 - i] = t;
    w[ne - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

void contour_rule(int ne, double lo, double hi, double rho, pdeshep_c128* z, pdeshep_c128* w) {
  std::vector<double> x(ne), om(ne);
  gauss_legendre(ne, x.data(), om.data());
  const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
  for (int k = 0; k < ne; ++k) {
    const double th = 0.5 * M_PI * (1.0 - x[k]);
    const double ct = cos(th), st = sin(th);
    z[k].re = c + r * ct;
    z[k].im = r * rho * st;
    w[k].re = 0.25 * om[k] * r * rho * ct;
    w[k].im = 0.25 * om[k] * r * st;
  }
}

// Midpoint trapezoid rule on the same half ellipse (the rule of Sakurai and Sugiura that the
// paper cites beside Gauss quadrature, Section 2.2): t_k = pi (k + 1/2) / ne, weights
// (1/(2 pi i)) z'(t_k) pi/ne = (r / (2 ne)) (rho cos t_k + i sin t_k).  On a circle (rho = 1)
// the filter is 1 / (1 + ((x - c)/r)^(2 ne)) for real x.
void contour_rule_trapezoid(int ne, double lo, double hi, double rho, pdeshep_c128* z, pdeshep_c128* w) {
  const double c = 0.5 * (lo + hi), r = 0.5 * (hi - lo);
  for (int k = 0; k < ne; ++k) {
    const double th = M_PI * (k + 0.5) / ne;
    const double ct = cos(th), st = sin(th);
    z[k].re = c + r * ct;
    z[k].im = r * rho * st;
    w[k].re = r / (2.0 * ne) * rho * ct;
    w[k].im = r / (2.0 * ne) * st;
  }
}

// Zolotarev rule (the improved rational filter Section 2.2 cites after eq. (10)): Zolotarev's
// best type (2m-1, 2m) approximation of sign(x) on [-1, -ell] U [ell, 1],
//   s(x) = M x prod_{j<m} (x^2 + c_{2j}) / prod_{j<=m} (x^2 + c_{2j-1}),
//   c_i = ell^2 sc^2(i K'/(2m); ell'),   c_i c_{2m-i} = ell^2,
// composed with the Moebius map x = sqrt(ell) (lambda - lo)/(hi - lambda), sqrt(ell) = gap/(1+gap),
// gives the filter (1 + s)/2, within E/2 of the indicator of [lo, hi] wherever lambda is at least
// gap (hi - lo) from both ends.  Its poles x = +-i sqrt(c_{2j-1}) lie on the circle with diameter
// [lo, hi]; the m upper ones are the nodes and w_j = -Res, so the rule's filter is (1 + s)/2 minus
// its value at infinity (size E/2), within E of the indicator.  Elliptic functions by the AGM
// scale of Abramowitz & Stegun 16.4 / 17.6, started from the complementary modulus ell itself; the
// coefficients past c_m come from the reflection c_{2m-i} = ell^2 / c_i, so that no argument
// exceeds K'/2.  There cn >= sqrt(ell/(1+ell)) is small for small ell, and sn/cn = tan(amplitude)
// would carry a relative error of about eps K'/sqrt(ell); for ell <= 1/2 sn/cn comes from the
// nome series of the imaginary transformation instead (sc_nome below), accurate to a few ulps
// for any ell.  Products are formed as bounded ratios and the nodes as points c + r e^{i theta}
// of the circle, so that nothing overflows for ne up to 256 or |lo|, |hi| up to 1e307.  What is
// left is rounding amplified by the partial fractions at large ne and tiny ell (measured: the
// filter within E + 1e-12 for gap >= 1e-4, E + 1e-10 for gap >= 1e-6, E + 1e-9 for gap >= 1e-8,
// ne <= 256); gap is held to >= 1e-8.
namespace {

struct AgmScale {
  double a[48], c[48];
  int n;
};

// a_0 = 1, b_0 = kc, c_0 = k; c_{i+1} = c_i^2 / (4 a_{i+1}) equals (a_i - b_i)/2 without cancellation.
AgmScale agm_scale(double k, double kc) {
  AgmScale g;
  double a = 1.0, b = kc, c = k;
  g.a[0] = a;
  g.c[0] = c;
  g.n = 0;
  while (fabs(c) > 1e-17 * a && g.n < 47) {
    const double an = 0.5 * (a + b);
    const double bn = sqrt(a * b);
    c = c * c / (4.0 * an);
    a = an;
    b = bn;
    ++g.n;
    g.a[g.n] = a;
    g.c[g.n] = c;
  }
  return g;
}

// tan(am(u)) = sn/cn of modulus k by the descending amplitude recursion.
double jacobi_sc(const AgmScale& g, double u) {
  double phi = ldexp(g.a[g.n] * u, g.n);
  for (int i = g.n; i > 0; --i) phi = 0.5 * (phi + asin(g.c[i] / g.a[i] * sin(phi)));
  return tan(phi);
}

// sc(u; ell') for a small complement ell by Jacobi's imaginary transformation (A&S 16.20), sc(u; ell') =
// -i sn(iu; ell), and the nome (Fourier) series of sn (Abramowitz & Stegun 16.23.1):
//   sc(u; ell') = (2 pi / (ell K)) sum_{n>=0} q^{n+1/2} sinh((2n+1) w) / (1 - q^{2n+1}),
// K = K(ell), q = exp(-pi K'/K), w = pi u / (2K).  For 0 <= u <= K'/2 every term is positive and
// the ratio of consecutive terms is about sqrt(q) ~ ell/4, so the sum is accurate to a few ulps
// where the amplitude recursion loses eps/cn.  Each term is formed as one exponential
// e^{(n+1/2)(ln q + 2w)} (1 - e^{-2(2n+1)w})/2 / (1 - q^{2n+1}) with ln q + 2w <= ln q / 2 < 0,
// so nothing overflows.
double sc_nome(double u, double K, double lnq, double ell) {
  const double w = M_PI * u / (2.0 * K);
  double sum = 0.0;
  for (int n = 0; n < 200; ++n) {
    const double a = 2.0 * n + 1.0;
    const double t = exp((n + 0.5) * (lnq + 2.0 * w)) * (-0.5 * expm1(-2.0 * a * w)) / (-expm1(a * lnq));
    sum += t;
    if (t <= 1e-17 * sum) break;
  }
  return 2.0 * M_PI / (ell * K) * sum;
}

// s(x) / M as a product of bounded ratios: x / (x^2 + c_{2m-1}) prod_{j<m} (x^2 + c_{2j})/(x^2 + c_{2j-1}).
double zolo_shape(double x, const double* c, int m) {
  const double x2 = x * x;
  double v = x / (x2 + c[2 * m - 2]);
  for (int j = 1; j < m; ++j) v *= (x2 + c[2 * j - 1]) / (x2 + c[2 * j - 2]);
  return v;
}

}  // namespace

void contour_rule_zolotarev(int ne, double lo, double hi, double gap, pdeshep_c128* z, pdeshep_c128* w,
                            double* err) {
  const int m = ne;
  const double q = gap / (1.0 + gap);  // sqrt(ell)
  const double ell = q * q;
  const double kp = sqrt((1.0 - ell) * (1.0 + ell));
  const AgmScale g = agm_scale(kp, ell);
  const double Kp = M_PI / (2.0 * g.a[g.n]);
  std::vector<double> c(2 * m - 1);  // c[i-1] = c_i
  // sn/cn at i K'/(2m), i < m: the nome series for ell <= 1/2 (there cn at K'/2 is below 0.58 and
  // shrinks like sqrt(ell)); the amplitude recursion otherwise (its series converges slowly as
  // ell -> 1, while cn stays large).  dn = sqrt(ell^2 + ell'^2 cn^2) with cn^2 = 1/(1 + sc^2).
  const bool nome = ell <= 0.5;
  double K = 0.0, lnq = 0.0;
  if (nome) {
    const AgmScale gk = agm_scale(ell, kp);  // K(ell) = pi / (2 AGM(1, ell'))
    K = M_PI / (2.0 * gk.a[gk.n]);
    lnq = -M_PI * Kp / K;
  }
  double dn1 = q;  // dn(K'/2; ell') = sqrt(ell): the value for m = 1
  for (int i = 1; i < m; ++i) {
    const double u = i * Kp / (2.0 * m);
    const double sc = nome ? sc_nome(u, K, lnq, ell) : jacobi_sc(g, u);
    c[i - 1] = ell * sc * sc * ell;
    if (i == 1) dn1 = sqrt(ell * ell + kp * kp / (1.0 + sc * sc));
  }
  c[m - 1] = ell;  // sc^2(K'/2; ell') = 1/ell
  for (int i = m + 1; i <= 2 * m - 1; ++i) c[i - 1] = ell * ell / c[2 * m - i - 1];
  // M equalises the error at the first two equioscillation points ell and ell / dn(K'/(2m)).
  const double s0 = zolo_shape(ell, c.data(), m), s1 = zolo_shape(ell / dn1, c.data(), m);
  const double M = 2.0 / (s0 + s1);
  if (err) *err = fabs(1.0 - M * s0);
  const double cen = 0.5 * lo + 0.5 * hi, rad = 0.5 * hi - 0.5 * lo;
  for (int j = 0; j < m; ++j) {
    const double cj = c[2 * j];  // c_{2j+1}
    // Res_x s at i sqrt(cj) = (M/2) prod_{i<m} (c_{2i} - cj) / prod_{k != j} (c_{2k-1} - cj), paired:
    // even index k+1 against odd index k below j, even index k against odd index k+1 above it.
    double ratio = 1.0;
    for (int k = 0; k < j; ++k) ratio *= (c[2 * k + 1] - cj) / (c[2 * k] - cj);
    for (int k = j + 1; k < m; ++k) ratio *= (c[2 * k - 1] - cj) / (c[2 * k] - cj);
    const double res = 0.5 * M * ratio;
    // u = i y maps to lambda = (lo + hi u)/(1 + u) = c + r e^{i theta}, theta = 2 atan(1/y), and
    // -(1/2) res dlambda/dx = -(1/2) res 2r / (sqrt(ell) (1 + i y)^2) = res r sin^2(theta/2) e^{i theta}
    // / sqrt(ell): no y^2 is formed, so no overflow for wide spectra or tiny gaps.
    const double y = sqrt(cj) / q;
    const double th = 2.0 * atan2(1.0, y);
    const double ct = cos(th), st = sin(th), sh = sin(0.5 * th);
    z[j].re = cen + rad * ct;
    z[j].im = rad * st;
    const double f = rad * (res * (sh * sh / q));  // dimensionless factor first: |w| <= r
    w[j].re = f * ct;
    w[j].im = f * st;
  }
}

// Batched bisection: enclosures [lo_t, hi_t) of eigenvalue idx_t with
// count(lo) <= idx < count(hi).  Each round evaluates `fanout` interior
// points per unfinished enclosure in one inertia launch.
int bisect(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nidx, const int64_t* idx,
           double rtol, int fanout, double glo, double ghi, double* lo, double* hi, void* work,
           size_t wbytes, cudaStream_t st) {
  if (fanout < 1) fanout = 1;
  const double span = ghi - glo;
  const double pad = 1e-3 * (span > 0 ? span : 1.0) + 1e-300;
  for (int t = 0; t < nidx; ++t) {
    lo[t] = glo - pad;
    hi[t] = ghi + pad;
  }
  std::vector<double> sig;
  std::vector<int64_t> neg;
  std::vector<int> owner;
  for (int round = 0; round < 400; ++round) {
    sig.clear();
    owner.clear();
    for (int t = 0; t < nidx; ++t) {
      const double w = hi[t] - lo[t];
      if (w <= rtol * std::max(1.0, std::max(fabs(lo[t]), fabs(hi[t])))) continue;
      for (int f = 1; f <= fanout; ++f) {
        const double s = lo[t] + w * f / (fanout + 1);
        if (s <= lo[t] || s >= hi[t]) continue;
        sig.push_back(s);
        owner.push_back(t);
      }
    }
    if (sig.empty()) break;
    neg.assign(sig.size(), 0);
    if (inertia_ws_bytes(b, cplx, (int)sig.size()) > wbytes) return PDESHEP_WORKSPACE_TOO_SMALL;
    bool bad = false;
    PD_TRY(inertia_counts(n, b, cplx, band, ldab, (int)sig.size(), sig.data(), neg.data(), nullptr, work,
                          wbytes, st, &bad));
    if (bad) return PDESHEP_NONFINITE_INPUT;
    for (size_t e = 0; e < sig.size(); ++e) {
      const int t = owner[e];
      if (neg[e] <= idx[t]) {
        if (sig[e] > lo[t]) lo[t] = sig[e];
      } else {
        if (sig[e] < hi[t]) hi[t] = sig[e];
      }
    }
  }
  return 0;
}

int gershgorin_host(int64_t n, int b, int cplx, const void* band, int64_t ldab, double* glo,
                    double* ghi, void* work, size_t wbytes, cudaStream_t st) {
  if (wbytes < sizeof(double) * gershgorin_ws_doubles()) return PDESHEP_WORKSPACE_TOO_SMALL;
  double* lo = (double*)work;
  double* hi = lo + gershgorin_ws_doubles() / 2;
  PD_TRY(gershgorin_device(n, b, cplx, band, ldab, lo, hi, st));
  PD_CK(cudaMemcpyAsync(glo, lo, sizeof(double), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(ghi, hi, sizeof(double), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  return 0;
}

size_t bisect_ws_bytes(int b, int cplx, int nidx, int fanout) {
  size_t a = inertia_ws_bytes(b, cplx, std::max(1, nidx * std::max(1, fanout)));
  size_t g = sizeof(double) * gershgorin_ws_doubles();
  return std::max(a, g);
}

// ||B||_2 = max(|lambda_min|, |lambda_max|) to relative accuracy rtol.
int spectral_norm(int64_t n, int b, int cplx, const void* band, int64_t ldab, double rtol, double* out,
                  void* work, size_t wbytes, cudaStream_t st) {
  double glo, ghi;
  PD_TRY(gershgorin_host(n, b, cplx, band, ldab, &glo, &ghi, work, wbytes, st));
  int64_t idx[2] = {0, n - 1};
  double lo[2], hi[2];
  PD_TRY(bisect(n, b, cplx, band, ldab, 2, idx, rtol, 16, glo, ghi, lo, hi, work, wbytes, st));
  *out = std::max(std::max(fabs(lo[0]), fabs(hi[0])), std::max(fabs(lo[1]), fabs(hi[1])));
  return 0;
}

}  // namespace pdeshep

using namespace pdeshep;

extern "C" const char* pdeshep_last_error(void) { return g_last_error; }

extern "C" const char* pdeshep_version(void) { return "pdeshep-gb300 0.1 (sm_103a)"; }

extern "C" uint64_t pdeshep_kernel_launches(void) { return (uint64_t)launches_so_far(); }

extern "C" const char* pdeshep_status_string(int s) {
  switch (s) {
    case PDESHEP_OK: return "ok";
    case PDESHEP_NOT_CONVERGED: return "not converged";
    case PDESHEP_COUNT_MISMATCH: return "subspace smaller than the slice's eigenvalue count";
    case PDESHEP_CHOLQR_BREAKDOWN: return "CholQR breakdown";
    case PDESHEP_NONFINITE_INPUT: return "non-finite input";
    case PDESHEP_WORKSPACE_TOO_SMALL: return "workspace too small";
    case PDESHEP_DEVICE_TIMEOUT: return "device-side wait timed out";
    case PDESHEP_SINGULAR: return "singular shifted system";
    case PDESHEP_CUDA_ERROR: return "CUDA error";
    case PDESHEP_EIG_NOT_CONVERGED: return "small eigensolver did not converge";
    default: return s < 0 ? "invalid argument" : "unknown status";
  }
}

extern "C" void pdeshep_opts_default(pdeshep_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->max_iter = 20;
  o->precision = PDESHEP_MIXED;
  o->refine_policy = PDESHEP_REFINE_RESIDUAL;
  o->rhs_chunk = 0;
  o->ellipse_ratio = 0.3;
  o->bnorm = 0.0;
  o->seed = 0;
  o->hbm_cap_bytes = 0;
  o->autotune = 0;
  o->verbose = 0;
  o->stream = nullptr;
  o->rr_arith = PDESHEP_RR_TENSOR;
  o->tune_cache = nullptr;
  o->graphs = 0;
}

extern "C" int pdeshep_contour_rule(int32_t ne, double lo, double hi, double rho, pdeshep_c128* h_z,
                                    pdeshep_c128* h_w) {
  if (ne < 1 || ne > 256) return -1;
  if (!(lo < hi)) return -2;
  if (!(rho > 0.0)) return -4;
  if (!h_z) return -5;
  if (!h_w) return -6;
  contour_rule(ne, lo, hi, rho, h_z, h_w);
  return 0;
}

extern "C" int pdeshep_contour_rule_trapezoid(int32_t ne, double lo, double hi, double rho, pdeshep_c128* h_z,
                                              pdeshep_c128* h_w) {
  if (ne < 1 || ne > 256) return -1;
  if (!(lo < hi)) return -2;
  if (!(rho > 0.0)) return -4;
  if (!h_z) return -5;
  if (!h_w) return -6;
  contour_rule_trapezoid(ne, lo, hi, rho, h_z, h_w);
  return 0;
}

extern "C" int pdeshep_contour_rule_zolotarev(int32_t ne, double lo, double hi, double gap, pdeshep_c128* h_z,
                                              pdeshep_c128* h_w, double* h_err) {
  if (ne < 1 || ne > 256) return -1;
  if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) return -2;
  if (!(gap >= 1e-8) || !std::isfinite(gap)) return -4;
  if (!h_z) return -5;
  if (!h_w) return -6;
  contour_rule_zolotarev(ne, lo, hi, gap, h_z, h_w, h_err);
  return 0;
}

extern "C" size_t pdeshep_bisect_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nidx,
                                                int32_t fanout) {
  (void)n;
  return bisect_ws_bytes(b, is_complex ? 1 : 0, nidx, fanout);
}

extern "C" int pdeshep_bisect(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                              int32_t nidx, const int64_t* h_idx, double rtol, int32_t fanout, double* h_lo,
                              double* h_hi, void* d_work, size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (nidx < 0) return -6;
  if (!h_idx && nidx > 0) return -7;
  for (int t = 0; t < nidx; ++t)
    if (h_idx[t] < 0 || h_idx[t] >= n) return -7;
  if (!(rtol > 0.0)) return -8;
  if (fanout < 1 || fanout > 1024) return -9;
  if (!h_lo && nidx > 0) return -10;
  if (!h_hi && nidx > 0) return -11;
  if (!d_work) return -12;
  if (nidx == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  double glo, ghi;
  PD_TRY(gershgorin_host(n, b, is_complex ? 1 : 0, d_band, ldab, &glo, &ghi, d_work, work_bytes, st));
  return bisect(n, b, is_complex ? 1 : 0, d_band, ldab, nidx, h_idx, rtol, fanout, glo, ghi, h_lo, h_hi,
                d_work, work_bytes, st);
}
