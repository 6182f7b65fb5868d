// feast.cu -- FEAST spectrum slicing on a band matrix (Algorithm 1 of
// arXiv 2012.00506, run for every slice of step (II) of Algorithm 2).
//
// Per FEAST iteration and for all unconverged slices together:
//   filter   Q = sum_j [w_j (z_j I - B)^{-1} + conj(w_j) (conj(z_j) I - B)^{-1}] Y
//            (eqs. (9)-(10); real B: Q = 2 Re sum_j w_j (z_j I - B)^{-1} Y).  The
//            shifted factorizations of all (slice, node) pairs are a batch (the
//            paper's L1 x L2 process groups become one batch); when all factors
//            fit in the workspace they are computed once and reused by every
//            iteration, otherwise they stream through it in waves.
//   CholQR2  Q <- Q R^{-1} with Q^H Q = R^H R, twice (FP64).
//   RR       A_q = Q^H B Q, A_q W = W Lambda (FP64 Jacobi), X = Q W.
//   check    res_i = ||B x_i - lambda_i x_i|| / (||B||_2 ||x_i||); a slice is
//            done when as many Ritz pairs inside it have res_i <= tol as its
//            exact inertia count (Section 3.2).
// Precision PDESHEP_MIXED runs the filter in complex64 (FP32 accumulation).
// With PDESHEP_REFINE_RESIDUAL the filter is applied to the FP64 Ritz
// residuals r_i = B x_i - lambda_i x_i, using
//   (zI - B)^{-1} x = [x + (zI - B)^{-1} r] / (z - lambda),
// so r(B) x_i = r(lambda_i) x_i + sum_j w_j/(z_j - lambda_i) (z_j I - B)^{-1} r_i
// (+ conjugate terms): the complex64 error then scales with ||r_i|| and the
// iteration reaches FP64 residuals.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "band_lu.cuh"
#include "dense.cuh"
#include "tcgemm.cuh"

namespace pdeshep {

// from other translation units
size_t inertia_ws_bytes(int b, int cplx, int nsigma);
std::string tune_key(const char* what, int64_t n, int b, int cplx, int precision, int nsys, int max_cols);
int tune_lookup(const char* path, const std::string& key, int* value);
void tune_store(const char* path, const std::string& key, int value);
int inertia_counts_async(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                         const double* h_sigma, void* work, size_t wbytes, cudaStream_t st,
                         const int64_t** d_neg, const int** d_bad);
int inertia_counts(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                   const double* h_sigma, int64_t* h_neg, double* d_piv, void* work, size_t wbytes,
                   cudaStream_t st, bool* nonfinite_out);
void contour_rule(int ne, double lo, double hi, double rho, pdeshep_c128* z, pdeshep_c128* w);
int spectral_norm(int64_t n, int b, int cplx, const void* band, int64_t ldab, double rtol, double* out,
                  void* work, size_t wbytes, cudaStream_t st);
size_t bisect_ws_bytes(int b, int cplx, int nidx, int fanout);

// Column block of one slice in the n x sum(m0) arrays.
struct SliceDesc {
  int64_t col_off;  // first column of the slice in the internal n x M arrays
  int m0;
  int slice;
  double lo, hi;
  int64_t io_off;   // first column of the slice's block in d_x0 / d_evals / d_evecs
};

// Node range [j0, j1) of one slice inside a wave of systems.
struct AccDesc {
  int64_t col_off;
  int64_t xoff0;    // element offset of system (slice, j0)'s X^N in the X arena
  int64_t xstride;  // elements per system in the X arena
  int64_t coef_off; // offset of coef[slice][0][0]
  int m0;
  int j0, j1;
  int pad;
};

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
template <typename S, typename C>
__global__ void make_rhs_kernel(int64_t n, const SliceDesc* sd, const S* __restrict__ src,
                                const double* __restrict__ colscale, C* __restrict__ Y) {
  const SliceDesc d = sd[blockIdx.y];
  const int64_t total = n * d.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = d.col_off + e / n, i = e % n;
    const double s = colscale ? 1.0 / colscale[c] : 1.0;
    C v;
    if constexpr (std::is_same<S, double>::value) {
      v.x = (typename real_of<C>::type)(src[i + c * n] * s);
      v.y = 0;
    } else {
      const double2 a = src[i + c * n];
      v.x = (typename real_of<C>::type)(a.x * s);
      v.y = (typename real_of<C>::type)(a.y * s);
    }
    Y[i + c * n] = v;
  }
}

// Library-drawn start vectors: entry (i, c) of the slice block whose output
// column is io_off + c takes word k = (io_off + c) n + i of the SplitMix64
// stream: real bands uniform_pm1(splitmix64(seed + k)); complex bands
// re = uniform_pm1(splitmix64(seed + 2k)), im = uniform_pm1(splitmix64(seed + 2k + 1)).
template <typename S>
__global__ void random_start_kernel(int64_t n, const SliceDesc* sd, uint64_t seed, S* __restrict__ X) {
  const SliceDesc d = sd[blockIdx.y];
  const int64_t total = n * d.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    const uint64_t k = (uint64_t)((d.io_off + c) * n + i);
    if constexpr (std::is_same<S, double>::value) {
      X[i + (d.col_off + c) * n] = uniform_pm1(splitmix64(seed + k));
    } else {
      X[i + (d.col_off + c) * n] =
          make_double2(uniform_pm1(splitmix64(seed + 2 * k)), uniform_pm1(splitmix64(seed + 2 * k + 1)));
    }
  }
}

// coef[slice][j][c] and beta[c] for the columns of one slice.
// mode 0: coef = w_j (plain filter of Algorithm 1), beta = 0.
// mode 1: coef = w_j colscale_c / (z_j - lambda_c), beta = r(lambda_c).
__global__ void coef_kernel(const SliceDesc* sd, int ne, const double2* __restrict__ zw,
                            const double* __restrict__ lam, const double* __restrict__ colscale, int mode,
                            double2* __restrict__ coef, double* __restrict__ beta) {
  const SliceDesc d = sd[blockIdx.y];
  const double2* z = zw + (int64_t)d.slice * 2 * ne;
  const double2* w = z + ne;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.m0; c += gridDim.x * blockDim.x) {
    const int64_t col = d.col_off + c;
    double2* cf = coef + (int64_t)ne * d.col_off;
    if (mode == 0) {
      for (int j = 0; j < ne; ++j) cf[(int64_t)j * d.m0 + c] = w[j];
      beta[col] = 0.0;
    } else {
      const double l = lam[col], s = colscale[col];
      double r = 0.0;
      for (int j = 0; j < ne; ++j) {
        const double2 den = make_double2(z[j].x - l, z[j].y);
        const double2 q = cmul(w[j], crecip(den));  // w_j / (z_j - lambda)
        r += 2.0 * q.x;
        cf[(int64_t)j * d.m0 + c] = make_double2(q.x * s, q.y * s);
      }
      beta[col] = r;
    }
  }
}

template <typename S>
__global__ void q_init_kernel(int64_t n, const SliceDesc* sd, const double* __restrict__ beta,
                              const S* __restrict__ X, S* __restrict__ Q, int use_beta) {
  const SliceDesc d = sd[blockIdx.y];
  const int64_t total = n * d.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = d.col_off + e / n, i = e % n;
    Q[i + c * n] = use_beta ? sc<S>::scale(X[i + c * n], beta[c]) : sc<S>::zero();
  }
}

// Q[:, slice cols] += sum_{j in [j0,j1)} coef_j X_j^N (+ conj(coef_j) X_j^C), or 2 Re(.) for real B.
// The node sum runs in the precision of the solves (complex64 solves: FP32 sums, then added to the
// FP64 subspace): it only adds up FP32-class solutions, and in the refined filter it is the
// correction term, of the size of the residuals.
template <typename S, typename C>
__global__ void accumulate_kernel(int64_t n, const AccDesc* ad, const double2* __restrict__ coef,
                                  const C* __restrict__ X, S* __restrict__ Q, int cplx) {
  using R = typename real_of<C>::type;
  const AccDesc d = ad[blockIdx.y];
  const int64_t total = n * d.m0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n);
    const int64_t i = e % n;
    C acc = cmk<C>(R(0), R(0));
    for (int j = d.j0; j < d.j1; ++j) {
      const double2 cd = coef[d.coef_off + (int64_t)j * d.m0 + c];
      const C cf = cmk<C>((R)cd.x, (R)cd.y);
      const int64_t xo = d.xoff0 + (int64_t)(j - d.j0) * d.xstride + i + (int64_t)c * n;
      cfma(acc, cf, X[xo]);
      if (cplx) cfma(acc, cconj(cf), X[xo + n * (int64_t)d.m0]);
    }
    S* q = Q + i + (d.col_off + c) * n;
    if constexpr (std::is_same<S, double>::value) {
      *q += 2.0 * (double)acc.x;
    } else {
      *q = cadd(*q, make_double2((double)acc.x, (double)acc.y));
    }
  }
}

// G <- G + rel * max_i G_ii * I for each small block (shifted Cholesky)
template <typename S>
__global__ void shift_diag_kernel(const SmallDesc* desc, S* Gall, double rel) {
  const SmallDesc d = desc[blockIdx.x];
  S* G = Gall + d.off;
  __shared__ double red[32];
  double mx = 0.0;
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) mx = fmax(mx, sc<S>::re(G[i + (int64_t)i * d.m]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
    S* g = G + i + (int64_t)i * d.m;
    *g = sc<S>::from_re(sc<S>::re(*g) + rel * t);
  }
}

// A <- (A + A^H)/2 for each small block
template <typename S>
__global__ void symmetrize_kernel(const SmallDesc* desc, S* Aall) {
  const SmallDesc d = desc[blockIdx.y];
  S* A = Aall + d.off;
  const int m = d.m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), k = (int)(e / m);
    if (i > k) continue;
    const S a = A[i + (int64_t)k * m], b = sc<S>::conj(A[k + (int64_t)i * m]);
    const S v = sc<S>::scale(sc<S>::add(a, b), 0.5);
    if (i == k) {
      A[e] = sc<S>::from_re(sc<S>::re(v));
    } else {
      A[i + (int64_t)k * m] = v;
      A[k + (int64_t)i * m] = sc<S>::conj(v);
    }
  }
}

// ratio[t] = off(A)^2 / ||A - mu I||_F^2 of each small block, mu = mean of the diagonal
// (the eigenvalues of a slice's projected matrix cluster around mu)
template <typename S>
__global__ void offratio_kernel(const SmallDesc* desc, const S* Aall, double* ratio) {
  const SmallDesc d = desc[blockIdx.x];
  const S* A = Aall + d.off;
  __shared__ double s1[32], s2[32], s3[32];
  __shared__ double mu;
  double dsum = 0.0;
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) dsum += sc<S>::re(A[i + (int64_t)i * d.m]);
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
  if ((threadIdx.x & 31) == 0) s3[threadIdx.x >> 5] = dsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s3[w];
    mu = t / d.m;
  }
  __syncthreads();
  double off = 0.0, fro = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)d.m * d.m; e += blockDim.x) {
    if (e % d.m != e / d.m) {
      const double a = sc<S>::abs2(A[e]);
      off += a;
      fro += a;
    } else {
      const double a = sc<S>::re(A[e]) - mu;
      fro += a * a;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_down_sync(0xffffffffu, off, o);
    fro += __shfl_down_sync(0xffffffffu, fro, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = off;
    s2[threadIdx.x >> 5] = fro;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s1[w];
      b += s2[w];
    }
    ratio[blockIdx.x] = b > 0.0 ? a / b : 0.0;
  }
}

// R = BX - X diag(lam) (in place on BX), res = ||R||/(bnorm ||X||), colscale = ||R|| (1 if 0)
template <typename S>
__global__ void residual_kernel(int64_t n, const SliceDesc* sd, const S* __restrict__ X, S* __restrict__ BX,
                                const double* __restrict__ lam, double bnorm, double* __restrict__ res,
                                double* __restrict__ colscale) {
  const SliceDesc d = sd[blockIdx.y];
  const int c = blockIdx.x;
  if (c >= d.m0) return;
  const int64_t col = d.col_off + c;
  const double l = lam[col];
  double nr = 0.0, nx = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const S x = X[i + col * n];
    const S r = sc<S>::sub(BX[i + col * n], sc<S>::scale(x, l));
    BX[i + col * n] = r;
    nr += sc<S>::abs2(r);
    nx += sc<S>::abs2(x);
  }
  __shared__ double s1[32], s2[32];
  for (int o = 16; o > 0; o >>= 1) {
    nr += __shfl_down_sync(0xffffffffu, nr, o);
    nx += __shfl_down_sync(0xffffffffu, nx, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = nr;
    s2[threadIdx.x >> 5] = nx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += s1[w];
      b += s2[w];
    }
    const double rn = sqrt(a), xn = sqrt(b);
    res[col] = rn / (bnorm * (xn > 0.0 ? xn : 1.0));
    colscale[col] = rn > 0.0 ? rn : 1.0;
  }
}

// nconv[slice] = #{c : lo <= lam_c < hi and res_c <= tol}
__global__ void nconv_kernel(const SliceDesc* sd, const double* lam, const double* res, double tol,
                             int* nconv) {
  const SliceDesc d = sd[blockIdx.x];
  int cnt = 0;
  for (int c = threadIdx.x; c < d.m0; c += blockDim.x) {
    const double l = lam[d.col_off + c];
    cnt += (l >= d.lo && l < d.hi && res[d.col_off + c] <= tol);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  __shared__ int s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    nconv[d.slice] = t;
  }
}

// destination of each Ritz pair: converged in-slice pairs first (ascending), then the rest.
__global__ void order_kernel(const SliceDesc* sd, const double* lam, const double* res, double tol,
                             int64_t* dest) {
  const SliceDesc d = sd[blockIdx.x];
  int ngood = 0;
  for (int c = 0; c < d.m0; ++c) {
    const double l = lam[d.col_off + c];
    ngood += (l >= d.lo && l < d.hi && res[d.col_off + c] <= tol);
  }
  for (int c = threadIdx.x; c < d.m0; c += blockDim.x) {
    const double l = lam[d.col_off + c];
    const int good = (l >= d.lo && l < d.hi && res[d.col_off + c] <= tol);
    int before = 0;
    for (int c2 = 0; c2 < c; ++c2) {
      const double l2 = lam[d.col_off + c2];
      const int g2 = (l2 >= d.lo && l2 < d.hi && res[d.col_off + c2] <= tol);
      before += (g2 == good);
    }
    dest[d.col_off + c] = d.io_off + (good ? before : ngood + before);
  }
}

template <typename S>
__global__ void scatter_out_kernel(int64_t n, int64_t M, const int64_t* dest, const double* lam, const S* X,
                                   double* evals, S* evecs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * M;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    const int64_t dc = dest[c];
    evecs[i + dc * n] = X[i + c * n];
    if (i == 0) evals[dc] = lam[c];
  }
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------
static int grid1(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

struct Plan {
  // fixed buffers
  void* Xt;        // S n x M  Ritz vectors (current)
  void* Q;         // S n x M
  void* Q2;        // S n x M
  void* BQ;        // S n x M  (B Q, then B X - X Lambda)
  void* Yc;        // C n x M  filter right-hand sides
  double* lam;     // M
  double* res;     // M
  double* colscale;// M
  double* beta;    // M
  double2* coef;   // ne * M
  double2* zw;     // K * 2 * ne
  void* small_G;   // S sum m0^2 (Gram / R)
  void* small_I;   // S sum m0^2 (R^{-1}, Jacobi work)
  void* small_W;   // S sum m0^2 (eigenvectors)
  void* small_A;   // S sum m0^2 (projected matrix before the basis change)
  void* small_T;   // S sum m0^2 (temporary)
  double* offratio;// K
  GemmItem<double2>* d_items_small; // K
  void* part;      // S splits * sum m0^2
  int* info;       // K (Cholesky)
  double* minratio;// K (Cholesky conditioning indicator)
  double* diag0;   // M (Gram diagonal)
  int* sweeps;     // K
  int* sweeps32;   // K
  int* nconv;      // K
  int64_t* dest;   // M (output column of each Ritz pair)
  int* sys_status; // max systems
  double* jscratch;// K * 2 * 16
  SliceDesc* d_sd; // K
  SmallDesc* d_small; // K
  GemmItem<double2>* d_items; // 4K (storage reused for double)
  AccDesc* d_acc;  // K
  SysDesc* d_sys;  // K * ne
  char* inertia_ws;
  size_t inertia_bytes;
  void* band_ff;   // float-float copy of the band (mixed precision only)
  TcScratch tc;    // digit planes of the tensor-core products (PDESHEP_RR_TENSOR only)
  void* solve_queue; // work list of the persistent solves
  // wave area
  char* wave_base;
  size_t wave_bytes;
  int splits;
};

// CUDA-event timing of kernel groups (only when the caller asks for stats).
struct KTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> grp;
  int used = 0, cur_g = 0;
  unsigned long long cur_l0 = 0;
  double ms[PDESHEP_KG_COUNT] = {};
  long long nl[PDESHEP_KG_COUNT] = {};
  double fl[PDESHEP_KG_COUNT] = {};
  int begin(int g) {
    if (!on) return 0;
    while ((int)ev.size() < used + 2) {
      cudaEvent_t e;
      PD_CK(cudaEventCreate(&e));
      ev.push_back(e);
    }
    PD_CK(cudaEventRecord(ev[used], st));
    cur_g = g;
    cur_l0 = launches_so_far();
    return 0;
  }
  int end(double flops) {
    if (!on) return 0;
    PD_CK(cudaEventRecord(ev[used + 1], st));
    grp.push_back(cur_g);
    nl[cur_g] += (long long)(launches_so_far() - cur_l0);
    fl[cur_g] += flops;
    used += 2;
    return 0;
  }
  int collect() {
    if (!on || used == 0) return 0;
    PD_CK(cudaEventSynchronize(ev[used - 1]));
    for (int i = 0; i < used / 2; ++i) {
      float t = 0;
      PD_CK(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
      ms[grp[i]] += t;
    }
    used = 0;
    grp.clear();
    return 0;
  }
  // an interval measured elsewhere (e.g. on a side stream)
  void add(int g, double t_ms, long long launches, double flops) {
    if (!on) return;
    ms[g] += t_ms;
    nl[g] += launches;
    fl[g] += flops;
  }
  ~KTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// A non-blocking stream forked from the caller's stream by an event; `done`
// marks the end of the work enqueued on it.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t forked = nullptr, done = nullptr, t0 = nullptr, t1 = nullptr;
  int fork(cudaStream_t st) {
    PD_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    PD_CK(cudaEventCreateWithFlags(&forked, cudaEventDisableTiming));
    PD_CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    PD_CK(cudaEventCreate(&t0));
    PD_CK(cudaEventCreate(&t1));
    PD_CK(cudaEventRecord(forked, st));
    PD_CK(cudaStreamWaitEvent(s, forked, 0));
    return 0;
  }
  int join(cudaStream_t) {
    PD_CK(cudaEventRecord(done, s));
    return 0;
  }
  ~SideStream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    for (cudaEvent_t e : {forked, done, t0, t1})
      if (e) cudaEventDestroy(e);
  }
};

template <typename S, typename C>
struct Feast {
  int64_t n;
  int b, cplx, K, ne;
  const void* band;
  int64_t ldab;
  std::vector<int> m0;
  std::vector<int64_t> col_off;
  std::vector<int64_t> small_off;
  std::vector<int64_t> io_col;  // first column of each slice's block in d_x0 / d_evals / d_evecs
  int64_t M, Msq;
  int max_m0;
  const pdeshep_opts* o;
  cudaStream_t st;
  FactorGeom g;
  Plan p;
  std::vector<double> bounds;
  std::vector<pdeshep_c128> zh, wh;  // K*ne
  double bnorm;
  size_t fb, es;
  bool resident;
  bool factored;
  pdeshep_stats stats;
  std::vector<int> active;  // slice indices
  std::vector<SmallDesc> h_small;  // small-block descriptors of the active slices
  EighScratch<S> eig;
  KTimer kt;
  double cw() const { return cplx ? 8.0 : 2.0; }  // real flops per multiply-add of the FP64 subspace type

  size_t fixed_bytes(Arena& a, bool carve) {
    Plan q;
    q.Xt = a.take<S>((size_t)(n * M));
    q.Q = a.take<S>((size_t)(n * M));
    q.Q2 = a.take<S>((size_t)(n * M));
    q.BQ = a.take<S>((size_t)(n * M));
    q.Yc = a.take<C>((size_t)(n * M));
    q.lam = a.take<double>(M);
    q.res = a.take<double>(M);
    q.colscale = a.take<double>(M);
    q.beta = a.take<double>(M);
    q.coef = a.take<double2>((size_t)ne * M);
    q.zw = a.take<double2>((size_t)K * 2 * ne);
    q.small_G = a.take<S>(Msq);
    q.small_I = a.take<S>(Msq);
    q.small_W = a.take<S>(Msq);
    q.small_A = a.take<S>(Msq);
    q.small_T = a.take<S>(Msq);
    q.offratio = a.take<double>(K);
    q.d_items_small = a.take<GemmItem<double2>>(K);
    q.splits = 8;
    q.part = a.take<S>((size_t)q.splits * Msq);
    q.info = a.take<int>(K);
    q.minratio = a.take<double>(K);
    q.diag0 = a.take<double>(M);
    q.sweeps = a.take<int>(K);
    q.sweeps32 = a.take<int>(K);
    q.nconv = a.take<int>(K);
    q.dest = a.take<int64_t>(M);
    q.sys_status = a.take<int>((size_t)K * ne);
    q.jscratch = a.take<double>((size_t)K * 2 * 16);
    q.d_sd = a.take<SliceDesc>(K);
    q.d_small = a.take<SmallDesc>(K);
    q.d_items = a.take<GemmItem<double2>>((size_t)4 * K);
    q.d_acc = a.take<AccDesc>(K);
    q.d_sys = a.take<SysDesc>((size_t)K * ne);
    {
      EighScratch<S> e = plan_eigh_scratch<S>(a, Msq, M, K);
      if (carve) eig = e;
    }
    q.inertia_bytes = std::max(inertia_ws_bytes(b, cplx, K + 1), bisect_ws_bytes(b, cplx, 2, 16));
    q.inertia_ws = a.take<char>(q.inertia_bytes);
    q.band_ff = ff() && !tc() ? (void*)a.take<char>(band_split_bytes(n, b, cplx)) : nullptr;
    if (tc()) q.tc = plan_tc_scratch(a, TcShape{n, cplx, m0}, b);
    q.solve_queue = a.take<char>(solve_queue_bytes(K * ne, max_m0));
    if (carve) {
      p = q;
      eig.ff = ff();
    }
    return a.used();
  }

  // Mixed precision runs the FP64-class products of the Rayleigh-Ritz step in
  // float-float arithmetic on the FP32 pipes (band products, small m0 x m0
  // products, eigensolver refinement) and, with PDESHEP_RR_TENSOR, the tall
  // products (Gram matrix, projection, basis update) as bf16 digit products on
  // the tensor cores; plain FEAST keeps everything in FP64.
  int ff() const {
    return o->precision == PDESHEP_MIXED && o->rr_arith != PDESHEP_RR_FP64 && !rr_fp64_now ? 1 : 0;
  }
  int tc() const { return o->precision == PDESHEP_MIXED && o->rr_arith == PDESHEP_RR_TENSOR ? 1 : 0; }
  // Float-float products resolve eigenvector components down to ~1e-13 ||B|| / gap;
  // slices whose spectrum is dense enough that this stalls their residuals above the
  // tolerance are finished with FP64 products (set after kFFIterations iterations;
  // the tensor-core tall products are FP64-class already and stay).
  bool rr_fp64_now = false;
  static constexpr int kFFIterations = 3;

  // autotuned choices (see tune.cu).  Solve width of a filter pass: chunk_early, the tensor-core
  // solve (when available and measured faster than every FP32-FMA width), for the first
  // kTcIterations passes, then chunk_late, the fastest FP32-FMA solve.  The tensor core truncates
  // its FP32 accumulator at every MMA, which leaves its solves 2-3x less accurate; the refined
  // iteration contracts with the solve error, so a slice still unconverged after kTcIterations
  // passes finishes with the round-to-nearest kernels (measured on the C5 sequence: tensor-core
  // solves on every pass and on the first four give the same throughput, but the first lets single
  // steps run to 7 iterations; two or three passes are slower).  An explicit rhs_chunk serves every
  // pass.
  int rhs_chunk = 32;  // width of the current pass
  int chunk_late = 32, chunk_early = 0;
  int iter_now = 1;
  static constexpr int kTcIterations = 4;
  int pass_chunk() const { return (chunk_early && iter_now <= kTcIterations) ? chunk_early : chunk_late; }
  int gram_splits = 0;  // 0: heuristic
  bool tune_solve = false, tune_gram = false;

  // the default solve: the tensor-memory kernel for complex64 factors when its window fits
  int default_chunk() const {
    return (o->precision == PDESHEP_MIXED && solve_tm_supported(g)) ? kTmChunk : 32;
  }
  void setup_tuning() {
    if (o->rhs_chunk > 0) {
      chunk_late = o->rhs_chunk;
      chunk_early = 0;
    } else {
      chunk_late = default_chunk();
      chunk_early = (o->precision == PDESHEP_MIXED && solve_tc_supported(g)) ? kTcChunk : 0;
    }
    rhs_chunk = pass_chunk();
    if (o->autotune <= 0) return;
    int v = 0;
    if (o->rhs_chunk <= 0) {
      // the stored choice: chunk_late + 1000 if the tensor-core solve serves the first passes
      const std::string k = tune_key("solve", n, b, cplx, o->precision, K * ne, max_m0);
      if (o->autotune == 1 && tune_lookup(o->tune_cache, k, &v)) {
        chunk_late = v % 1000;
        chunk_early = v >= 1000 ? kTcChunk : 0;
        rhs_chunk = pass_chunk();
      } else {
        tune_solve = true;
      }
    }
    if (tc()) return;  // the tensor-core products choose their own split
    const std::string kg = tune_key("gram", n, b, cplx, o->precision * 2 + ff(), K, max_m0);
    if (o->autotune == 1 && tune_lookup(o->tune_cache, kg, &v))
      gram_splits = v;
    else
      tune_gram = true;
  }

  size_t per_system_bytes(int s) const {
    return fb + (((size_t)n * m0[s] * (cplx ? 2 : 1) * es + 255) & ~size_t(255));
  }
};

}  // namespace pdeshep

namespace pdeshep {

template <typename S, typename C>
struct FeastRun : Feast<S, C> {
  using B = Feast<S, C>;
  using B::n; using B::b; using B::cplx; using B::K; using B::ne; using B::band; using B::ldab;
  using B::m0; using B::col_off; using B::small_off; using B::M; using B::Msq; using B::max_m0;
  using B::o; using B::st; using B::g; using B::p; using B::bounds; using B::zh; using B::wh;
  using B::bnorm; using B::fb; using B::es; using B::resident; using B::factored; using B::stats;
  using B::active;

  std::vector<int64_t> sys_off;  // resident layout: byte offset of system s*ne+j
  std::vector<SliceDesc> h_sd;
  std::vector<int> counts, nconv, iters;
  int mode = 0;

  int upload_active() {
    const int na = (int)active.size();
    h_sd.resize(na);
    this->h_small.resize(na);
    for (int a = 0; a < na; ++a) {
      const int s = active[a];
      h_sd[a] = SliceDesc{col_off[s], m0[s], s, bounds[s], bounds[s + 1], this->io_col[s]};
      this->h_small[a] = SmallDesc{small_off[s], col_off[s], m0[s], 0};
    }
    PD_CK(cudaMemcpyAsync(p.d_sd, h_sd.data(), sizeof(SliceDesc) * na, cudaMemcpyHostToDevice, st));
    PD_CK(cudaMemcpyAsync(p.d_small, this->h_small.data(), sizeof(SmallDesc) * na, cudaMemcpyHostToDevice, st));
    return 0;
  }

  int act_max_m0() const {
    int mm = 0;
    for (int s : active) mm = std::max(mm, m0[s]);
    return mm;
  }

  // C = op(A) B over the active slices; kind 0: C(m0 x m0) = A^H B with A,B n x m0 blocks;
  // kind 1: C(n x m0) = A(n x m0) * B(m0 x m0 small block).
  int gemm(int kind, const S* A, const S* Bm, S* Cm, int tri = 0, int force_fp64 = 0, int reuse_a = 0) {
    const int na = (int)active.size();
    if (this->tc()) {
      // tensor-core digit products (FP64-class: no escalation needed)
      double fl = 0.0;
      for (int s : active) fl += this->cw() * (double)n * m0[s] * m0[s] * ((kind == 0 && A == Bm) ? 0.5 : 1.0);
      PD_TRY(this->kt.begin(PDESHEP_KG_GEMM));
      const TcShape sh{n, cplx, m0};
      std::vector<int64_t> xo(K);
      for (int t = 0; t < K; ++t) xo[t] = col_off[t] * n;
      if (kind == 0)
        PD_TRY(tc_gemm_herm<S>(p.tc, sh, active, xo, small_off, A, Bm, Cm, A == Bm, reuse_a && A != Bm, A == Bm, st));
      else
        PD_TRY(tc_gemm_update<S>(p.tc, sh, active, xo, small_off, A, Bm, Cm, st));
      return this->kt.end(fl);
    }
    std::vector<GemmItem<S>> it(na);
    for (int a = 0; a < na; ++a) {
      const int s = active[a];
      GemmItem<S> x;
      if (kind == 0) {
        x.A = A + col_off[s] * n;
        x.B = Bm + col_off[s] * n;
        x.C = Cm + small_off[s];
        x.m = m0[s];
        x.n = m0[s];
        x.k = (int)n;
        x.lda = (int)n;
        x.ldb = (int)n;
        x.ldc = m0[s];
        x.part_off = small_off[s];
      } else {
        x.A = A + col_off[s] * n;
        x.B = Bm + small_off[s];
        x.C = Cm + col_off[s] * n;
        x.m = (int)n;
        x.n = m0[s];
        x.k = m0[s];
        x.lda = (int)n;
        x.ldb = m0[s];
        x.ldc = (int)n;
        x.part_off = 0;
      }
      it[a] = x;
    }
    GemmItem<S>* d_it = (GemmItem<S>*)p.d_items;
    PD_CK(cudaMemcpyAsync(d_it, it.data(), sizeof(GemmItem<S>) * na, cudaMemcpyHostToDevice, st));
    const int mm = act_max_m0();
    S one = sc_host_one(), zero = sc_host_zero();
    double fl = 0.0;  // algorithmic: Hermitian or triangular products count half
    for (int s : active) fl += this->cw() * (double)n * m0[s] * m0[s] * ((kind == 0 || tri) ? 0.5 : 1.0);
    PD_TRY(this->kt.begin(PDESHEP_KG_GEMM));
    const int ff = this->ff() && !force_fp64;
    if (kind == 0) {
      const int64_t t1 = ceil_div(mm, ff ? 64 : 32);
      const int64_t tiles = (int64_t)na * t1 * (t1 + 1) / 2;
      int splits = (int)std::min<int64_t>(p.splits, std::max<int64_t>(1, ceil_div(8 * 152, tiles)));
      splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, n / 512));
      if (this->tune_gram) {
        cudaEvent_t e0, e1;
        PD_CK(cudaEventCreate(&e0));
        PD_CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_s = splits;
        for (int sp : {2, 4, 8}) {
          if (sp > p.splits || (int64_t)sp > std::max<int64_t>(1, n / 256)) continue;
          PD_CK(cudaEventRecord(e0, st));
          PD_TRY(launch_gemm<S>(true, na, d_it, mm, mm, (int)n, one, zero, sp, (S*)p.part, Msq, st, 1, 0, ff));
          PD_CK(cudaEventRecord(e1, st));
          PD_CK(cudaEventSynchronize(e1));
          float ms = 0;
          PD_CK(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            best_s = sp;
          }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        this->gram_splits = best_s;
        this->tune_gram = false;
        stats.tuned += 1;
        tune_store(o->tune_cache, tune_key("gram", n, b, cplx, o->precision * 2 + ff, K, max_m0), best_s);
      }
      if (this->gram_splits > 0) splits = std::min(this->gram_splits, p.splits);
      stats.gram_splits_used = splits;
      PD_TRY(launch_gemm<S>(true, na, d_it, mm, mm, (int)n, one, zero, splits, (S*)p.part, Msq, st, 1, 0, ff));
    } else {
      PD_TRY(launch_gemm<S>(false, na, d_it, (int)n, mm, mm, one, zero, 1, (S*)p.part, Msq, st, 0, tri, ff));
    }
    return this->kt.end(fl);
  }

  static S sc_host_one() {
    if constexpr (std::is_same<S, double>::value) return 1.0; else return make_double2(1.0, 0.0);
  }
  static S sc_host_zero() {
    if constexpr (std::is_same<S, double>::value) return 0.0; else return make_double2(0.0, 0.0);
  }

  int band_mm(const S* X, S* Y) {
    double fl = 0.0;
    for (int s : active) fl += this->cw() * (2.0 * b + 1.0) * (double)n * m0[s];
    PD_TRY(this->kt.begin(PDESHEP_KG_BANDMM));
    if (this->tc()) {  // tensor-core digit products (FP64-class, like the tall products: no escalation)
      std::vector<int64_t> xo(K);
      for (int t = 0; t < K; ++t) xo[t] = col_off[t] * n;
      PD_TRY(tc_band_matmul<S>(p.tc, TcShape{n, cplx, m0}, active, xo, X, Y, st));
      return this->kt.end(fl);
    }
    for (int s : active) {
      if (this->ff())
        PD_TRY(launch_band_matmul_ff<S>(n, b, p.band_ff, m0[s], X + col_off[s] * n, Y + col_off[s] * n, st));
      else
        PD_TRY(launch_band_matmul<S>(n, b, band, ldab, m0[s], X + col_off[s] * n, Y + col_off[s] * n, st));
    }
    return this->kt.end(fl);
  }

  // Gram matrix, Cholesky and R^{-1} of the active slices' blocks of p.Q (Q itself unchanged).
  // shift_rel > 0: factor G + shift_rel max_i G_ii I instead (shifted CholQR)
  // fp64_gram: the Gram matrix in FP64 arithmetic even in float-float mode
  int chol_factor(double shift_rel = 0.0, int fp64_gram = 0) {
    const int na = (int)active.size();
    S* G = (S*)p.small_G;
    S* I = (S*)p.small_I;
    double flsmall = 0.0;
    for (int s : active) flsmall += this->cw() * (double)m0[s] * m0[s] * m0[s] / 3.0;
    PD_TRY(gemm(0, (S*)p.Q, (S*)p.Q, G, 0, fp64_gram));
    PD_TRY(this->kt.begin(PDESHEP_KG_SMALL));
    if (shift_rel > 0.0) {
      shift_diag_kernel<S><<<na, 256, 0, st>>>(p.d_small, G, shift_rel);
      PD_CK_LAUNCH();
    }
    PD_TRY(launch_cholesky<S>(na, p.d_small, G, p.info, st, p.diag0, p.minratio));
    PD_TRY(launch_triinv<S>(na, p.d_small, G, I, st));
    return this->kt.end(flsmall);
  }

  int small_mm(bool conjA, S* A, S* Bm, S* Cm, int herm, int tri) {
    S* abc[3] = {A, Bm, Cm};
    double fl = 0.0;
    for (int s : active) fl += this->cw() * (double)m0[s] * m0[s] * m0[s] * ((herm || tri) ? 0.5 : 1.0);
    PD_TRY(this->kt.begin(PDESHEP_KG_SMALL));
    PD_TRY(small_gemm<S>(conjA, this->h_small, act_max_m0(), abc, herm, tri, (GemmItem<S>*)p.d_items_small, st,
                         this->ff()));
    return this->kt.end(fl);
  }

  // Rayleigh-Ritz on span(Q) for the active slices -> Xt, lam, BQ = residuals, res, colscale, nconv.
  // CholQR is fused: with Q^H Q = R^H R, the orthonormal basis Q R^{-1} is never formed;
  // A~ = R^{-H} (Q^H B Q) R^{-1}, A~ W = W Lambda, X = Q (R^{-1} W).  Slices whose columns
  // are far from orthogonal get an explicit first pass Q <- Q R1^{-1} (CholQR2).
  int rr() {
    const int na = (int)active.size();
    if (!na) return 0;
    PD_TRY(upload_active());
    const int mm = act_max_m0();
    S* G = (S*)p.small_G;
    S* I = (S*)p.small_I;
    S* W = (S*)p.small_W;
    S* Aq = (S*)p.small_A;
    S* T = (S*)p.small_T;
    // Orthonormalisation.  Every active slice gets Q^H Q = R^H R.  A slice whose
    // Cholesky breaks down is refactored with a small diagonal shift (shifted
    // CholQR); slices with a shifted factor or nearly dependent columns
    // (min_c R_cc^2 / G_cc < 1/4) get explicit passes Q <- Q R^{-1} (at most 3)
    // before the final factor, which the Rayleigh-Ritz step applies implicitly.
    const std::vector<int> keep = active;
    std::vector<int> info_s(K, 0), shifted(K, 0);
    std::vector<double> mr_s(K, 1.0);
    auto read_status = [&](const std::vector<int>& set) -> int {
      std::vector<int> info(K, 0);
      std::vector<double> mr(K, 1.0);
      PD_CK(cudaMemcpyAsync(info.data(), p.info, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
      PD_CK(cudaMemcpyAsync(mr.data(), p.minratio, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
      PD_CK(cudaStreamSynchronize(st));
      // per-slice kernel outputs are indexed by position in the batch
      for (size_t a = 0; a < set.size(); ++a) {
        info_s[set[a]] = info[a];
        mr_s[set[a]] = mr[a];
      }
      return 0;
    };
    PD_TRY(chol_factor());
    PD_TRY(read_status(active));
    // Float-float Gram entries carry ~1e-13 relative error, which enters R through
    // cond(Q)^2: an explicit pass still repairs a basis of condition up to ~1e6, but
    // beyond that the Cholesky factor breaks down.  Slices whose float-float Gram
    // breaks down get their Gram matrices in FP64 for the rest of this
    // orthonormalisation (a shift below 1e-13 would not help there).
    std::vector<int> gram64(K, 0);
    if (this->ff() && !this->tc()) {
      std::vector<int> ill;
      for (int s : keep)
        if (info_s[s]) {
          ill.push_back(s);
          gram64[s] = 1;
        }
      if (!ill.empty()) {
        active = ill;
        PD_TRY(upload_active());
        PD_TRY(chol_factor(0.0, 1));
        PD_TRY(read_status(active));
        stats.gram_fp64 += (int)ill.size();
      }
    }
    auto any64 = [&](const std::vector<int>& set) {
      for (int s : set)
        if (gram64[s]) return 1;
      return 0;
    };
    const double shift_rel = 1e-14;
    for (int pass = 0;; ++pass) {
      std::vector<int> bad, again;
      for (int s : keep) {
        if (info_s[s])
          bad.push_back(s);
        else if (mr_s[s] < 0.25 || shifted[s] == 1)
          again.push_back(s);
      }
      if (!bad.empty()) {
        for (int s : bad) {
          if (shifted[s] || pass >= 3) return PDESHEP_CHOLQR_BREAKDOWN;
          shifted[s] = 1;
        }
        active = bad;
        PD_TRY(upload_active());
        PD_TRY(chol_factor(shift_rel, any64(bad)));
        PD_TRY(read_status(active));
        for (int s : bad) {
          if (info_s[s]) return PDESHEP_CHOLQR_BREAKDOWN;
          again.push_back(s);
        }
        stats.cholqr_shifted += (int)bad.size();
      }
      if (again.empty() || pass >= 3) break;
      active = again;
      PD_TRY(upload_active());
      PD_TRY(gemm(1, (S*)p.Q, I, (S*)p.Q2, 1));   // Q R^{-1}
      for (int s : active)
        PD_CK(cudaMemcpyAsync((S*)p.Q + col_off[s] * n, (S*)p.Q2 + col_off[s] * n, sizeof(S) * n * m0[s],
                              cudaMemcpyDeviceToDevice, st));
      PD_TRY(chol_factor(0.0, any64(again)));
      PD_TRY(read_status(active));
      for (int s : again) shifted[s] = shifted[s] ? 2 : 0;  // a shifted slice had its explicit pass
    }
    active = keep;
    PD_TRY(upload_active());
    PD_TRY(band_mm((S*)p.Q, (S*)p.BQ));
    PD_TRY(gemm(0, (S*)p.Q, (S*)p.BQ, Aq, 0, 0, 1));  // Q^H B Q (Q's digits from its last Gram matrix)
    PD_TRY(small_mm(false, Aq, I, T, 0, 1));         // (Q^H B Q) R^{-1}
    PD_TRY(small_mm(true, I, T, G, 1, 0));           // A~ = R^{-H} (Q^H B Q) R^{-1}
    PD_TRY(this->kt.begin(PDESHEP_KG_EIG));
    symmetrize_kernel<S><<<dim3(grid1((int64_t)mm * mm), na), 256, 0, st>>>(p.d_small, G);
    PD_CK_LAUNCH();
    offratio_kernel<S><<<na, 256, 0, st>>>(p.d_small, G, p.offratio);
    PD_CK_LAUNCH();
    std::vector<double> orat(K, 1.0);
    PD_CK(cudaMemcpyAsync(orat.data(), p.offratio, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    std::vector<unsigned char> fp32(na);
    for (int a = 0; a < na; ++a) fp32[a] = orat[a] > 1e-6 ? 1 : 0;  // off(A~) > 1e-3 ||A~||_F
    PD_CK(cudaMemsetAsync(p.sweeps32, 0, sizeof(int) * K, st));
    EighReport rep;
    PD_TRY(eigh_mixed<S>(na, p.d_small, this->h_small.data(), mm, G, p.lam, W, this->eig, st, p.sweeps,
                         fp32.data(), p.sweeps32, &rep));
    stats.eig_refine_steps += rep.refine_steps;
    stats.eig_clusters += rep.clusters;
    stats.eig_max_cluster = std::max(stats.eig_max_cluster, rep.max_cluster);
    stats.eig_fallback_unconverged += rep.fallback_unconverged;
    stats.eig_fallback_wide += rep.fallback_wide;
    PD_TRY(this->kt.end(0.0));
    PD_TRY(small_mm(false, I, W, T, 0, 0));          // R^{-1} W
    PD_TRY(gemm(1, (S*)p.Q, T, (S*)p.Xt));           // X = Q R^{-1} W
    PD_TRY(band_mm((S*)p.Xt, (S*)p.BQ));
    PD_TRY(this->kt.begin(PDESHEP_KG_BANDMM));
    residual_kernel<S><<<dim3(mm, na), 256, 0, st>>>(n, p.d_sd, (S*)p.Xt, (S*)p.BQ, p.lam, bnorm, p.res,
                                                     p.colscale);
    PD_CK_LAUNCH();
    PD_TRY(this->kt.end(0.0));
    nconv_kernel<<<na, 256, 0, st>>>(p.d_sd, p.lam, p.res, o->tol, p.nconv);
    PD_CK_LAUNCH();
    std::vector<int> sw(K, 0), sw32(K, 0);
    PD_CK(cudaMemcpyAsync(nconv.data(), p.nconv, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(sw.data(), p.sweeps, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(sw32.data(), p.sweeps32, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    int mx64 = 0, mx32 = 0;
    for (int a = 0; a < na; ++a) {
      if (sw[a] < 0) return PDESHEP_EIG_NOT_CONVERGED;
      mx64 = std::max(mx64, sw[a]);
      mx32 = std::max(mx32, sw32[a] < 0 ? 20 : sw32[a]);
    }
    stats.jacobi_sweeps64 += mx64;
    stats.jacobi_sweeps32 += mx32;
    stats.rr_calls += 1;
    return this->kt.collect();
  }

  SysDesc sys_desc(int s, int j, int64_t off) const {
    SysDesc d;
    d.factor_off = off;
    d.zre = zh[(size_t)s * ne + j].re;
    d.zim = zh[(size_t)s * ne + j].im;
    d.rhs_off = col_off[s] * n;
    d.out_off = (off + (int64_t)fb) / (int64_t)es;
    d.out2_off = d.out_off + n * m0[s];
    d.ncols = m0[s];
    d.pad = 0;
    return d;
  }

  int factor_batch(const std::vector<SysDesc>& sd) {
    const int ns = (int)sd.size();
    if (!ns) return 0;
    PD_CK(cudaMemcpyAsync(p.d_sys, sd.data(), sizeof(SysDesc) * ns, cudaMemcpyHostToDevice, st));
    PD_TRY(this->kt.begin(PDESHEP_KG_FACTOR));
    PD_TRY(launch_factor<C>(g, cplx, band, ldab, ns, p.d_sys, p.wave_base, p.sys_status, nullptr, st));
    PD_TRY(this->kt.end(16.0 * ns * (double)n * b * b));
    std::vector<int> status(ns, 0);
    PD_CK(cudaMemcpyAsync(status.data(), p.sys_status, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    for (int v : status)
      if (v) return PDESHEP_SINGULAR;
    stats.factorizations += ns;
    return 0;
  }

  int solve_and_accumulate(const std::vector<SysDesc>& sd, const std::vector<AccDesc>& acc) {
    const int ns = (int)sd.size();
    if (!ns) return 0;
    int mcols = 0;
    for (auto& d : sd) mcols = std::max(mcols, d.ncols);
    PD_CK(cudaMemcpyAsync(p.d_sys, sd.data(), sizeof(SysDesc) * ns, cudaMemcpyHostToDevice, st));
    double cols = 0.0;
    for (auto& d : sd) cols += d.ncols;
    PD_TRY(this->kt.begin(PDESHEP_KG_SOLVE));
    if (this->tune_solve) {
      // time the forward solves at each column block on these very systems
      // (each run rewrites the same outputs) and keep the fastest
      cudaEvent_t t0, t1;
      PD_CK(cudaEventCreate(&t0));
      PD_CK(cudaEventCreate(&t1));
      float best = 1e30f, t_tc = 1e30f;
      int best_cw = this->default_chunk();
      for (int cw : {16, 32, 64, kTmChunk, kTcChunk}) {
        if (cw == kTmChunk   ? !(sizeof(C) == sizeof(float2) && solve_tm_supported(g))
            : cw == kTcChunk ? !(sizeof(C) == sizeof(float2) && solve_tc_supported(g))
                             : solve_smem_bytes(g, cw, sizeof(C), 0) > 227 * 1024)
          continue;
        PD_CK(cudaEventRecord(t0, st));
        PD_TRY(launch_solve<C>(g, 0, ns, sd.data(), p.d_sys, p.wave_base, (const C*)p.Yc, (C*)p.wave_base, cw,
                               p.solve_queue, st));
        PD_CK(cudaEventRecord(t1, st));
        PD_CK(cudaEventSynchronize(t1));
        float ms = 0;
        PD_CK(cudaEventElapsedTime(&ms, t0, t1));
        if (cw == kTcChunk) {
          t_tc = ms;
        } else if (ms < best) {
          best = ms;
          best_cw = cw;
        }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      this->chunk_late = best_cw;
      this->chunk_early = t_tc < best ? kTcChunk : 0;
      this->rhs_chunk = this->pass_chunk();
      this->tune_solve = false;
      stats.tuned += 1;
      tune_store(o->tune_cache, tune_key("solve", n, b, cplx, o->precision, K * ne, max_m0),
                 this->chunk_late + (this->chunk_early ? 1000 : 0));
    }
    const int chunk = this->rhs_chunk;
    stats.rhs_chunk_early = this->chunk_early;
    stats.rhs_chunk_used = chunk;
    PD_TRY(launch_solve<C>(g, 0, ns, sd.data(), p.d_sys, p.wave_base, (const C*)p.Yc, (C*)p.wave_base, chunk,
                           p.solve_queue, st));
    if (cplx)
      PD_TRY(launch_solve<C>(g, 1, ns, sd.data(), p.d_sys, p.wave_base, (const C*)p.Yc, (C*)p.wave_base, chunk,
                             p.solve_queue, st));
    PD_TRY(this->kt.end(24.0 * (double)n * b * cols * (cplx ? 2 : 1)));
    for (auto& d : sd) stats.rhs_sweeps += ceil_div(d.ncols, 32) * (cplx ? 2 : 1);
    stats.rhs_columns += (int64_t)cols * (cplx ? 2 : 1);
    const int na = (int)acc.size();
    PD_CK(cudaMemcpyAsync(p.d_acc, acc.data(), sizeof(AccDesc) * na, cudaMemcpyHostToDevice, st));
    PD_TRY(this->kt.begin(PDESHEP_KG_ACCUM));
    accumulate_kernel<S, C><<<dim3(grid1(n * mcols), na), 256, 0, st>>>(n, p.d_acc, p.coef,
                                                                       (const C*)p.wave_base, (S*)p.Q, cplx);
    PD_CK_LAUNCH();
    return this->kt.end(8.0 * (double)n * cols * (cplx ? 2 : 1));
  }

  // systems and accumulation descriptors of the active slices (resident factors)
  void resident_descs(std::vector<SysDesc>& sd, std::vector<AccDesc>& acc) const {
    sd.clear();
    acc.clear();
    for (int s : active) {
      for (int j = 0; j < ne; ++j) sd.push_back(sys_desc(s, j, sys_off[(size_t)s * ne + j]));
      AccDesc a;
      a.col_off = col_off[s];
      a.xoff0 = sd[sd.size() - ne].out_off;
      a.xstride = (ne > 1) ? (sd[sd.size() - ne + 1].out_off - sd[sd.size() - ne].out_off) : 0;
      a.coef_off = (int64_t)ne * col_off[s];
      a.m0 = m0[s];
      a.j0 = 0;
      a.j1 = ne;
      a.pad = 0;
      acc.push_back(a);
    }
  }

  // CUDA graphs of the filter pass, one per (active slices, mode)
  struct FilterGraph {
    std::vector<int> active;
    int mode, chunk;
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::vector<FilterGraph> fgraphs;
  ~FeastRun() {
    for (auto& f : fgraphs) cudaGraphExecDestroy(f.exec);
  }
  bool graph_ready() const {
    return o->graphs && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread && resident &&
           factored && !this->tune_solve;
  }

  // the filter launches after the descriptors are on the device
  int filter_launches(int na, int mm, int nitems) {
    const S* src = mode ? (const S*)p.BQ : (const S*)p.Xt;
    make_rhs_kernel<S, C><<<dim3(grid1(n * mm), na), 256, 0, st>>>(n, p.d_sd, src, mode ? p.colscale : nullptr,
                                                                  (C*)p.Yc);
    PD_CK_LAUNCH();
    coef_kernel<<<dim3((unsigned)ceil_div(mm, 128), na), 128, 0, st>>>(p.d_sd, ne, p.zw, p.lam, p.colscale,
                                                                       mode, p.coef, p.beta);
    PD_CK_LAUNCH();
    q_init_kernel<S><<<dim3(grid1(n * mm), na), 256, 0, st>>>(n, p.d_sd, p.beta, (const S*)p.Xt, (S*)p.Q, mode);
    PD_CK_LAUNCH();
    PD_TRY(launch_solve_queued<C>(g, 0, nitems, p.d_sys, p.wave_base, (const C*)p.Yc, (C*)p.wave_base,
                                  this->rhs_chunk, p.solve_queue, st));
    if (cplx)
      PD_TRY(launch_solve_queued<C>(g, 1, nitems, p.d_sys, p.wave_base, (const C*)p.Yc, (C*)p.wave_base,
                                    this->rhs_chunk, p.solve_queue, st));
    accumulate_kernel<S, C><<<dim3(grid1(n * mm), na), 256, 0, st>>>(n, p.d_acc, p.coef, (const C*)p.wave_base,
                                                                      (S*)p.Q, cplx);
    PD_CK_LAUNCH();
    return 0;
  }

  // the filter pass replayed from a CUDA graph (resident factors)
  int filter_graph() {
    const int na = (int)active.size();
    PD_TRY(upload_active());
    const int mm = act_max_m0();
    std::vector<SysDesc> sd;
    std::vector<AccDesc> acc;
    resident_descs(sd, acc);
    PD_CK(cudaMemcpyAsync(p.d_sys, sd.data(), sizeof(SysDesc) * sd.size(), cudaMemcpyHostToDevice, st));
    PD_CK(cudaMemcpyAsync(p.d_acc, acc.data(), sizeof(AccDesc) * acc.size(), cudaMemcpyHostToDevice, st));
    int nitems = 0;
    PD_TRY(upload_solve_items((int)sd.size(), sd.data(), this->rhs_chunk, p.solve_queue, st, &nitems));
    FilterGraph* fg = nullptr;
    for (auto& f : fgraphs)
      if (f.mode == mode && f.active == active && f.chunk == this->rhs_chunk) fg = &f;
    if (!fg) {
      const unsigned long long l0 = launches_so_far();
      cudaGraph_t graph;
      PD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      const int r = filter_launches(na, mm, nitems);
      const cudaError_t ec = cudaStreamEndCapture(st, &graph);
      if (r) return r;
      PD_CK(ec);
      FilterGraph f;
      f.active = active;
      f.mode = mode;
      f.chunk = this->rhs_chunk;
      f.kernels = (long long)(launches_so_far() - l0);
      count_launches(-f.kernels);  // counted when they run
      const cudaError_t ei = cudaGraphInstantiate(&f.exec, graph, 0);
      cudaGraphDestroy(graph);
      PD_CK(ei);
      fgraphs.push_back(f);
      fg = &fgraphs.back();
    }
    double cols = 0.0;
    for (auto& d : sd) cols += d.ncols;
    PD_TRY(this->kt.begin(PDESHEP_KG_SOLVE));
    PD_CK(cudaGraphLaunch(fg->exec, st));
    count_launches(fg->kernels);
    PD_TRY(this->kt.end(24.0 * (double)n * b * cols * (cplx ? 2 : 1)));
    for (auto& d : sd) stats.rhs_sweeps += ceil_div(d.ncols, this->rhs_chunk) * (cplx ? 2 : 1);
    stats.rhs_columns += (int64_t)cols * (cplx ? 2 : 1);
    stats.rhs_chunk_used = this->rhs_chunk;
    stats.rhs_chunk_early = this->chunk_early;
    stats.graph_launches += 1;
    return 0;
  }

  // Q = filter(Xt or residuals) for the active slices
  int filter() {
    const int na = (int)active.size();
    if (!na) return 0;
    if (!this->tune_solve) this->rhs_chunk = this->pass_chunk();
    if (graph_ready()) return filter_graph();
    PD_TRY(upload_active());
    const int mm = act_max_m0();
    const S* src = mode ? (const S*)p.BQ : (const S*)p.Xt;
    PD_TRY(this->kt.begin(PDESHEP_KG_ACCUM));
    make_rhs_kernel<S, C><<<dim3(grid1(n * mm), na), 256, 0, st>>>(n, p.d_sd, src, mode ? p.colscale : nullptr,
                                                                  (C*)p.Yc);
    PD_CK_LAUNCH();
    coef_kernel<<<dim3((unsigned)ceil_div(mm, 128), na), 128, 0, st>>>(p.d_sd, ne, p.zw, p.lam, p.colscale,
                                                                       mode, p.coef, p.beta);
    PD_CK_LAUNCH();
    q_init_kernel<S><<<dim3(grid1(n * mm), na), 256, 0, st>>>(n, p.d_sd, p.beta, (const S*)p.Xt, (S*)p.Q, mode);
    PD_CK_LAUNCH();
    PD_TRY(this->kt.end(0.0));
    if (resident) {
      if (!factored) {
        std::vector<SysDesc> all;
        for (int s = 0; s < K; ++s)
          for (int j = 0; j < ne; ++j) all.push_back(sys_desc(s, j, sys_off[(size_t)s * ne + j]));
        PD_TRY(factor_batch(all));
        factored = true;
        stats.waves += 1;
      }
      std::vector<SysDesc> sd;
      std::vector<AccDesc> acc;
      resident_descs(sd, acc);
      return solve_and_accumulate(sd, acc);
    }
    // streaming waves: systems of the active slices packed while they fit
    size_t used = 0;
    std::vector<SysDesc> sd;
    std::vector<AccDesc> acc;
    auto flush = [&]() -> int {
      if (sd.empty()) return 0;
      PD_TRY(factor_batch(sd));
      PD_TRY(solve_and_accumulate(sd, acc));
      stats.waves += 1;
      sd.clear();
      acc.clear();
      used = 0;
      return 0;
    };
    for (int s : active) {
      const size_t ps = this->per_system_bytes(s);
      for (int j = 0; j < ne; ++j) {
        if (used + ps > p.wave_bytes) PD_TRY(flush());
        if (ps > p.wave_bytes) return PDESHEP_WORKSPACE_TOO_SMALL;
        sd.push_back(sys_desc(s, j, (int64_t)used));
        used += ps;
        if (acc.empty() || acc.back().col_off != col_off[s] || acc.back().j1 != j) {
          AccDesc a;
          a.col_off = col_off[s];
          a.xoff0 = sd.back().out_off;
          a.xstride = (int64_t)(ps / es);
          a.coef_off = (int64_t)ne * col_off[s];
          a.m0 = m0[s];
          a.j0 = j;
          a.j1 = j + 1;
          a.pad = 0;
          acc.push_back(a);
        } else {
          acc.back().j1 = j + 1;
        }
      }
    }
    return flush();
  }
};

}  // namespace pdeshep

using namespace pdeshep;

namespace {

// One batch of slices whose factors are planned together (all resident in the
// workspace, or streamed in waves when they do not fit).  h_io_col[s]: first
// column of slice s's block in d_x0 / d_evals / d_evecs (NULL: packed by m0).
// h_known_neg: exact counts below h_bounds[0..K] when the caller already has
// them (NULL: counted here on a side stream beside the first filter pass).
template <typename S, typename C>
int feast_entry(int64_t n, int b, int cplx, const void* band, int64_t ldab, int K, const double* h_bounds,
                int ne, const pdeshep_c128* h_nodes, const pdeshep_c128* h_weights, const int32_t* h_m0,
                const int64_t* h_io_col, const int64_t* h_known_neg,
                const void* d_x0, void* d_work, size_t work_bytes, const pdeshep_opts* o, double* d_evals,
                void* d_evecs, int32_t* h_counts, int32_t* h_nfound, pdeshep_stats* h_stats, size_t* size_only) {
  FeastRun<S, C> F;
  F.n = n;
  F.b = b;
  F.cplx = cplx;
  F.K = K;
  F.ne = ne;
  F.band = band;
  F.ldab = ldab;
  F.o = o;
  F.st = (cudaStream_t)o->stream;
  F.g = make_geom(n, b);
  F.es = sizeof(C);
  F.fb = factor_bytes(F.g, sizeof(C));
  F.kt.on = (h_stats != nullptr);
  F.kt.st = (cudaStream_t)o->stream;
  F.m0.assign(h_m0, h_m0 + K);
  F.col_off.assign(K, 0);
  F.small_off.assign(K, 0);
  int64_t acc = 0, accs = 0;
  F.max_m0 = 0;
  for (int s = 0; s < K; ++s) {
    F.col_off[s] = acc;
    F.small_off[s] = accs;
    acc += F.m0[s];
    accs += (int64_t)F.m0[s] * F.m0[s];
    F.max_m0 = std::max(F.max_m0, F.m0[s]);
  }
  F.M = acc;
  F.Msq = accs;
  F.io_col = h_io_col ? std::vector<int64_t>(h_io_col, h_io_col + K) : F.col_off;
  memset(&F.stats, 0, sizeof(F.stats));
  F.setup_tuning();
  // workspace plan
  Arena a(d_work, work_bytes);
  F.fixed_bytes(a, true);
  const size_t fixed = a.used();
  size_t all_sys = 0;
  F.sys_off.assign((size_t)K * ne, 0);
  for (int s = 0; s < K; ++s)
    for (int j = 0; j < ne; ++j) {
      F.sys_off[(size_t)s * ne + j] = (int64_t)all_sys;
      all_sys += F.per_system_bytes(s);
    }
  size_t max_sys = 0;
  for (int s = 0; s < K; ++s) max_sys = std::max(max_sys, F.per_system_bytes(s));
  if (size_only) {
    size_t wave = all_sys;
    if (o->hbm_cap_bytes > 0) wave = std::min(wave, std::max((size_t)o->hbm_cap_bytes, max_sys));
    *size_only = fixed + wave + 256;
    return 0;
  }
  if (work_bytes < fixed + max_sys) return PDESHEP_WORKSPACE_TOO_SMALL;
  F.p.wave_base = (char*)d_work + fixed;
  F.p.wave_bytes = work_bytes - fixed;
  if (o->hbm_cap_bytes > 0) F.p.wave_bytes = std::min(F.p.wave_bytes, (size_t)o->hbm_cap_bytes);
  F.resident = all_sys <= F.p.wave_bytes;
  F.factored = false;
  cudaStream_t st = F.st;
  if (F.tc()) PD_TRY(tc_clear_error(F.p.tc, st));
  if (o->precision == PDESHEP_MIXED) PD_TRY(solve_tc_error(nullptr, 1, st));

  cudaEvent_t e0, e1;
  PD_CK(cudaEventCreate(&e0));
  PD_CK(cudaEventCreate(&e1));
  PD_CK(cudaEventRecord(e0, st));
  F.bounds.assign(h_bounds, h_bounds + K + 1);
  // ||B||_2 (synchronous; uses the inertia workspace before the counts do)
  F.bnorm = o->bnorm;
  if (!(F.bnorm > 0.0))
    PD_TRY(spectral_norm(n, b, cplx, band, ldab, 1e-6, &F.bnorm, F.p.inertia_ws, F.p.inertia_bytes, st));
  // Exact counts by inertia at every boundary (Section 3.2).  The LDL^T sweeps
  // occupy one SM per boundary, so they run on a side stream next to the first
  // two filter passes and are read back with the second Rayleigh-Ritz results (or
  // the first, when max_iter is 1); a slice whose subspace is smaller than its
  // count is reported then.
  SideStream side;
  const int64_t* d_neg = nullptr;
  const int* d_bad = nullptr;
  if (!h_known_neg) {
    PD_TRY(side.fork(st));
    PD_CK(cudaEventRecord(side.t0, side.s));
    PD_TRY(inertia_counts_async(n, b, cplx, band, ldab, K + 1, h_bounds, F.p.inertia_ws, F.p.inertia_bytes,
                                side.s, &d_neg, &d_bad));
    PD_CK(cudaEventRecord(side.t1, side.s));
    PD_TRY(side.join(st));
  }
  const long long inertia_launches = 2;
  if (F.ff()) {
    PD_TRY(F.kt.begin(PDESHEP_KG_BANDMM));
    if (F.tc())
      PD_TRY(tc_band_split<S>(F.p.tc, n, b, band, ldab, st));
    else
      PD_TRY(launch_band_split<S>(n, b, band, ldab, F.p.band_ff, st));
    PD_TRY(F.kt.end(0.0));
  }
  F.counts.assign(K, 0);
  F.nconv.assign(K, 0);
  F.iters.assign(K, 0);
  bool counts_ready = false;
  auto read_counts = [&]() -> int {
    if (counts_ready) return 0;
    if (h_known_neg) {
      counts_ready = true;
      for (int s = 0; s < K; ++s) {
        F.counts[s] = (int)(h_known_neg[s + 1] - h_known_neg[s]);
        if (h_counts) h_counts[s] = F.counts[s];
      }
      for (int s = 0; s < K; ++s)
        if (F.m0[s] < F.counts[s]) return PDESHEP_COUNT_MISMATCH;
      return 0;
    }
    std::vector<int64_t> neg(K + 1);
    int bad = 0;
    PD_CK(cudaStreamWaitEvent(st, side.done, 0));
    PD_CK(cudaMemcpyAsync(neg.data(), d_neg, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    counts_ready = true;
    float ms = 0;
    PD_CK(cudaEventElapsedTime(&ms, side.t0, side.t1));
    F.stats.ms_inertia = ms;
    F.kt.add(PDESHEP_KG_INERTIA, ms, inertia_launches, (K + 1) * (double)n * b * b * (cplx ? 4.0 : 1.0));
    if (bad) return PDESHEP_NONFINITE_INPUT;
    for (int s = 0; s < K; ++s) {
      F.counts[s] = (int)(neg[s + 1] - neg[s]);
      if (h_counts) h_counts[s] = F.counts[s];
    }
    for (int s = 0; s < K; ++s)
      if (F.m0[s] < F.counts[s]) return PDESHEP_COUNT_MISMATCH;
    return 0;
  };
  // quadrature per slice
  F.zh.resize((size_t)K * ne);
  F.wh.resize((size_t)K * ne);
  for (int s = 0; s < K; ++s) {
    if (h_nodes && h_weights) {
      for (int j = 0; j < ne; ++j) {
        F.zh[(size_t)s * ne + j] = h_nodes[(size_t)s * ne + j];
        F.wh[(size_t)s * ne + j] = h_weights[(size_t)s * ne + j];
      }
    } else {
      contour_rule(ne, h_bounds[s], h_bounds[s + 1], o->ellipse_ratio, &F.zh[(size_t)s * ne], &F.wh[(size_t)s * ne]);
    }
  }
  {
    std::vector<double2> zw((size_t)K * 2 * ne);
    for (int s = 0; s < K; ++s)
      for (int j = 0; j < ne; ++j) {
        zw[(size_t)s * 2 * ne + j] = make_double2(F.zh[(size_t)s * ne + j].re, F.zh[(size_t)s * ne + j].im);
        zw[(size_t)s * 2 * ne + ne + j] = make_double2(F.wh[(size_t)s * ne + j].re, F.wh[(size_t)s * ne + j].im);
      }
    PD_CK(cudaMemcpyAsync(F.p.zw, zw.data(), sizeof(double2) * zw.size(), cudaMemcpyHostToDevice, st));
  }
  F.mode = (o->precision == PDESHEP_MIXED && o->refine_policy == PDESHEP_REFINE_RESIDUAL) ? 1 : 0;
  std::vector<int> done(K, 0);
  F.active.clear();
  for (int s = 0; s < K; ++s) F.active.push_back(s);
  // start vectors: the caller's blocks, or drawn here (counter-based SplitMix64 stream)
  bool packed = true;
  for (int s = 0; s < K; ++s) packed = packed && F.io_col[s] == F.io_col[0] + F.col_off[s];
  if (d_x0 && packed) {
    PD_CK(cudaMemcpyAsync(F.p.Xt, (const S*)d_x0 + F.io_col[0] * n, sizeof(S) * (size_t)(n * F.M),
                          cudaMemcpyDeviceToDevice, st));
  } else if (d_x0) {
    for (int s = 0; s < K; ++s)
      PD_CK(cudaMemcpyAsync((S*)F.p.Xt + F.col_off[s] * n, (const S*)d_x0 + F.io_col[s] * n,
                            sizeof(S) * (size_t)(n * F.m0[s]), cudaMemcpyDeviceToDevice, st));
  } else {
    PD_TRY(F.upload_active());
    random_start_kernel<S><<<dim3(grid1(n * F.max_m0), K), 256, 0, st>>>(n, F.p.d_sd, o->seed, (S*)F.p.Xt);
    PD_CK_LAUNCH();
  }
  int status = 0;
  double ms_filter = 0, ms_rr = 0;
  auto timed = [&](double& acc_ms, auto&& fn) -> int {
    PD_CK(cudaEventRecord(e0, st));
    int r = fn();
    if (r) return r;
    PD_CK(cudaEventRecord(e1, st));
    PD_CK(cudaEventSynchronize(e1));
    float ms = 0;
    PD_CK(cudaEventElapsedTime(&ms, e0, e1));
    acc_ms += ms;
    return 0;
  };
  auto update_active = [&](int it) {
    std::vector<int> next;
    for (int s : F.active) {
      F.iters[s] = it;
      if (counts_ready && F.nconv[s] == F.counts[s])
        done[s] = 1;
      else
        next.push_back(s);
    }
    F.active.swap(next);
  };
  // The first iteration filters the start vectors themselves (Algorithm 1); in
  // mixed precision with residual refinement the later ones filter the FP64
  // residuals of the Ritz pairs.
  const int refine = F.mode;
  int it = 1;
  for (; it <= o->max_iter && !F.active.empty(); ++it) {
    F.mode = (refine && it > 1) ? 1 : 0;
    F.iter_now = it;
    if (it > F.kFFIterations && F.ff()) {
      F.rr_fp64_now = true;
      F.eig.ff = 0;
      F.stats.rr_fp64_from = it;
    }
    // a failure of the counts (non-finite band, subspace too small) takes precedence
    auto first_error = [&](int r) -> int {
      if (!r) return 0;
      const int rc = read_counts();
      return rc ? rc : r;
    };
    PD_TRY(first_error(timed(ms_filter, [&]() { return F.filter(); })));
    PD_TRY(first_error(timed(ms_rr, [&]() { return F.rr(); })));
    // the counts are read (and a slice can be declared converged) from the second iteration on:
    // the first pass almost never converges, and the inertia sweeps then overlap two passes
    if (it >= 2 || it >= o->max_iter) PD_TRY(read_counts());
    update_active(it);
  }
  PD_TRY(read_counts());
  if (F.tc()) PD_TRY(tc_read_error(F.p.tc, st));  // a tensor-core product whose bounded wait gave up
  if (o->precision == PDESHEP_MIXED) {
    int e = 0;
    PD_TRY(solve_tc_error(&e, 0, st));
    if (e) return PDESHEP_DEVICE_TIMEOUT;
  }
  if (!F.active.empty()) status = PDESHEP_NOT_CONVERGED;
  // outputs for every slice
  F.active.clear();
  for (int s = 0; s < K; ++s) F.active.push_back(s);
  PD_TRY(F.upload_active());
  order_kernel<<<K, 256, 0, st>>>(F.p.d_sd, F.p.lam, F.p.res, o->tol, F.p.dest);
  PD_CK_LAUNCH();
  scatter_out_kernel<S><<<grid1(n * F.M), 256, 0, st>>>(n, F.M, F.p.dest, F.p.lam, (const S*)F.p.Xt, d_evals,
                                                        (S*)d_evecs);
  PD_CK_LAUNCH();
  std::vector<double> res(F.M), lam(F.M);
  PD_CK(cudaMemcpyAsync(res.data(), F.p.res, sizeof(double) * F.M, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(lam.data(), F.p.lam, sizeof(double) * F.M, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  double maxres = 0.0;
  for (int s = 0; s < K; ++s) {
    int nf = 0;
    for (int c = 0; c < F.m0[s]; ++c) {
      const int64_t col = F.col_off[s] + c;
      if (lam[col] >= h_bounds[s] && lam[col] < h_bounds[s + 1] && res[col] <= o->tol) {
        ++nf;
        maxres = std::max(maxres, res[col]);
      }
    }
    if (h_nfound) h_nfound[s] = nf;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (h_stats) {
    F.stats.iterations = 0;
    for (int s = 0; s < K; ++s) F.stats.iterations = std::max(F.stats.iterations, F.iters[s]);
    F.stats.ms_solve = ms_filter;
    F.stats.ms_rr = ms_rr;
    F.stats.ms_total = ms_filter + ms_rr;  // the counts overlap the first filter pass
    F.stats.max_residual = maxres;
    PD_TRY(F.kt.collect());
    for (int gi = 0; gi < PDESHEP_KG_COUNT; ++gi) {
      F.stats.kg_ms[gi] = F.kt.ms[gi];
      F.stats.kg_launches[gi] = F.kt.nl[gi];
      F.stats.kg_flops[gi] = F.kt.fl[gi];
    }
    F.stats.ms_factor = F.kt.ms[PDESHEP_KG_FACTOR];
    F.stats.cluster_ctas = cluster_ctas_used();
    *h_stats = F.stats;
  }
  return status;
}

int check_slice_args(int64_t n, int32_t b, const void* d_band, int64_t ldab, int32_t K, const double* h_bounds,
                     int32_t ne, const pdeshep_c128* h_nodes, const pdeshep_c128* h_weights, const int32_t* h_m0,
                     const pdeshep_opts* o) {
  if (n <= 0) return -1;
  if (b < 0 || b >= n + 1) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (K <= 0) return -6;
  if (!h_bounds) return -7;
  for (int s = 0; s < K; ++s)
    if (!(h_bounds[s] < h_bounds[s + 1])) return -7;
  if (ne < 1 || ne > 64) return -8;
  if ((h_nodes == nullptr) != (h_weights == nullptr)) return -9;
  if (!h_m0) return -11;
  for (int s = 0; s < K; ++s)
    if (h_m0[s] < 1 || h_m0[s] > n || h_m0[s] > 4096) return -11;
  if (o && (!(o->tol > 0.0) || o->max_iter < 0 || (o->precision != PDESHEP_FP64 && o->precision != PDESHEP_MIXED) ||
            !(o->ellipse_ratio > 0.0) ||
            (o->rhs_chunk != 0 && o->rhs_chunk != 16 && o->rhs_chunk != 32 && o->rhs_chunk != 64 &&
             o->rhs_chunk != 128 && o->rhs_chunk != 256) ||
            (o->rr_arith != PDESHEP_RR_FLOATFLOAT && o->rr_arith != PDESHEP_RR_FP64 &&
             o->rr_arith != PDESHEP_RR_TENSOR) || o->autotune < 0 ||
            o->autotune > 2 || (o->m0_resize != 0 && o->m0_resize != 1)))
    return -15;
  if (o && o->m0_resize) {
    if (o->m0_cap < 1 || o->m0_cap > n || o->m0_cap > 4096) return -15;
    for (int s = 0; s < K; ++s)
      if (h_m0[s] > o->m0_cap) return -11;
  }
  return 0;
}

void merge_stats(pdeshep_stats& t, const pdeshep_stats& g) {
  t.iterations = std::max(t.iterations, g.iterations);
  t.waves += g.waves;
  t.factorizations += g.factorizations;
  t.rhs_sweeps += g.rhs_sweeps;
  t.ms_inertia += g.ms_inertia;
  t.ms_factor += g.ms_factor;
  t.ms_solve += g.ms_solve;
  t.ms_rr += g.ms_rr;
  t.ms_total += g.ms_total;
  t.max_residual = std::max(t.max_residual, g.max_residual);
  for (int i = 0; i < PDESHEP_KG_COUNT; ++i) {
    t.kg_ms[i] += g.kg_ms[i];
    t.kg_launches[i] += g.kg_launches[i];
    t.kg_flops[i] += g.kg_flops[i];
  }
  t.rhs_columns += g.rhs_columns;
  t.cluster_ctas = std::max(t.cluster_ctas, g.cluster_ctas);
  t.jacobi_sweeps64 += g.jacobi_sweeps64;
  t.jacobi_sweeps32 += g.jacobi_sweeps32;
  t.rr_calls += g.rr_calls;
  t.eig_refine_steps += g.eig_refine_steps;
  t.eig_clusters += g.eig_clusters;
  t.eig_max_cluster = std::max(t.eig_max_cluster, g.eig_max_cluster);
  t.eig_fallback_unconverged += g.eig_fallback_unconverged;
  t.eig_fallback_wide += g.eig_fallback_wide;
  t.rhs_chunk_used = g.rhs_chunk_used;
  t.rhs_chunk_early = std::max(t.rhs_chunk_early, g.rhs_chunk_early);
  t.gram_splits_used = g.gram_splits_used;
  t.tuned += g.tuned;
  t.graph_launches += g.graph_launches;
  t.cholqr_shifted += g.cholqr_shifted;
  t.gram_fp64 += g.gram_fp64;
  if (g.rr_fp64_from && (!t.rr_fp64_from || g.rr_fp64_from < t.rr_fp64_from)) t.rr_fp64_from = g.rr_fp64_from;
}

// The whole call.  (1) With opts.m0_resize, the exact counts m_i come first and
// a slice whose m0 is below m_i + 10 runs with max(ceil(1.3 m_i), m_i + 10)
// columns (at most opts.m0_cap), the subspace rule of Section 3.2 applied by
// the library instead of a failed run and a rerun.  (2) The slices are run in
// consecutive groups whose factorizations all stay resident in the workspace
// (and, with hbm_cap_bytes, within that cap), each group iterating to
// convergence on factors computed once: the paper's level L1 (slices) becomes
// the sequence of groups.  A call that fits whole is one group.  A slice whose
// own factors exceed the budget forms a group that streams its factors in
// waves every iteration.
template <typename S, typename C>
int band_slice_run(int64_t n, int b, int cplx, const void* band, int64_t ldab, int K, const double* h_bounds,
                   int ne, const pdeshep_c128* h_nodes, const pdeshep_c128* h_weights, const int32_t* h_m0,
                   const void* d_x0, void* d_work, size_t work_bytes, const pdeshep_opts* o, double* d_evals,
                   void* d_evecs, int32_t* h_counts, int32_t* h_nfound, pdeshep_stats* h_stats, size_t* size_only) {
  const bool resize = o->m0_resize != 0;
  cudaStream_t st = (cudaStream_t)o->stream;
  std::vector<int32_t> m0(h_m0, h_m0 + K);
  std::vector<int64_t> io(K, 0);
  for (int s = 1; s < K; ++s) io[s] = resize ? (int64_t)s * o->m0_cap : io[s - 1] + m0[s - 1];
  std::vector<int64_t> neg;
  if (resize) {
    if (size_only) {
      for (int s = 0; s < K; ++s) m0[s] = o->m0_cap;  // the largest subspaces the call may use
    } else {
      neg.assign(K + 1, 0);
      if (work_bytes < inertia_ws_bytes(b, cplx, K + 1)) return PDESHEP_WORKSPACE_TOO_SMALL;
      bool bad = false;
      PD_TRY(inertia_counts(n, b, cplx, band, ldab, K + 1, h_bounds, neg.data(), nullptr, d_work, work_bytes, st,
                            &bad));
      if (bad) return PDESHEP_NONFINITE_INPUT;
      bool short_cap = false;
      for (int s = 0; s < K; ++s) {
        const int64_t m = neg[s + 1] - neg[s];
        if (h_counts) h_counts[s] = (int32_t)m;
        if (m0[s] < m + 10) m0[s] = (int32_t)std::max<int64_t>((13 * m + 9) / 10, m + 10);
        m0[s] = std::min(m0[s], o->m0_cap);
        if (m0[s] < m) short_cap = true;
      }
      if (o->h_m0_used)
        for (int s = 0; s < K; ++s) o->h_m0_used[s] = m0[s];
      if (short_cap) return PDESHEP_COUNT_MISMATCH;
    }
  } else if (o->h_m0_used && !size_only) {
    for (int s = 0; s < K; ++s) o->h_m0_used[s] = m0[s];
  }
  // workspace of a group of slices [s0, s1) with all factors resident
  auto resident_bytes = [&](int s0, int s1) -> size_t {
    pdeshep_opts og = *o;
    og.hbm_cap_bytes = 0;
    size_t sz = 0;
    feast_entry<S, C>(n, b, cplx, nullptr, ldab, s1 - s0, nullptr, ne, nullptr, nullptr, m0.data() + s0, nullptr,
                      nullptr, nullptr, nullptr, 0, &og, nullptr, nullptr, nullptr, nullptr, nullptr, &sz);
    return sz;
  };
  const FactorGeom g = make_geom(n, b);
  const size_t fb = factor_bytes(g, sizeof(C));
  auto sys_bytes = [&](int s0, int s1) -> size_t {
    size_t t = 0;
    for (int s = s0; s < s1; ++s)
      t += (size_t)ne * (fb + (((size_t)n * m0[s] * (cplx ? 2 : 1) * sizeof(C) + 255) & ~size_t(255)));
    return t;
  };
  const size_t cap = o->hbm_cap_bytes;
  const size_t budget = size_only ? ~size_t(0) : work_bytes;
  auto fits = [&](int s0, int s1) {
    return (cap == 0 || sys_bytes(s0, s1) <= cap) && resident_bytes(s0, s1) <= budget;
  };
  std::vector<std::pair<int, int>> groups;
  if (fits(0, K)) {
    groups.push_back({0, K});
  } else {
    int s0 = 0;
    while (s0 < K) {
      int s1 = s0 + 1;
      if (fits(s0, s1))
        while (s1 < K && fits(s0, s1 + 1)) ++s1;
      groups.push_back({s0, s1});
      s0 = s1;
    }
  }
  if (size_only) {
    size_t mx = 0;
    for (auto& gr : groups) {
      size_t sz = 0;
      PD_TRY((feast_entry<S, C>(n, b, cplx, nullptr, ldab, gr.second - gr.first, nullptr, ne, nullptr, nullptr,
                                m0.data() + gr.first, nullptr, nullptr, nullptr, nullptr, 0, o, nullptr, nullptr,
                                nullptr, nullptr, nullptr, &sz)));
      mx = std::max(mx, sz);
    }
    *size_only = std::max(mx, resize ? inertia_ws_bytes(b, cplx, K + 1) : size_t(0));
    return 0;
  }
  pdeshep_stats total;
  memset(&total, 0, sizeof(total));
  int status = 0;
  for (auto& gr : groups) {
    const int s0 = gr.first, kg = gr.second - gr.first;
    pdeshep_stats gs;
    const int r = feast_entry<S, C>(n, b, cplx, band, ldab, kg, h_bounds + s0, ne,
                                    h_nodes ? h_nodes + (size_t)s0 * ne : nullptr,
                                    h_weights ? h_weights + (size_t)s0 * ne : nullptr, m0.data() + s0,
                                    io.data() + s0, resize ? neg.data() + s0 : nullptr, d_x0, d_work, work_bytes, o,
                                    d_evals, d_evecs, h_counts ? h_counts + s0 : nullptr,
                                    h_nfound ? h_nfound + s0 : nullptr, h_stats ? &gs : nullptr, nullptr);
    if (r != 0 && r != PDESHEP_NOT_CONVERGED) return r;
    if (r) status = r;
    if (h_stats) merge_stats(total, gs);
  }
  if (h_stats) *h_stats = total;
  return status;
}

}  // namespace

extern "C" size_t pdeshep_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nslices,
                                         const int32_t* h_m0, int32_t ne, const pdeshep_opts* opts) {
  pdeshep_opts def;
  pdeshep_opts_default(&def);
  const pdeshep_opts* o = opts ? opts : &def;
  if (n <= 0 || b < 0 || nslices <= 0 || !h_m0 || ne < 1) return 0;
  if (o->m0_resize && (o->m0_cap < 1 || o->m0_cap > 4096)) return 0;
  size_t sz = 0;
  int r;
  if (is_complex) {
    if (o->precision == PDESHEP_MIXED)
      r = band_slice_run<double2, float2>(n, b, 1, nullptr, b + 1, nslices, nullptr, ne, nullptr, nullptr, h_m0,
                                          nullptr, nullptr, 0, o, nullptr, nullptr, nullptr, nullptr, nullptr, &sz);
    else
      r = band_slice_run<double2, double2>(n, b, 1, nullptr, b + 1, nslices, nullptr, ne, nullptr, nullptr, h_m0,
                                           nullptr, nullptr, 0, o, nullptr, nullptr, nullptr, nullptr, nullptr, &sz);
  } else {
    if (o->precision == PDESHEP_MIXED)
      r = band_slice_run<double, float2>(n, b, 0, nullptr, b + 1, nslices, nullptr, ne, nullptr, nullptr, h_m0,
                                         nullptr, nullptr, 0, o, nullptr, nullptr, nullptr, nullptr, nullptr, &sz);
    else
      r = band_slice_run<double, double2>(n, b, 0, nullptr, b + 1, nslices, nullptr, ne, nullptr, nullptr, h_m0,
                                          nullptr, nullptr, 0, o, nullptr, nullptr, nullptr, nullptr, nullptr, &sz);
  }
  return r ? 0 : sz;
}

extern "C" int pdeshep_band_slice(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                  int32_t nslices, const double* h_bounds, int32_t ne, const pdeshep_c128* h_nodes,
                                  const pdeshep_c128* h_weights, const int32_t* h_m0, const void* d_x0,
                                  void* d_work, size_t work_bytes, const pdeshep_opts* opts, double* d_evals,
                                  void* d_evecs, int32_t* h_counts, int32_t* h_nfound, pdeshep_stats* h_stats) {
  pdeshep_opts def;
  pdeshep_opts_default(&def);
  const pdeshep_opts* o = opts ? opts : &def;
  int r = check_slice_args(n, b, d_band, ldab, nslices, h_bounds, ne, h_nodes, h_weights, h_m0, opts);
  if (r) return r;
  if (!d_work) return -13;
  if (!d_evals) return -16;
  if (!d_evecs) return -17;
  if (is_complex) {
    if (o->precision == PDESHEP_MIXED)
      return band_slice_run<double2, float2>(n, b, 1, d_band, ldab, nslices, h_bounds, ne, h_nodes, h_weights, h_m0,
                                             d_x0, d_work, work_bytes, o, d_evals, d_evecs, h_counts, h_nfound,
                                             h_stats, nullptr);
    return band_slice_run<double2, double2>(n, b, 1, d_band, ldab, nslices, h_bounds, ne, h_nodes, h_weights, h_m0,
                                            d_x0, d_work, work_bytes, o, d_evals, d_evecs, h_counts, h_nfound,
                                            h_stats, nullptr);
  }
  if (o->precision == PDESHEP_MIXED)
    return band_slice_run<double, float2>(n, b, 0, d_band, ldab, nslices, h_bounds, ne, h_nodes, h_weights, h_m0,
                                          d_x0, d_work, work_bytes, o, d_evals, d_evecs, h_counts, h_nfound, h_stats,
                                          nullptr);
  return band_slice_run<double, double2>(n, b, 0, d_band, ldab, nslices, h_bounds, ne, h_nodes, h_weights, h_m0,
                                         d_x0, d_work, work_bytes, o, d_evals, d_evecs, h_counts, h_nfound, h_stats,
                                         nullptr);
}

namespace {
template <typename S>
__global__ void random_block_kernel(int64_t n, int64_t col0, int ncols, uint64_t seed, S* __restrict__ X) {
  const int64_t total = n * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    const uint64_t k = (uint64_t)((col0 + c) * n + i);
    if constexpr (std::is_same<S, double>::value)
      X[e] = uniform_pm1(splitmix64(seed + k));
    else
      X[e] = make_double2(uniform_pm1(splitmix64(seed + 2 * k)), uniform_pm1(splitmix64(seed + 2 * k + 1)));
  }
}
}  // namespace

extern "C" int pdeshep_random_start(int64_t n, int32_t is_complex, int64_t col0, int32_t ncols, uint64_t seed,
                                    void* d_x, void* stream) {
  if (n <= 0) return -1;
  if (col0 < 0) return -3;
  if (ncols < 0) return -4;
  if (!d_x && ncols > 0) return -6;
  if (ncols == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = grid1(n * ncols);
  if (is_complex)
    random_block_kernel<double2><<<blocks, 256, 0, st>>>(n, col0, ncols, seed, (double2*)d_x);
  else
    random_block_kernel<double><<<blocks, 256, 0, st>>>(n, col0, ncols, seed, (double*)d_x);
  PD_CK_LAUNCH();
  return 0;
}
