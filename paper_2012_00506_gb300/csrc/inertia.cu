// inertia.cu -- Sylvester inertia of B - sigma I by a pivot-free LDL^T (real)
// or LDL^H (complex) factorization in FP64, one CTA per shift sigma.
//
// The paper counts the eigenvalues of each slice from the inertia of
// D - b_i I at both ends of the slice (Section 3.2, "Validation and Other
// Details"), using a band LDL^H that keeps no L.  Here the count is computed
// for many shifts at once (one thread block per shift).  The active
// (b+1)-column window of the band lives in shared memory when it fits,
// otherwise in a per-shift slice of the workspace (L2 resident); each step
// eliminates one column with a rank-1 update of the trailing b x b triangle.
//
// Every floating-point operation is an explicitly rounded __dmul_rn /
// __dsub_rn / __ddiv_rn (no contraction), in the same order as the CPU
// reference, so the counts and pivots are bit-reproducible:
//   d_k = W(k,k) (zero -> -pivmin);  l_i = W(i,k) / d_k;
//   W(i,j) -= l_i * conj(W(j,k))  for k < j <= i <= k+b,
// with t = l*conj(a) formed as (l.re*a.re + l.im*a.im, l.im*a.re - l.re*a.im)
// and only the real part applied on the diagonal.
#include <float.h>


#include "common.cuh"

namespace pdeshep {

// ---------------------------------------------------------------------------
// max over stored entries of max(|Re|,|Im|) (as ordered uint64 bits of a
// non-negative double) and a non-finite flag.
// ---------------------------------------------------------------------------
__global__ void band_amax_kernel(int64_t n, int b, int cplx, const double* __restrict__ band,
                                 int64_t ldab, unsigned long long* amax_bits, int* nonfinite) {
  const int64_t per = cplx ? 2 : 1;
  const int64_t total = n * (int64_t)(b + 1);
  double m = 0.0;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / (b + 1);
    int d = (int)(e - j * (b + 1));
    if (j + d >= n) continue;
    const double* p = band + (d + j * ldab) * per;
    for (int c = 0; c < per; ++c) {
      double v = p[c];
      if (!isfinite(v)) bad = 1;
      double a = fabs(v);
      if (a > m) m = a;
    }
  }
  // warp reduce
  for (int o = 16; o > 0; o >>= 1) {
    double t = __shfl_down_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(amax_bits, (unsigned long long)__double_as_longlong(m));
    if (bad) atomicOr(nonfinite, 1);
  }
}

template <bool CPLX>
struct InertiaElem;
template <>
struct InertiaElem<false> {
  using T = double;
};
template <>
struct InertiaElem<true> {
  using T = double2;
};

// The active window (rows and columns k..k+b at step k) is stored by
// diagonals: diagonal d (d = i - j, 0..b) is a ring of R_d = b + 1 - d
// entries, entry (i, j) at ring_base(d) + (j mod R_d).  At step k column j
// = k + s of the window holds rows j..k+b, so diagonal d holds the columns
// k..k+b-d: exactly R_d entries, (b+1)(b+2)/2 in all (half of a square
// window).  After step k the entries of column k are dead; the row k+b+1 that
// enters next lands in exactly those slots (its entry on diagonal d is column
// k+b+1-d = k + R_d).
__host__ __device__ __forceinline__ int ring_base(int d, int b) { return d * (b + 1) - d * (d - 1) / 2; }

// Row r of B - sigma I (entries (r, j), j = max(0, r-b)..r) into the rings; h[d] = k mod R_d for the
// step k that first uses the row (only the column index modulo R_d is needed: j mod R_d).
template <bool CPLX>
__device__ __forceinline__ void load_row(typename InertiaElem<CPLX>::T* W, int b, int64_t r, int64_t k,
                                         const int* h, const double* band, int64_t ldab, double sigma) {
  for (int d = threadIdx.x; d <= b; d += blockDim.x) {
    const int64_t j = r - d;
    if (j < 0 || j < k) continue;
    // j - k = b - d' for the row r = k + b (window bottom row), so j mod R_d = h[d] + (j - k) wrapped
    const int R = b + 1 - d;
    int pos = h[d] + (int)(j - k);
    if (pos >= R) pos -= R;
    const int e = ring_base(d, b) + pos;
    if constexpr (CPLX) {
      const double* p = band + 2 * (d + j * ldab);
      double2 v = make_double2(p[0], p[1]);
      if (d == 0) v = make_double2(__dsub_rn(v.x, sigma), 0.0);
      W[e] = v;
    } else {
      double v = band[d + j * ldab];
      if (d == 0) v = __dsub_rn(v, sigma);
      W[e] = v;
    }
  }
}

// One CTA per shift.  Shared memory: pair table (s,u) packed as int32, the
// multipliers L[0..b], the ring heads h[0..b] and (if `gwin` is null) the
// window rings W[(b+1)(b+2)/2].
template <bool CPLX>
__global__ void __launch_bounds__(256) inertia_kernel(int64_t n, int b, const double* __restrict__ band,
                                                      int64_t ldab, const double* __restrict__ sigmas,
                                                      const unsigned long long* amax_bits,
                                                      int64_t* __restrict__ neg_out,
                                                      double* __restrict__ piv_out, char* gwin,
                                                      size_t gwin_stride) {
  using T = typename InertiaElem<CPLX>::T;
  extern __shared__ __align__(16) char smem[];
  const int B1 = b + 1;
  const int npairs = b * (b + 1) / 2;
  int* pairs = (int*)smem;
  T* L = (T*)(smem + (((size_t)npairs * 4 + 15) & ~size_t(15)));
  int* h = (int*)(L + B1);
  T* W = gwin ? (T*)(gwin + gwin_stride * blockIdx.x)
              : (T*)((char*)h + (((size_t)B1 * sizeof(int) + 15) & ~size_t(15)));

  const int sid = blockIdx.x;
  const double sigma = sigmas[sid];
  const double amax = __longlong_as_double((long long)*amax_bits);
  const double a2 = __dmul_rn(amax, amax);
  const double pivmin = DBL_MIN * (a2 > 1.0 ? a2 : 1.0);

  // pair table: s in 1..b (column offset), u in 0..b-s (row offset from the column)
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    // invert p = sum_{s'<s} (b - s' + 1) + u  -- small loop, done once
    int s = 1, rem = p;
    while (rem >= b - s + 1) {
      rem -= b - s + 1;
      ++s;
    }
    pairs[p] = (s << 16) | rem;
  }
  for (int d = threadIdx.x; d < B1; d += blockDim.x) h[d] = 0;  // k = 0: 0 mod R_d
  __syncthreads();
  // rows 0..b of the first window: entry (r, j) of diagonal d = r - j at ring position j (j < R_d)
  for (int64_t r = 0; r < B1 && r < n; ++r) {
    for (int d = threadIdx.x; d <= b; d += blockDim.x) {
      const int64_t j = r - d;
      if (j < 0) continue;
      const int e = ring_base(d, b) + (int)j;
      if constexpr (CPLX) {
        const double* pp = band + 2 * (d + j * ldab);
        double2 v = make_double2(pp[0], pp[1]);
        if (d == 0) v = make_double2(__dsub_rn(v.x, sigma), 0.0);
        W[e] = v;
      } else {
        double v = band[d + j * ldab];
        if (d == 0) v = __dsub_rn(v, sigma);
        W[e] = v;
      }
    }
  }
  __syncthreads();

  int64_t neg = 0;
  for (int64_t k = 0; k < n; ++k) {
    const int kmax = (int)((n - 1 - k) < b ? (n - 1 - k) : b);  // rows below k inside the matrix
    // column k sits at ring position h[d] of every diagonal d
    double dk;
    if constexpr (CPLX)
      dk = W[h[0]].x;
    else
      dk = W[h[0]];
    if (dk == 0.0) dk = -pivmin;
    if (threadIdx.x == 0) {
      if (dk < 0.0) ++neg;
      if (piv_out) piv_out[(int64_t)sid * n + k] = dk;
    }
    for (int d = 1 + threadIdx.x; d <= kmax; d += blockDim.x) {
      T a = W[ring_base(d, b) + h[d]];
      if constexpr (CPLX)
        L[d] = make_double2(__ddiv_rn(a.x, dk), __ddiv_rn(a.y, dk));
      else
        L[d] = __ddiv_rn(a, dk);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
      const int pr = pairs[p];
      const int s = pr >> 16, u = pr & 0xffff;
      if (s + u > kmax) continue;
      // W(k+s+u, k+s): diagonal u, column k+s -> position h[u] + s (mod R_u; s <= b - u < R_u)
      int pos = h[u] + s;
      const int R = B1 - u;
      if (pos >= R) pos -= R;
      T a = W[ring_base(s, b) + h[s]];  // W(k+s, k)
      T l = L[s + u];
      T* e = &W[ring_base(u, b) + pos];
      if constexpr (CPLX) {
        double p1 = __dmul_rn(l.x, a.x);
        double p2 = __dmul_rn(l.y, a.y);
        double tre = __dadd_rn(p1, p2);
        if (u == 0) {
          e->x = __dsub_rn(e->x, tre);
        } else {
          double p3 = __dmul_rn(l.y, a.x);
          double p4 = __dmul_rn(l.x, a.y);
          double tim = __dsub_rn(p3, p4);
          double2 v = *e;
          v.x = __dsub_rn(v.x, tre);
          v.y = __dsub_rn(v.y, tim);
          *e = v;
        }
      } else {
        *e = __dsub_rn(*e, __dmul_rn(l, a));
      }
    }
    __syncthreads();
    // column k is finished: advance the ring heads to k + 1 and bring in row k + 1 + b
    for (int d = threadIdx.x; d < B1; d += blockDim.x) {
      const int R = B1 - d;
      h[d] = h[d] + 1 == R ? 0 : h[d] + 1;
    }
    __syncthreads();
    if (k + B1 < n) load_row<CPLX>(W, b, k + B1, k + 1, h, band, ldab, sigma);
    __syncthreads();
  }
  if (threadIdx.x == 0) neg_out[sid] = neg;
}

static size_t window_bytes(int b, int cplx) {
  return (size_t)(b + 1) * (b + 2) / 2 * (cplx ? 16 : 8);
}
static size_t inertia_smem_base(int b, int cplx) {
  size_t npairs = (size_t)b * (b + 1) / 2;
  return ((npairs * 4 + 15) & ~size_t(15)) + (size_t)(b + 1) * (cplx ? 16 : 8) +
         (((size_t)(b + 1) * sizeof(int) + 15) & ~size_t(15));
}
static bool window_in_smem(int b, int cplx) {
  return inertia_smem_base(b, cplx) + window_bytes(b, cplx) <= 226 * 1024;
}

// Workspace layout: amax bits, nonfinite flag, sigma[], neg[], global windows.
struct InertiaWs {
  unsigned long long* amax;
  int* nonfinite;
  double* sigma;
  int64_t* neg;
  char* gwin;
  size_t gwin_stride;
};

static InertiaWs plan_inertia(Arena& a, int b, int cplx, int nsigma) {
  InertiaWs w;
  w.amax = a.take<unsigned long long>(1);
  w.nonfinite = a.take<int>(1);
  w.sigma = a.take<double>(nsigma);
  w.neg = a.take<int64_t>(nsigma);
  w.gwin = nullptr;
  w.gwin_stride = 0;
  if (!window_in_smem(b, cplx)) {
    w.gwin_stride = (window_bytes(b, cplx) + 255) & ~size_t(255);
    w.gwin = a.take<char>(w.gwin_stride * nsigma);
  }
  return w;
}

// Computes amax (and the non-finite flag) of a band into ws.  Async.
int launch_band_amax(int64_t n, int b, int cplx, const void* band, int64_t ldab,
                     unsigned long long* amax, int* nonfinite, cudaStream_t st) {
  PD_CK(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st));
  PD_CK(cudaMemsetAsync(nonfinite, 0, sizeof(int), st));
  int64_t total = n * (int64_t)(b + 1);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  band_amax_kernel<<<blocks, 256, 0, st>>>(n, b, cplx, (const double*)band, ldab, amax, nonfinite);
  PD_CK_LAUNCH();
  return 0;
}

// Batched inertia with sigma already on the device; results into d_neg.  Async.
int launch_inertia(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                   const double* d_sigma, const unsigned long long* amax, int64_t* d_neg,
                   double* d_piv, char* gwin, size_t gwin_stride, cudaStream_t st) {
  if (nsigma <= 0) return 0;
  size_t smem = inertia_smem_base(b, cplx) + (gwin ? 0 : window_bytes(b, cplx));
  if (cplx) {
    PD_CK(cudaFuncSetAttribute(inertia_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
    inertia_kernel<true><<<nsigma, 256, smem, st>>>(n, b, (const double*)band, ldab, d_sigma, amax,
                                                    d_neg, d_piv, gwin, gwin_stride);
  } else {
    PD_CK(cudaFuncSetAttribute(inertia_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
    inertia_kernel<false><<<nsigma, 256, smem, st>>>(n, b, (const double*)band, ldab, d_sigma, amax,
                                                     d_neg, d_piv, gwin, gwin_stride);
  }
  PD_CK_LAUNCH();
  return 0;
}

size_t inertia_ws_bytes(int b, int cplx, int nsigma) {
  Arena a;
  plan_inertia(a, b, cplx, nsigma);
  return a.used();
}

// Asynchronous counts: everything is enqueued on st; the counts (nsigma int64)
// and the non-finite flag (int) stay in the workspace at *d_neg / *d_bad.
int inertia_counts_async(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                         const double* h_sigma, void* work, size_t wbytes, cudaStream_t st,
                         const int64_t** d_neg, const int** d_bad) {
  Arena a(work, wbytes);
  InertiaWs w = plan_inertia(a, b, cplx, nsigma);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  PD_TRY(launch_band_amax(n, b, cplx, band, ldab, w.amax, w.nonfinite, st));
  PD_CK(cudaMemcpyAsync(w.sigma, h_sigma, sizeof(double) * nsigma, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_inertia(n, b, cplx, band, ldab, nsigma, w.sigma, w.amax, w.neg, nullptr, w.gwin,
                        w.gwin_stride, st));
  *d_neg = w.neg;
  *d_bad = w.nonfinite;
  return 0;
}

// Synchronous helper used by the host-side drivers (bisection, slicing).
int inertia_counts(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma,
                   const double* h_sigma, int64_t* h_neg, double* d_piv, void* work, size_t wbytes,
                   cudaStream_t st, bool* nonfinite_out) {
  Arena a(work, wbytes);
  InertiaWs w = plan_inertia(a, b, cplx, nsigma);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  PD_TRY(launch_band_amax(n, b, cplx, band, ldab, w.amax, w.nonfinite, st));
  PD_CK(cudaMemcpyAsync(w.sigma, h_sigma, sizeof(double) * nsigma, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_inertia(n, b, cplx, band, ldab, nsigma, w.sigma, w.amax, w.neg, d_piv, w.gwin,
                        w.gwin_stride, st));
  int bad = 0;
  PD_CK(cudaMemcpyAsync(h_neg, w.neg, sizeof(int64_t) * nsigma, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(&bad, w.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  if (nonfinite_out) *nonfinite_out = bad != 0;
  return 0;
}

// ---------------------------------------------------------------------------
// Gershgorin interval: per row, centre Re B(i,i), radius sum_{j != i} |B(i,j)|.
// ---------------------------------------------------------------------------
__global__ void gershgorin_kernel(int64_t n, int b, int cplx, const double* __restrict__ band,
                                  int64_t ldab, double* part_lo, double* part_hi) {
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // Row i of the Hermitian band in ascending column order, |b_ij| = sqrt(re^2 + im^2)
    // rounded step by step (no FMA): the interval is a fixed function of the band's bits,
    // so bin decisions taken against it (the proposer's histogram) are reproducible.
    double r = 0.0;
    const int64_t j0 = i - b < 0 ? 0 : i - b, j1 = i + b > n - 1 ? n - 1 : i + b;
    for (int64_t j = j0; j <= j1; ++j) {
      if (j == i) continue;
      // B(i, j) for j < i is stored in column j at row offset i - j; for j > i it is
      // conj(B(j, i)), stored in column i at offset j - i (the modulus ignores the conjugate)
      const int64_t e = j < i ? (i - j) + j * ldab : (j - i) + i * ldab;
      double a;
      if (cplx) {
        const double re = band[2 * e], im = band[2 * e + 1];
        a = __dsqrt_rn(__dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im)));
      } else {
        const double re = band[e];
        a = __dsqrt_rn(__dmul_rn(re, re));
      }
      r = __dadd_rn(r, a);
    }
    double c = cplx ? band[2 * (i * ldab)] : band[i * ldab];
    lo = fmin(lo, __dsub_rn(c, r));
    hi = fmax(hi, __dadd_rn(c, r));
  }
  __shared__ double slo[32], shi[32];
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    slo[threadIdx.x >> 5] = lo;
    shi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, slo[w]);
      hi = fmax(hi, shi[w]);
    }
    part_lo[blockIdx.x] = lo;
    part_hi[blockIdx.x] = hi;
  }
}

__global__ void minmax_final_kernel(int nparts, double* part_lo, double* part_hi) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double lo = INFINITY, hi = -INFINITY;
    for (int p = 0; p < nparts; ++p) {
      lo = fmin(lo, part_lo[p]);
      hi = fmax(hi, part_hi[p]);
    }
    part_lo[0] = lo;
    part_hi[0] = hi;
  }
}

static const int kGershBlocks = 256;

int gershgorin_device(int64_t n, int b, int cplx, const void* band, int64_t ldab, double* d_lo,
                      double* d_hi, cudaStream_t st) {
  gershgorin_kernel<<<kGershBlocks, 256, 0, st>>>(n, b, cplx, (const double*)band, ldab, d_lo, d_hi);
  PD_CK_LAUNCH();
  minmax_final_kernel<<<1, 32, 0, st>>>(kGershBlocks, d_lo, d_hi);
  PD_CK_LAUNCH();
  return 0;
}
size_t gershgorin_ws_doubles() { return 2 * kGershBlocks; }

// ---------------------------------------------------------------------------
// Allocation-free variant.  Its scratch (the amax word, the non-finite flag,
// the shifts and the counts) lives in a fixed device array that every GPU
// loading this library holds until the process exits; the LDL^T window must
// then fit in shared memory.  Host code cannot use the array's name as a
// device address, so every call looks the address up on the current device
// with cudaGetSymbolAddress (cheap next to the synchronous inertia launch; no
// cached pointer can outlive a cudaDeviceReset or a change of context).
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxSigma = 1024;
constexpr size_t kNoAllocBytes = 20 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static int noalloc_scratch_address(void** out) {
  void* p = nullptr;
  PD_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = p;
  return 0;
}

}  // namespace pdeshep

using namespace pdeshep;

extern "C" int pdeshep_inertia_noalloc(int64_t n, int32_t b, int32_t is_complex, const void* d_band,
                                       int64_t ldab, int32_t nsigma, const double* h_sigma,
                                       int64_t* h_neg, void* stream) {
  if (n < 0) return -1;
  const int cplx = is_complex ? 1 : 0;
  if (b < 0) {
    set_last_error_msg("pdeshep_inertia_noalloc: negative semi-bandwidth");
    return -2;
  }
  if (!window_in_smem(b, cplx)) {
    set_last_error_msg("pdeshep_inertia_noalloc: band too wide for the shared-memory window "
                       "(real b <= 194, complex b <= 149)");
    return -2;
  }
  if (!d_band && n > 0) return -4;
  if (ldab < b + 1) return -5;
  if (nsigma < 0 || nsigma > kNoAllocMaxSigma) {
    set_last_error_msg("pdeshep_inertia_noalloc: nsigma must be in [0, 1024]");
    return -6;
  }
  if (!h_sigma && nsigma > 0) return -7;
  if (!h_neg && nsigma > 0) return -8;
  if (n == 0 || nsigma == 0) {
    for (int s = 0; s < nsigma; ++s) h_neg[s] = 0;
    return 0;
  }
  void* base = nullptr;
  PD_TRY(noalloc_scratch_address(&base));
  char* p = (char*)base;
  unsigned long long* amax = (unsigned long long*)p;
  int* nonfinite = (int*)(p + 64);
  double* sigma = (double*)(p + 256);
  int64_t* neg = (int64_t*)(p + 256 + sizeof(double) * kNoAllocMaxSigma);
  cudaStream_t st = (cudaStream_t)stream;
  // amax and the flag are cleared here; sigma and neg are overwritten by this call
  PD_TRY(launch_band_amax(n, b, cplx, d_band, ldab, amax, nonfinite, st));
  PD_CK(cudaMemcpyAsync(sigma, h_sigma, sizeof(double) * nsigma, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_inertia(n, b, cplx, d_band, ldab, nsigma, sigma, amax, neg, nullptr, nullptr, 0, st));
  int bad = 0;
  PD_CK(cudaMemcpyAsync(h_neg, neg, sizeof(int64_t) * nsigma, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(&bad, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  return bad ? PDESHEP_NONFINITE_INPUT : 0;
}

extern "C" size_t pdeshep_inertia_workspace_size(int64_t n, int32_t b, int32_t is_complex,
                                                 int32_t nsigma) {
  (void)n;
  if (b < 0 || nsigma < 0) return 0;
  return inertia_ws_bytes(b, is_complex ? 1 : 0, nsigma);
}

extern "C" int pdeshep_inertia(int64_t n, int32_t b, int32_t is_complex, const void* d_band,
                               int64_t ldab, int32_t nsigma, const double* h_sigma, int64_t* h_neg,
                               double* d_pivots, void* d_work, size_t work_bytes, void* stream) {
  if (n < 0) return -1;
  if (b < 0 || b > 4096) return -2;
  if (!d_band && n > 0) return -4;
  if (ldab < b + 1) return -5;
  if (nsigma < 0) return -6;
  if (!h_sigma && nsigma > 0) return -7;
  if (!h_neg && nsigma > 0) return -8;
  if (n == 0 || nsigma == 0) {
    for (int s = 0; s < nsigma; ++s) h_neg[s] = 0;
    return 0;
  }
  if (!d_work) return -10;
  bool bad = false;
  int st = inertia_counts(n, b, is_complex ? 1 : 0, d_band, ldab, nsigma, h_sigma, h_neg, d_pivots,
                          d_work, work_bytes, (cudaStream_t)stream, &bad);
  if (st) return st;
  return bad ? PDESHEP_NONFINITE_INPUT : 0;
}

extern "C" int pdeshep_gershgorin(int64_t n, int32_t b, int32_t is_complex, const void* d_band,
                                  int64_t ldab, double* h_lo, double* h_hi, void* d_work,
                                  size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (!h_lo) return -6;
  if (!h_hi) return -7;
  if (!d_work || work_bytes < sizeof(double) * gershgorin_ws_doubles()) return -8;
  cudaStream_t st = (cudaStream_t)stream;
  double* lo = (double*)d_work;
  double* hi = lo + kGershBlocks;
  PD_TRY(gershgorin_device(n, b, is_complex ? 1 : 0, d_band, ldab, lo, hi, st));
  PD_CK(cudaMemcpyAsync(h_lo, lo, sizeof(double), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(h_hi, hi, sizeof(double), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  return 0;
}
