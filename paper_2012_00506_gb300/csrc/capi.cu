// capi.cu -- C-ABI entry points for the individual steps of the slicing path
// (shifted solves of eq. (10), CholQR, small Hermitian eigensolver, band
// product), used by callers that drive the steps themselves and by the
// parity tests.  The FEAST driver is in feast.cu, inertia in inertia.cu.
#include <algorithm>
#include <vector>

#include "band_lu.cuh"
#include "dense.cuh"
#include "tcgemm.cuh"

namespace pdeshep {

template <typename A, typename Bt>
__global__ void cast_kernel(int64_t total, const A* __restrict__ src, Bt* __restrict__ dst) {
  using RB = typename real_of<Bt>::type;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const A v = src[e];
    Bt w;
    w.x = (RB)v.x;
    w.y = (RB)v.y;
    dst[e] = w;
  }
}

template <typename A, typename Bt>
static int launch_cast(int64_t total, const A* src, Bt* dst, cudaStream_t st) {
  if (total <= 0) return 0;
  int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 16);
  cast_kernel<A, Bt><<<(unsigned)blocks, 256, 0, st>>>(total, src, dst);
  PD_CK_LAUNCH();
  return 0;
}

struct ShiftedWs {
  char* factors;
  void* rhs;
  void* out;
  SysDesc* sys;
  int* status;
  void* queue;
};

static ShiftedWs plan_shifted(Arena& a, const FactorGeom& g, int nshift, int nrhs, size_t es) {
  ShiftedWs w;
  const size_t fb = factor_bytes(g, es);
  w.factors = a.take<char>(fb * nshift);
  w.rhs = a.take<char>((size_t)g.n * nrhs * es);
  w.out = a.take<char>((size_t)g.n * nrhs * nshift * es);
  w.sys = a.take<SysDesc>(nshift);
  w.status = a.take<int>(nshift);
  w.queue = a.take<char>(solve_queue_bytes(nshift, nrhs));
  return w;
}

template <typename C>
static int shifted_solve(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nshift,
                         const pdeshep_c128* shifts, int nrhs, const double2* d_rhs, int trans, double2* d_x,
                         int32_t* d_ipiv, void* work, size_t wbytes, cudaStream_t st) {
  const FactorGeom g = make_geom(n, b);
  Arena a(work, wbytes);
  ShiftedWs w = plan_shifted(a, g, nshift, nrhs, sizeof(C));
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  const size_t fb = factor_bytes(g, sizeof(C));
  std::vector<SysDesc> sd(nshift);
  for (int s = 0; s < nshift; ++s) {
    sd[s].factor_off = (int64_t)(fb * s);
    sd[s].zre = shifts[s].re;
    sd[s].zim = shifts[s].im;
    sd[s].rhs_off = 0;
    sd[s].out_off = (int64_t)s * n * nrhs;
    sd[s].out2_off = sd[s].out_off;
    sd[s].ncols = nrhs;
    sd[s].pad = 0;
  }
  PD_CK(cudaMemcpyAsync(w.sys, sd.data(), sizeof(SysDesc) * nshift, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_cast<double2, C>(n * nrhs, d_rhs, (C*)w.rhs, st));
  PD_TRY(launch_factor<C>(g, cplx, band, ldab, nshift, w.sys, w.factors, w.status, d_ipiv, st));
  // complex64: the tensor-core solve where its window fits
  const int chunk = (sizeof(C) == sizeof(float2) && solve_tc_supported(g)) ? kTcChunk : 0;
  if (chunk) PD_TRY(solve_tc_error(nullptr, 1, st));
  PD_TRY(launch_solve<C>(g, trans, nshift, sd.data(), w.sys, w.factors, (const C*)w.rhs, (C*)w.out, chunk, w.queue,
                         st));
  PD_TRY(launch_cast<C, double2>(n * nrhs * nshift, (const C*)w.out, d_x, st));
  if (chunk) {
    int e = 0;
    PD_TRY(solve_tc_error(&e, 1, st));
    if (e) return PDESHEP_DEVICE_TIMEOUT;
  }
  std::vector<int> status(nshift);
  PD_CK(cudaMemcpyAsync(status.data(), w.status, sizeof(int) * nshift, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  for (int v : status)
    if (v) return PDESHEP_SINGULAR;
  return 0;
}

// ---------------------------------------------------------------------------
// CholQR on column blocks
// ---------------------------------------------------------------------------
struct CholWs {
  void* G;
  void* I;
  void* Q2;
  void* part;
  int* info;
  SmallDesc* desc;
  void* items;
};

static const int kCholSplits = 8;

static CholWs plan_chol(Arena& a, int64_t n, int nblk, const int32_t* m, size_t es) {
  CholWs w;
  int64_t msq = 0, mtot = 0;
  for (int t = 0; t < nblk; ++t) {
    msq += (int64_t)m[t] * m[t];
    mtot += m[t];
  }
  w.G = a.take<char>(msq * es);
  w.I = a.take<char>(msq * es);
  w.Q2 = a.take<char>(n * mtot * es);
  w.part = a.take<char>(kCholSplits * msq * es);
  w.info = a.take<int>(nblk);
  w.desc = a.take<SmallDesc>(nblk);
  w.items = a.take<GemmItem<double2>>(nblk);
  return w;
}

template <typename S>
static int cholqr(int64_t n, int nblk, const int32_t* m, S* Q, int passes, S* R, void* work, size_t wbytes,
                  cudaStream_t st) {
  Arena a(work, wbytes);
  CholWs w = plan_chol(a, n, nblk, m, sizeof(S));
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  std::vector<int64_t> coff(nblk), soff(nblk);
  int64_t c = 0, so = 0, msq = 0;
  int mm = 0;
  std::vector<SmallDesc> desc(nblk);
  for (int t = 0; t < nblk; ++t) {
    coff[t] = c;
    soff[t] = so;
    desc[t] = SmallDesc{so, c, m[t], 0};
    c += m[t];
    so += (int64_t)m[t] * m[t];
    mm = std::max(mm, (int)m[t]);
  }
  msq = so;
  PD_CK(cudaMemcpyAsync(w.desc, desc.data(), sizeof(SmallDesc) * nblk, cudaMemcpyHostToDevice, st));
  S one, zero;
  if constexpr (std::is_same<S, double>::value) {
    one = 1.0;
    zero = 0.0;
  } else {
    one = make_double2(1.0, 0.0);
    zero = make_double2(0.0, 0.0);
  }
  S* cur = Q;
  S* nxt = (S*)w.Q2;
  for (int pass = 0; pass < passes; ++pass) {
    std::vector<GemmItem<S>> it(nblk);
    for (int t = 0; t < nblk; ++t)
      it[t] = GemmItem<S>{cur + coff[t] * n, cur + coff[t] * n, (S*)w.G + soff[t], m[t], m[t], (int)n, (int)n,
                          (int)n, m[t], soff[t]};
    PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(kCholSplits, n / 512));
    PD_TRY(launch_gemm<S>(true, nblk, (GemmItem<S>*)w.items, mm, mm, (int)n, one, zero, splits, (S*)w.part, msq, st,
                          1, 0));
    PD_TRY(launch_cholesky<S>(nblk, w.desc, (S*)w.G, w.info, st));
    PD_TRY(launch_triinv<S>(nblk, w.desc, (S*)w.G, (S*)w.I, st));
    for (int t = 0; t < nblk; ++t)
      it[t] = GemmItem<S>{cur + coff[t] * n, (S*)w.I + soff[t], nxt + coff[t] * n, (int)n, m[t], m[t], (int)n, m[t],
                          (int)n, 0};
    PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
    PD_TRY(launch_gemm<S>(false, nblk, (GemmItem<S>*)w.items, (int)n, mm, mm, one, zero, 1, (S*)w.part, msq, st,
                          0, 1));
    std::swap(cur, nxt);
  }
  if (cur != Q) PD_CK(cudaMemcpyAsync(Q, cur, sizeof(S) * n * c, cudaMemcpyDeviceToDevice, st));
  if (R) PD_CK(cudaMemcpyAsync(R, w.G, sizeof(S) * msq, cudaMemcpyDeviceToDevice, st));
  std::vector<int> info(nblk);
  PD_CK(cudaMemcpyAsync(info.data(), w.info, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  for (int v : info)
    if (v) return PDESHEP_CHOLQR_BREAKDOWN;
  return 0;
}

// ---------------------------------------------------------------------------
// small Hermitian eigensolver
// ---------------------------------------------------------------------------
template <typename S>
static int eigh(int nblk, const int32_t* m, S* A, double* lam, S* V, void* work, size_t wbytes, cudaStream_t st) {
  Arena a(work, wbytes);
  int64_t msq = 0, mtot = 0;
  for (int t = 0; t < nblk; ++t) {
    msq += (int64_t)m[t] * m[t];
    mtot += m[t];
  }
  EighScratch<S> w = plan_eigh_scratch<S>(a, msq, mtot, nblk);
  SmallDesc* d_desc = a.take<SmallDesc>(nblk);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  std::vector<SmallDesc> desc(nblk);
  int64_t so = 0, vo = 0;
  int mm = 0;
  for (int t = 0; t < nblk; ++t) {
    desc[t] = SmallDesc{so, vo, m[t], 0};
    so += (int64_t)m[t] * m[t];
    vo += m[t];
    mm = std::max(mm, (int)m[t]);
  }
  PD_CK(cudaMemcpyAsync(d_desc, desc.data(), sizeof(SmallDesc) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(eigh_mixed<S>(nblk, d_desc, desc.data(), mm, A, lam, V, w, st));
  std::vector<int> sw(nblk);
  PD_CK(cudaMemcpyAsync(sw.data(), w.sweeps, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  for (int v : sw)
    if (v < 0) return PDESHEP_EIG_NOT_CONVERGED;
  return 0;
}

static size_t eigh_ws(int nblk, const int32_t* m, size_t es) {
  Arena a;
  int64_t msq = 0, mtot = 0;
  for (int t = 0; t < nblk; ++t) {
    msq += (int64_t)m[t] * m[t];
    mtot += m[t];
  }
  if (es == sizeof(double2))
    plan_eigh_scratch<double2>(a, msq, mtot, nblk);
  else
    plan_eigh_scratch<double>(a, msq, mtot, nblk);
  a.take<SmallDesc>(nblk);
  return a.used();
}

}  // namespace pdeshep

using namespace pdeshep;

extern "C" size_t pdeshep_shifted_solve_workspace_size(int64_t n, int32_t b, int32_t nshift, int32_t nrhs,
                                                       int32_t precision) {
  if (n <= 0 || b < 0 || nshift <= 0 || nrhs <= 0) return 0;
  Arena a;
  plan_shifted(a, make_geom(n, b), nshift, nrhs, precision == PDESHEP_MIXED ? sizeof(float2) : sizeof(double2));
  return a.used();
}

extern "C" int pdeshep_shifted_solve(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                     int32_t nshift, const pdeshep_c128* h_shifts, int32_t nrhs,
                                     const pdeshep_c128* d_rhs, int32_t trans, int32_t precision, pdeshep_c128* d_x,
                                     int32_t* d_ipiv, void* d_work, size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (b < 0 || b > n) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (nshift <= 0 || nshift > 65535) return -6;
  if (!h_shifts) return -7;
  if (nrhs <= 0) return -8;
  if (!d_rhs) return -9;
  if (trans != 0 && trans != 1) return -10;
  if (precision != PDESHEP_FP64 && precision != PDESHEP_MIXED) return -11;
  if (!d_x) return -12;
  if (!d_work) return -14;
  const int cplx = is_complex ? 1 : 0;
  if (precision == PDESHEP_MIXED)
    return shifted_solve<float2>(n, b, cplx, d_band, ldab, nshift, h_shifts, nrhs, (const double2*)d_rhs, trans,
                                 (double2*)d_x, d_ipiv, d_work, work_bytes, (cudaStream_t)stream);
  return shifted_solve<double2>(n, b, cplx, d_band, ldab, nshift, h_shifts, nrhs, (const double2*)d_rhs, trans,
                                (double2*)d_x, d_ipiv, d_work, work_bytes, (cudaStream_t)stream);
}

extern "C" int pdeshep_band_matmul(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                   int32_t nrhs, const void* d_x, void* d_y, void* stream) {
  if (n <= 0) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (nrhs <= 0) return -6;
  if (!d_x) return -7;
  if (!d_y) return -8;
  cudaStream_t st = (cudaStream_t)stream;
  if (is_complex)
    PD_TRY(launch_band_matmul<double2>(n, b, d_band, ldab, nrhs, (const double2*)d_x, (double2*)d_y, st));
  else
    PD_TRY(launch_band_matmul<double>(n, b, d_band, ldab, nrhs, (const double*)d_x, (double*)d_y, st));
  PD_CK(cudaStreamSynchronize(st));
  return 0;
}

extern "C" size_t pdeshep_cholqr_workspace_size(int64_t n, int32_t nblk, const int32_t* h_m, int32_t is_complex) {
  if (n <= 0 || nblk <= 0 || !h_m) return 0;
  Arena a;
  plan_chol(a, n, nblk, h_m, is_complex ? sizeof(double2) : sizeof(double));
  return a.used();
}

extern "C" int pdeshep_cholqr(int64_t n, int32_t is_complex, int32_t nblk, const int32_t* h_m, void* d_q,
                              int32_t passes, void* d_r, void* d_work, size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (nblk <= 0) return -3;
  if (!h_m) return -4;
  for (int t = 0; t < nblk; ++t)
    if (h_m[t] < 1 || h_m[t] > n || h_m[t] > 4096) return -4;
  if (!d_q) return -5;
  if (passes < 1 || passes > 3) return -6;
  if (!d_work) return -8;
  cudaStream_t st = (cudaStream_t)stream;
  if (is_complex)
    return cholqr<double2>(n, nblk, h_m, (double2*)d_q, passes, (double2*)d_r, d_work, work_bytes, st);
  return cholqr<double>(n, nblk, h_m, (double*)d_q, passes, (double*)d_r, d_work, work_bytes, st);
}

extern "C" size_t pdeshep_eigh_workspace_size(int32_t nblk, const int32_t* h_m, int32_t is_complex) {
  if (nblk <= 0 || !h_m) return 0;
  return eigh_ws(nblk, h_m, is_complex ? sizeof(double2) : sizeof(double));
}

extern "C" int pdeshep_eigh(int32_t is_complex, int32_t nblk, const int32_t* h_m, void* d_a, double* d_lam,
                            void* d_v, void* d_work, size_t work_bytes, void* stream) {
  if (nblk <= 0) return -2;
  if (!h_m) return -3;
  for (int t = 0; t < nblk; ++t)
    if (h_m[t] < 1 || h_m[t] > 4096) return -3;
  if (!d_a) return -4;
  if (!d_lam) return -5;
  if (!d_v) return -6;
  if (!d_work) return -7;
  cudaStream_t st = (cudaStream_t)stream;
  if (is_complex) return eigh<double2>(nblk, h_m, (double2*)d_a, d_lam, (double2*)d_v, d_work, work_bytes, st);
  return eigh<double>(nblk, h_m, (double*)d_a, d_lam, (double*)d_v, d_work, work_bytes, st);
}

// ---------------------------------------------------------------------------
// ALU throughput probe: every thread runs 8 independent FMA chains of `iters`
// steps (FP32 or FP64), enough warps per SM to hide the FMA latency; the
// result is written so the chains cannot be removed.  TFLOP/s = 2 x FMAs /
// the launch's event time.  Used for the roofline denominators of the
// kernels bound by the FP32 or FP64 pipes.
// ---------------------------------------------------------------------------
namespace {
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T seed, T* out) {
  T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  const T m = (T)0.999999, c = (T)1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = a0 * m + c; a1 = a1 * m + c; a2 = a2 * m + c; a3 = a3 * m + c;
      a4 = a4 * m + c; a5 = a5 * m + c; a6 = a6 * m + c; a7 = a7 * m + c;
    }
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true; keeps the chains
}
}  // namespace

extern "C" int pdeshep_debug_wait_limit(int64_t polls) {
  using namespace pdeshep;
  const int64_t p = polls > 0 ? std::min<int64_t>(polls, 1 << 22) : 0;
  PD_TRY(tc_set_wait_polls((unsigned)p));
  PD_TRY(solve_tc_set_wait_polls((int)p));
  return 0;
}

extern "C" int pdeshep_alu_peak(int32_t fp64, int64_t iters, double* h_tflops, void* d_scratch, void* stream) {
  if (fp64 != 0 && fp64 != 1) return -1;
  if (iters < 1) return -2;
  if (!h_tflops) return -3;
  if (!d_scratch) return -4;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  PD_CK(cudaGetDevice(&dev));
  PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 8 x 256 threads = 64 warps per SM
  cudaEvent_t e0, e1;
  PD_CK(cudaEventCreate(&e0));
  PD_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    PD_CK(cudaEventRecord(e0, st));
    if (fp64)
      fma_probe_kernel<double><<<blocks, 256, 0, st>>>(iters, 1.0, (double*)d_scratch);
    else
      fma_probe_kernel<float><<<blocks, 256, 0, st>>>(iters, 1.0f, (float*)d_scratch);
    PD_CK_LAUNCH();
    PD_CK(cudaEventRecord(e1, st));
    PD_CK(cudaEventSynchronize(e1));
    float ms = 0;
    PD_CK(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double fmas = (double)blocks * 256 * 8 * 16 * (double)iters;
  *h_tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return 0;
}
