// tcgemm.cu -- FP64-class tall products on the tcgen05 tensor cores (digit
// splitting, TMA operand staging, TMEM accumulators); see tcgemm.cuh for the
// arithmetic.  Kernels:
//   tc_colexp_kernel / tc_split_cols_kernel   columns of n x m blocks -> digit rows (A^H B operands)
//   tc_rowexp_kernel / tc_split_rows_kernel   rows of n x m blocks    -> digit rows (A of A T)
//   tc_split_small_kernel                     columns of m x m blocks -> digit rows (T of A T)
//   tc_gemm_kernel                            128 x 64 real tiles of digit rows times digit rows
//   tc_reduce_kernel, tc_mirror_kernel        split-K sums, Hermitian completion
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "dense.cuh"
#include "tcgemm.cuh"

namespace pdeshep {
namespace {

constexpr int BM = 128;          // rows of A per tile (TMEM lanes)
constexpr int BN = 64;           // rows of B per tile (TMEM columns per accumulator)
constexpr int BK = 32;           // reduction elements per pipeline stage (64-byte swizzled rows)
constexpr int kStages = 3;
constexpr int kChunk = 4;        // stages per exact-level flush (128 elements)
constexpr int kATile = BM * BK * 2;
constexpr int kBTile = BN * BK * 2;
constexpr int kStage = kTcDigits * (kATile + kBTile);
constexpr int kThreads = 320;    // warp 0 TMA, warp 1 MMA (and TMEM owner), warps 2..9 accumulators
constexpr int kSmem = kStages * kStage + 1024 + 256;
constexpr int kMaxKSplit = 16384;  // keeps the integer level sums of one item below 2^31
constexpr uint32_t kTmemCols = 512;  // 5 exact-level accumulators + 1 tail accumulator, 64 columns each
constexpr int kExact = 5;            // digit levels d+d' = 0..4 summed exactly
constexpr int kMaxLevel = 6;         // digit pairs with d+d' > 6 are dropped (below 2^-56 |a||b| each)
constexpr uint32_t kIdesc = (1u << 4)                      // D: FP32
                            | (1u << 7) | (1u << 10)       // A, B: BF16, both K-major
                            | ((uint32_t)(BN >> 3) << 17)  // N
                            | ((uint32_t)(BM >> 4) << 24); // M

__host__ __device__ inline int64_t rup(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// digit splitting
// ---------------------------------------------------------------------------
// exponent e with |x| < 2^e for every x of the row (0 for a zero row)
__device__ inline int row_exponent(double amax) {
  int e = 0;
  if (amax > 0.0) frexp(amax, &e);
  return e;
}

// round(x 2^(47-e)) for |x| < 2^e, by integer operations on the FP64 encoding
// (subnormal x, below 2^-1022, counts as zero)
__device__ inline long long fixed47(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = 1028 + e - E;  // >= 6 because |x| < 2^e
  long long v = sh >= 60 ? 0 : (long long)((m + (1ull << (sh - 1))) >> sh);
  return (u >> 63) ? -v : v;
}

// the six bf16 digits of x (bit patterns): digit d = D_d 2^(-8d), |D_d| <= 128
__device__ inline void digits6(double x, int e, unsigned short (&dg)[kTcDigits]) {
  long long v = fixed47(x, e);
#pragma unroll
  for (int d = kTcDigits - 1; d >= 1; --d) {
    const int r = (int)((v + 128) & 255) - 128;
    v = (v - r) >> 8;
    const float f = (float)r * __int_as_float((127 - 8 * d) << 23);
    dg[d] = (unsigned short)(__float_as_uint(f) >> 16);
  }
  dg[0] = (unsigned short)(__float_as_uint((float)v) >> 16);
}

template <typename S>
struct tcs;
template <>
struct tcs<double> {
  static constexpr int C = 0;
  __device__ static double re(double v) { return v; }
  __device__ static double im(double) { return 0.0; }
};
template <>
struct tcs<double2> {
  static constexpr int C = 1;
  __device__ static double re(double2 v) { return v.x; }
  __device__ static double im(double2 v) { return v.y; }
};

// per listed block of a split launch
struct SplitInfo {
  int64_t x_off;  // operand offset (elements of S)
  int m;          // columns of the block
  int a_row0;     // first digit row of A for this block (-1: no A digits)
  int b_row0;     // first digit row of B (-1: no B digits)
  int k2;         // used reduction length of the rows written (update products)
  int c_off;      // offset of this block's column exponents (update products)
};

// B digit row of output column j (complex: real-part row and, 32 rows later, imaginary-part row)
template <int C>
__device__ inline int brow(int b_row0, int j) {
  return C ? b_row0 + 64 * (j >> 5) + (j & 31) : b_row0 + j;
}

// max |x| over column j of each listed n x m block -> exponents of its A row and B rows
template <typename S>
__global__ void tc_colexp_kernel(int64_t n, const SplitInfo* info, const S* X, int* ea, int* eb) {
  const SplitInfo f = info[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= f.m) return;
  const S* x = X + f.x_off + (int64_t)j * n;
  double mx = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const S v = x[k];
    mx = fmax(mx, fmax(fabs(tcs<S>::re(v)), fabs(tcs<S>::im(v))));
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    const int e = row_exponent(mx);
    constexpr int C = tcs<S>::C;
    if (f.a_row0 >= 0) ea[f.a_row0 + j] = e;
    if (f.b_row0 >= 0) {
      eb[brow<C>(f.b_row0, j)] = e;
      if (C) eb[brow<C>(f.b_row0, j) + 32] = e;
    }
  }
}

// digit rows of the columns: A row j = [Re x_j | Im x_j]; B rows of column j:
// [Re x_j | Im x_j] and [Im x_j | -Re x_j] (so that a.b gives Re and Im of a^H b)
template <typename S>
__global__ void tc_split_cols_kernel(int64_t n, const SplitInfo* info, const S* X, const int* ea, const int* eb,
                                     unsigned short* da, int64_t plane_a, int64_t pitch_a, unsigned short* db,
                                     int64_t plane_b, int64_t pitch_b) {
  constexpr int C = tcs<S>::C;
  const SplitInfo f = info[blockIdx.z];
  const int j = blockIdx.y;
  if (j >= f.m) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const S v = X[f.x_off + (int64_t)j * n + k];
  const int e = f.a_row0 >= 0 ? ea[f.a_row0 + j] : eb[brow<C>(f.b_row0, j)];
  unsigned short dr[kTcDigits], di[kTcDigits];
  digits6(tcs<S>::re(v), e, dr);
  if (C) digits6(tcs<S>::im(v), e, di);
  if (f.a_row0 >= 0) {
    unsigned short* p = da + (int64_t)(f.a_row0 + j) * pitch_a + k;
#pragma unroll
    for (int d = 0; d < kTcDigits; ++d) {
      p[d * plane_a] = dr[d];
      if (C) p[d * plane_a + n] = di[d];
    }
  }
  if (f.b_row0 >= 0) {
    unsigned short* p = db + (int64_t)brow<C>(f.b_row0, j) * pitch_b + k;
#pragma unroll
    for (int d = 0; d < kTcDigits; ++d) {
      p[d * plane_b] = dr[d];
      if (C) {
        p[d * plane_b + n] = di[d];
        p[d * plane_b + 32 * pitch_b] = di[d];
        p[d * plane_b + 32 * pitch_b + n] = dr[d] ^ 0x8000;
      }
    }
  }
}

// Update products A T equilibrate the columns of A first: A T = (A 2^-c)(2^c T) with
// c_k the exponent of column k's maximum (exact power-of-two scaling), so that the
// one fixed-point scale per row of A does not starve columns of small norm (the
// filtered bases of the Rayleigh-Ritz step have columns of very different size).
// The scaling never touches the data: it shifts the digit exponents.
template <typename S>
__global__ void tc_colscale_kernel(int64_t n, const SplitInfo* info, const S* X, int* ec) {
  const SplitInfo f = info[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= f.m) return;
  const S* x = X + f.x_off + (int64_t)j * n;
  double mx = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    const S v = x[k];
    mx = fmax(mx, fmax(fabs(tcs<S>::re(v)), fabs(tcs<S>::im(v))));
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    ec[f.c_off + j] = row_exponent(mx);
  }
}

// max |x(i, c)| 2^-c_c over row i (the block's m columns) -> exponent of A digit row i
template <typename S>
__global__ void tc_rowexp_kernel(int64_t n, const SplitInfo* info, const S* X, const int* ec, int* ea) {
  const SplitInfo f = info[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const S* x = X + f.x_off + i;
  double mx = 0.0;
  for (int c = 0; c < f.m; ++c) {
    const S v = x[(int64_t)c * n];
    mx = fmax(mx, ldexp(fmax(fabs(tcs<S>::re(v)), fabs(tcs<S>::im(v))), -ec[f.c_off + c]));
  }
  ea[f.a_row0 + i] = row_exponent(mx);
}

// digit rows of the rows: A row i = [Re x(i, 0:mp) | Im x(i, 0:mp)] with mp = k2/2
// (complex) or k2 (real) and zeros in columns m..mp-1; 32 x 32 tiles through shared memory
template <typename S>
__global__ void tc_split_rows_kernel(int64_t n, const SplitInfo* info, const S* X, const int* ec, const int* ea,
                                     unsigned short* da, int64_t plane_a, int64_t pitch_a) {
  constexpr int C = tcs<S>::C;
  const SplitInfo f = info[blockIdx.z];
  const int mp = C ? f.k2 / 2 : f.k2;
  const int c0 = blockIdx.y * 32;
  if (c0 >= mp) return;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  __shared__ double sr[32][33], si[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < 32; c += 8) {
    S v{};
    if (i0 + lane < n && c0 + c < f.m) v = X[f.x_off + (int64_t)(c0 + c) * n + i0 + lane];
    sr[lane][c] = tcs<S>::re(v);
    si[lane][c] = tcs<S>::im(v);
  }
  __syncthreads();
  if (c0 + lane >= mp) return;
  const int cs = c0 + lane < f.m ? ec[f.c_off + c0 + lane] : 0;
  for (int r = warp; r < 32; r += 8) {
    const int64_t i = i0 + r;
    if (i >= n) break;
    const int e = ea[f.a_row0 + i] + cs;   // digits of x 2^-c against the row scale
    unsigned short dr[kTcDigits], di[kTcDigits];
    digits6(sr[r][lane], e, dr);
    if (C) digits6(si[r][lane], e, di);
    unsigned short* p = da + (int64_t)(f.a_row0 + i) * pitch_a + c0 + lane;
#pragma unroll
    for (int d = 0; d < kTcDigits; ++d) {
      p[d * plane_a] = dr[d];
      if (C) p[d * plane_a + mp] = di[d];
    }
  }
}

// B digit rows of the columns of an m x m block T (ld m): complex column j gives
// [Re t_j | -Im t_j] and [Im t_j | Re t_j] (so that a.b gives Re and Im of (A T)(i, j))
template <typename S>
__global__ void tc_split_small_kernel(const SplitInfo* info, const S* T, const int* ec, int* eb, unsigned short* db,
                                      int64_t plane_b, int64_t pitch_b) {
  constexpr int C = tcs<S>::C;
  const SplitInfo f = info[blockIdx.y];
  const int j = blockIdx.x;
  if (j >= f.m) return;
  const int mp = C ? f.k2 / 2 : f.k2;
  const S* t = T + f.x_off + (int64_t)j * f.m;
  double mx = 0.0;
  for (int k = threadIdx.x; k < f.m; k += blockDim.x) {
    const S v = t[k];
    mx = fmax(mx, ldexp(fmax(fabs(tcs<S>::re(v)), fabs(tcs<S>::im(v))), ec[f.c_off + k]));
  }
  __shared__ double red[32];
  __shared__ int es;
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    es = row_exponent(mx);
    eb[brow<C>(f.b_row0, j)] = es;
    if (C) eb[brow<C>(f.b_row0, j) + 32] = es;
  }
  __syncthreads();
  const int e = es;
  unsigned short* p = db + (int64_t)brow<C>(f.b_row0, j) * pitch_b;
  for (int k = threadIdx.x; k < mp; k += blockDim.x) {
    S v{};
    int ek = e;
    if (k < f.m) {
      v = t[k];
      ek = e - ec[f.c_off + k];   // digits of t 2^c_k against the column scale
    }
    unsigned short dr[kTcDigits], di[kTcDigits];
    digits6(tcs<S>::re(v), ek, dr);
    if (C) digits6(tcs<S>::im(v), ek, di);
#pragma unroll
    for (int d = 0; d < kTcDigits; ++d) {
      p[d * plane_b + k] = dr[d];
      if (C) {
        p[d * plane_b + mp + k] = di[d] ^ 0x8000;
        p[d * plane_b + 32 * pitch_b + k] = di[d];
        p[d * plane_b + 32 * pitch_b + mp + k] = dr[d];
      }
    }
  }
}

// Band digits.  Row i of the Hermitian band (lower storage, B(i, k) = conj(B(k, i)) above the
// diagonal) over the window k = 128 (i / 128) - lo + w, w < W, of its 128-row tile: exponent
// over the row's band, then the digits ([Re | Im] windows for complex, zeros off the band).
template <typename S>
__device__ inline S band_at(const S* ab, int64_t ldab, int b, int64_t n, int64_t i, int64_t k) {
  if (k < 0 || k >= n || i - k > b || k - i > b) return S{};
  return k <= i ? ab[(i - k) + k * ldab] : sc<S>::conj(ab[(k - i) + i * ldab]);
}
template <typename S>
__global__ void tc_band_rowexp_kernel(int64_t n, int b, const S* ab, int64_t ldab, int* eband) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double mx = 0.0;
  for (int64_t k = max((int64_t)0, i - b); k <= min(n - 1, i + (int64_t)b); ++k) {
    const S v = band_at<S>(ab, ldab, b, n, i, k);
    mx = fmax(mx, fmax(fabs(tcs<S>::re(v)), fabs(tcs<S>::im(v))));
  }
  eband[i] = row_exponent(mx);
}
template <typename S>
__global__ void tc_band_digits_kernel(int64_t n, int b, const S* ab, int64_t ldab, const int* eband, int lo, int W,
                                      unsigned short* dband, int64_t plane, int64_t pitch) {
  constexpr int C = tcs<S>::C;
  const int64_t i = blockIdx.x;
  const int e = i < n ? eband[i] : 0;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    S v{};
    if (i < n) v = band_at<S>(ab, ldab, b, n, i, (i / BM) * BM - lo + w);
    unsigned short dr[kTcDigits], di[kTcDigits];
    digits6(tcs<S>::re(v), e, dr);
    if (C) digits6(tcs<S>::im(v), e, di);
    unsigned short* p = dband + i * pitch + w;
#pragma unroll
    for (int d = 0; d < kTcDigits; ++d) {
      p[d * plane] = dr[d];
      if (C) p[d * plane + W] = di[d];
    }
  }
}
// B rows of the band products: column j of X gives [Re x_j | -Im x_j] and [Im x_j | Re x_j]
// (halves of `half` elements, zero past n), so that a.b gives Re and Im of (B X)(i, j)
template <typename S>
__global__ void tc_split_xcols_kernel(int64_t n, int64_t half, const SplitInfo* info, const S* X, const int* eb,
                                      unsigned short* db, int64_t plane_b, int64_t pitch_b) {
  constexpr int C = tcs<S>::C;
  const SplitInfo f = info[blockIdx.z];
  const int j = blockIdx.y;
  if (j >= f.m) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= half) return;
  S v{};
  if (k < n) v = X[f.x_off + (int64_t)j * n + k];
  const int e = eb[brow<C>(f.b_row0, j)];
  unsigned short dr[kTcDigits], di[kTcDigits];
  digits6(tcs<S>::re(v), e, dr);
  if (C) digits6(tcs<S>::im(v), e, di);
  unsigned short* p = db + (int64_t)brow<C>(f.b_row0, j) * pitch_b + k;
#pragma unroll
  for (int d = 0; d < kTcDigits; ++d) {
    p[d * plane_b] = dr[d];
    if (C) {
      p[d * plane_b + half] = di[d] ^ 0x8000;
      p[d * plane_b + 32 * pitch_b] = di[d];
      p[d * plane_b + 32 * pitch_b + half] = dr[d];
    }
  }
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, TMA, tcgen05
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// polls after which the main waits of tc_gemm_kernel give up (a testing hook lowers it; the
// drains at the end of the kernel always use kDrainPolls)
constexpr unsigned kDrainPolls = 1u << 24;
__device__ unsigned g_tc_wait_polls = kDrainPolls;

// bounded wait for the phase of the given parity; false (and *err set) if it never completes
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, int* err, unsigned polls = kDrainPolls) {
  for (unsigned it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(128);
  }
  atomicExch(err, 1);
  return false;
}
__device__ inline void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ inline uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ inline void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ inline void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// wait for this thread's TMEM loads; the registers pass through so that no use moves above the wait
__device__ inline void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}

// ---------------------------------------------------------------------------
// the product kernel: persistent, one CTA per SM; CTA b takes items b, b + grid, ...
// (each item one 128 x 64 tile of A-rows . B-rows over one k range).  The stage ring,
// the chunk read-outs and the tail hand-over count across items, so the accumulator
// warps store one item's tile while the tensor core runs the next item.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const TcDesc* descs, const TcItem* items, int nitems, int plane_a, int plane_b, const int* ea,
                   const int* eb, S* out, S* part, int* err) {
  constexpr int C = tcs<S>::C;
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(sm + kStages * kStage);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages), accf = smem_u32(bars + 2 * kStages),
                 acce = smem_u32(bars + 2 * kStages + 1), done = smem_u32(bars + 2 * kStages + 2),
                 tfree = smem_u32(bars + 2 * kStages + 3);
  uint32_t* tslot = (uint32_t*)(bars + 2 * kStages + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto stages_of = [&](const TcItem& it, const TcDesc& d, int& k0) {
    k0 = it.split * d.ksplit;
    const int k1 = min(d.k2, k0 + d.ksplit);
    return (int)cdiv(k1 - k0, BK);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 8);
    mbar_init(done, 1);
    mbar_init(tfree, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const unsigned lim = g_tc_wait_polls;

  if (warp == 0) {
    if (lane == 0) {
      // producer: all six digit tiles of A and of B for each stage of 32 reduction elements
      int gs = 0;  // stages issued so far (all items)
      bool ok = true;
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const TcItem it = items[item];
        const TcDesc d = descs[it.desc];
        int k0;
        const int nst = stages_of(it, d, k0);
        const int ya = d.a_row0 + it.tm * BM, yb = d.b_row0 + it.tn * BN;
        for (int s = 0; s < nst; ++s) {
          const int G = gs, slot = G % kStages;
          if (!mbar_wait(empty0 + 8 * slot, ((G / kStages) & 1) ^ 1, err, lim)) { ok = false; break; }
          mbar_expect_tx(full0 + 8 * slot, kStage);
          const uint32_t sa = smem_u32(sm + slot * kStage);
          const int x = k0 + s * BK;
          // band products: the B coordinate follows the tile's window (it may start below 0 or end
          // past the data: TMA fills zeros there, and the band digits are zero outside the band)
          const int xb = d.band ? x + it.tm * BM - d.band_lo + (x >= d.band_w ? d.band_half - d.band_w : 0) : x;
          for (int g = 0; g < kTcDigits; ++g) {
            tma_load_2d(sa + g * kATile, &tmA, x, g * plane_a + ya, full0 + 8 * slot);
            tma_load_2d(sa + kTcDigits * kATile + g * kBTile, &tmB, xb, g * plane_b + yb, full0 + 8 * slot);
          }
          ++gs;
        }
      }
      // every issued copy has landed before the CTA may exit
      for (int G = max(0, gs - kStages); G < gs; ++G) mbar_wait(full0 + 8 * (G % kStages), (G / kStages) & 1, err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issue: 26 digit pairs per 16-element step.  Levels 0..4 go to the exact
      // accumulators (cleared at the start of every 128-element chunk, after the
      // accumulator warps have taken the previous chunk), levels 5..6 to the tail
      // accumulator (cleared at the start of every item, after the accumulator warps
      // have taken the previous item's tail).  The tail products of the chunk's first
      // stages (as many as are buffered) are issued before the wait for the accumulator
      // warps, so the tensor pipe works through the read-out of the previous chunk.
      bool ok = true;
      bool tail_started = false;
      auto tail = [&](int G) {
        const uint64_t da0 = sw64_desc(smem_u32(sm + (G % kStages) * kStage));
        const uint64_t db0 = da0 + ((kTcDigits * kATile) >> 4);
#pragma unroll 1
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int g = 0; g < kTcDigits; ++g) {
#pragma unroll
            for (int h = 0; h < kTcDigits; ++h) {
              if (g + h < kExact || g + h > kMaxLevel) continue;
              tc_mma(tbase + kExact * BN, da0 + ((g * kATile + kk * 32) >> 4), db0 + ((h * kBTile + kk * 32) >> 4),
                     tail_started ? 1u : 0u);
              tail_started = true;
            }
          }
        }
      };
      auto exact = [&](int G, bool first) {
        // descriptors are linear in the address (14-bit field, shared memory < 256 KB)
        const uint64_t da0 = sw64_desc(smem_u32(sm + (G % kStages) * kStage));
        const uint64_t db0 = da0 + ((kTcDigits * kATile) >> 4);
        uint32_t started = first ? 0u : 31u;  // bit L: exact level L already written in this chunk
#pragma unroll 1
        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
          for (int g = 0; g < kExact; ++g) {
#pragma unroll
            for (int h = 0; h < kExact - g; ++h) {
              const int L = g + h;
              tc_mma(tbase + L * BN, da0 + ((g * kATile + kk * 32) >> 4), db0 + ((h * kBTile + kk * 32) >> 4),
                     (started >> L) & 1u);
              started |= 1u << L;
            }
          }
        }
      };
      int gs = 0, gc = 0, ni = 0;  // stages, chunks and items consumed so far
      for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++ni) {
        const TcItem it = items[item];
        const TcDesc d = descs[it.desc];
        int k0;
        const int nst = stages_of(it, d, k0);
        const int nchunk = (int)cdiv(nst, kChunk);
        if (ni > 0) {
          if (!mbar_wait(tfree, (ni - 1) & 1, err, lim)) { ok = false; break; }
          tc_fence_after();
        }
        tail_started = false;
        for (int ch = 0; ch < nchunk && ok; ++ch, ++gc) {
          const int s0 = ch * kChunk, s1 = min(nst, s0 + kChunk);
          const int pre = min(s1 - s0, kStages);  // stages whose tails run ahead of the read-out wait
          for (int s = s0; s < s0 + pre; ++s) {
            const int G = gs + s;
            if (!mbar_wait(full0 + 8 * (G % kStages), (G / kStages) & 1, err, lim)) { ok = false; break; }
            tc_fence_after();
            tail(G);
          }
          if (!ok) break;
          if (gc > 0) {
            if (!mbar_wait(acce, (gc - 1) & 1, err, lim)) { ok = false; break; }
            tc_fence_after();
          }
          for (int s = s0; s < s1; ++s) {
            const int G = gs + s;
            if (s >= s0 + pre) {
              if (!mbar_wait(full0 + 8 * (G % kStages), (G / kStages) & 1, err, lim)) { ok = false; break; }
              tc_fence_after();
              tail(G);
            }
            exact(G, s == s0);
            tc_commit(empty0 + 8 * (G % kStages));
          }
          if (!ok) break;
          tc_commit(accf);
        }
        gs += nst;
      }
      // all MMAs complete before teardown (also on the error path)
      tc_commit(done);
      mbar_wait(done, 0, err);
    }
  } else {
    // accumulator warps: sub-partition p of the TMEM lanes, column half h
    const int p = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lanebase = tbase + ((uint32_t)(32 * p) << 16);
    const int cA = C ? 16 * h : 32 * h, cB = C ? 32 + 16 * h : 32 * h + 16;
    bool ok = true;
    int gc = 0;  // chunks read so far (all items)
    for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
      const TcItem it = items[item];
      const TcDesc d = descs[it.desc];
      int k0;
      const int nst = stages_of(it, d, k0);
      const int nchunk = (int)cdiv(nst, kChunk);
      // exact levels 0..4 of each entry as one integer in units of 2^-32 (|T| < 2^60 for 16384 elements)
      long long T[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) T[q] = 0;
      for (int ch = 0; ch < nchunk; ++ch, ++gc) {
        if (!mbar_wait(accf, gc & 1, err, lim)) { ok = false; break; }
        tc_fence_after();
        // level L holds integer multiples of 2^(-8L), below 2^24 of them: exact in FP32 and in int32
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const uint32_t cc = half ? cB : cA;
          {
            uint32_t r0[16], r1[16], r2[16];
            tmem_ld16(lanebase + 0 * BN + cc, r0);
            tmem_ld16(lanebase + 1 * BN + cc, r1);
            tmem_ld16(lanebase + 2 * BN + cc, r2);
            tmem_wait16(r0);
            tmem_wait16(r1);
            tmem_wait16(r2);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const long long i0 = __float2int_rn(__uint_as_float(r0[q]));
              const long long i1 = __float2int_rn(__uint_as_float(r1[q]) * 256.0f);
              const long long i2 = __float2int_rn(__uint_as_float(r2[q]) * 65536.0f);
              T[16 * half + q] += (i0 << 32) + (i1 << 24) + (i2 << 16);
            }
          }
          {
            uint32_t r3[16], r4[16];
            tmem_ld16(lanebase + 3 * BN + cc, r3);
            tmem_ld16(lanebase + 4 * BN + cc, r4);
            tmem_wait16(r3);
            tmem_wait16(r4);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const long long i3 = __float2int_rn(__uint_as_float(r3[q]) * 16777216.0f);
              const long long i4 = __float2int_rn(__uint_as_float(r4[q]) * 4294967296.0f);
              T[16 * half + q] += (i3 << 8) + i4;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce);
      }
      if (!ok) break;
      // the tail of this item (complete: the last read-out waited for all of its MMAs), then
      // hand the tail accumulator back before the epilogue
      uint32_t ta[16], tb[16];
      tmem_ld16(lanebase + kExact * BN + cA, ta);
      tmem_ld16(lanebase + kExact * BN + cB, tb);
      tmem_wait16(ta);
      tmem_wait16(tb);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tfree);
      const int i = it.tm * BM + 32 * p + lane;
      if (i < d.m) {
        const int er = ea[d.a_row0 + i] - 14;
        const int jb0 = d.b_row0 + it.tn * BN;
        // value of TMEM column group entry q (q < 16: columns cA.., else cB..)
        auto value = [&](int q) -> double {
          const int jb = jb0 + (q < 16 ? cA + q : cB + q - 16);
          const float t3 = __uint_as_float(q < 16 ? ta[q] : tb[q - 16]);
          const double sum = ldexp((double)T[q], -32) + (double)t3;
          return ldexp(sum, er + eb[jb]);
        };
        S* dst = d.nsplit > 1 ? part + d.part_off + (int64_t)it.split * d.m * d.m : out + d.out_off;
        const int64_t ld = d.nsplit > 1 ? d.m : d.ldc;
        if (C) {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int j = it.tn * 32 + 16 * h + q;
            if (j < d.ncols) *(double2*)(dst + i + (int64_t)j * ld) = make_double2(value(q), value(16 + q));
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = it.tn * BN + 32 * h + q;
            if (j < d.ncols) *(double*)(dst + i + (int64_t)j * ld) = value(q);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTmemCols) : "memory");
  }
}

// C = sum of the split partials (upper triangle only when tri), then written with ld ldc
template <typename S>
__global__ void tc_reduce_kernel(const TcDesc* descs, const int* list, S* out, const S* part, int tri) {
  const TcDesc d = descs[list[blockIdx.y]];
  const int64_t mm = (int64_t)d.m * d.m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < mm; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % d.m), j = (int)(idx / d.m);
    if (tri && i > j) continue;
    S acc = part[d.part_off + idx];
    for (int s = 1; s < d.nsplit; ++s) acc = sc<S>::add(acc, part[d.part_off + s * mm + idx]);
    out[d.out_off + i + (int64_t)j * d.ldc] = acc;
  }
}

// C(i, j) = conj(C(j, i)) for i > j; real diagonal
template <typename S>
__global__ void tc_mirror_kernel(const TcDesc* descs, const int* list, S* out) {
  const TcDesc d = descs[list[blockIdx.y]];
  const int64_t mm = (int64_t)d.m * d.m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < mm; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % d.m), j = (int)(idx / d.m);
    if (i > j) out[d.out_off + i + (int64_t)j * d.ldc] = sc<S>::conj(out[d.out_off + j + (int64_t)i * d.ldc]);
    if (i == j) out[d.out_off + i + (int64_t)j * d.ldc] = sc<S>::from_re(sc<S>::re(out[d.out_off + i + (int64_t)j * d.ldc]));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// 2-D map over `rows` digit rows of `k` used elements (row pitch `pitch`), box 32 x box_rows, 64-byte swizzle
int make_map(CUtensorMap* map, void* base, int64_t k, int64_t pitch, int64_t rows, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_last_error_msg("cuTensorMapEncodeTiled is not available from the driver");
    return PDESHEP_CUDA_ERROR;
  }
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error_msg("cuTensorMapEncodeTiled rejected a digit-plane map");
    return PDESHEP_CUDA_ERROR;
  }
  return 0;
}

int rows_b_of(int cplx, int m) { return cplx ? 64 * (int)cdiv(m, 32) : (int)rup(m, 64); }
int k2_update(int cplx, int m) { return cplx ? 2 * (int)rup(m, 16) : (int)rup(m, 32); }

template <typename S>
int launch_products(const TcScratch& w, const CUtensorMap& ma, const CUtensorMap& mb, int plane_a, int plane_b,
                    const std::vector<TcDesc>& hd, const std::vector<TcItem>& hi, const int* ea, S* out,
                    cudaStream_t st) {
  if (hi.empty()) return 0;
  if ((int64_t)hi.size() > w.max_items || (int64_t)hd.size() > w.max_blocks) {
    set_last_error_msg("tensor-core product: item list exceeds its scratch");
    return PDESHEP_WORKSPACE_TOO_SMALL;
  }
  PD_CK(cudaMemcpyAsync(w.desc, hd.data(), sizeof(TcDesc) * hd.size(), cudaMemcpyHostToDevice, st));
  PD_CK(cudaMemcpyAsync(w.items, hi.data(), sizeof(TcItem) * hi.size(), cudaMemcpyHostToDevice, st));
  PD_CK(cudaFuncSetAttribute(tc_gemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    PD_CK(cudaGetDevice(&dev));
    PD_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  const int nitems = (int)hi.size();
  const int grid = std::min(nitems, std::max(1, nsm));  // one CTA per SM (222 KB shared memory each)
  tc_gemm_kernel<S><<<(unsigned)grid, kThreads, kSmem, st>>>(ma, mb, w.desc, w.items, nitems, plane_a, plane_b, ea,
                                                            w.eb, out, (S*)w.part, w.err);
  PD_CK_LAUNCH();
  return 0;
}

}  // namespace

size_t tc_band_bytes(int64_t n, int b, int cplx) {
  const int64_t lo = rup(b, BK), W = BM + 2 * lo;
  return (size_t)(kTcDigits * rup(n, BM) * (cplx ? 2 : 1) * W * 2 + rup(n, BM) * 4 + 1024);
}

TcScratch plan_tc_scratch(Arena& a, const TcShape& sh, int band_b) {
  TcScratch w;
  const int K = (int)sh.m.size();
  const int64_t n = sh.n;
  int64_t ra = 0, rb = 0, ku = 32, tiles_h = 0, tiles_u = 0, part = 0;
  for (int m : sh.m) {
    ra += rup(m, BM);
    rb += rows_b_of(sh.cplx, m);
    ku = std::max<int64_t>(ku, k2_update(sh.cplx, m));
    const int64_t tn = sh.cplx ? cdiv(m, 32) : cdiv(m, 64);
    tiles_h += cdiv(m, BM) * tn;
    tiles_u += cdiv(n, BM) * tn;
    part += (int64_t)m * m;
  }
  w.rows_a = ra;
  w.rows_b = rb;
  w.pitch_a = rup((sh.cplx ? 2 : 1) * n, 8);
  w.pitch_u = ku;
  w.rows_u = (int64_t)K * rup(n, BM);
  w.pitch_b = std::max<int64_t>(w.pitch_a, ku);
  if (band_b >= 0) {
    w.band_lo = rup(band_b, BK);
    w.band_w = BM + 2 * w.band_lo;
    w.band_half = rup(n, BK);
    w.rows_band = rup(n, BM);
    w.pitch_band = (sh.cplx ? 2 : 1) * w.band_w;
    w.pitch_b = std::max<int64_t>(w.pitch_b, (sh.cplx ? 2 : 1) * w.band_half);
  }
  w.max_split = (int)std::max<int64_t>(8, cdiv((sh.cplx ? 2 : 1) * n, kMaxKSplit));
  w.max_blocks = K;
  w.max_items = std::max<int64_t>(tiles_h * w.max_split, tiles_u);
  w.part_elems = part * w.max_split;
  w.da = a.take<unsigned short>((size_t)(kTcDigits * w.rows_a * w.pitch_a));
  w.du = a.take<unsigned short>((size_t)(kTcDigits * w.rows_u * w.pitch_u));
  w.db = a.take<unsigned short>((size_t)(kTcDigits * w.rows_b * w.pitch_b));
  w.ea = a.take<int>((size_t)w.rows_a);
  w.eu = a.take<int>((size_t)w.rows_u);
  w.eb = a.take<int>((size_t)w.rows_b);
  int64_t mtot = 0;
  for (int m : sh.m) mtot += m;
  w.ec = a.take<int>((size_t)mtot);
  w.desc = a.take<TcDesc>((size_t)K);
  w.items = a.take<TcItem>((size_t)w.max_items);
  w.info = a.take<char>((size_t)K * 2 * sizeof(SplitInfo));
  w.list = a.take<int>((size_t)K);
  w.err = a.take<int>(1);
  w.part = a.take<char>((size_t)w.part_elems * (sh.cplx ? 16 : 8));
  if (band_b >= 0) {
    w.dband = a.take<unsigned short>((size_t)(kTcDigits * w.rows_band * w.pitch_band));
    w.eband = a.take<int>((size_t)w.rows_band);
  }
  return w;
}

template <typename S>
int tc_gemm_herm(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                 const std::vector<int64_t>& x_off, const std::vector<int64_t>& c_off, const S* a, const S* b, S* c,
                 bool same_ab, bool reuse_a, bool triangle, cudaStream_t st) {
  constexpr int C = tcs<S>::C;
  const int K = (int)sh.m.size();
  const int64_t n = sh.n;
  const int nl = (int)blocks.size();
  if (!nl) return 0;
  // digit-row offsets of every block (fixed by the shape, whatever subset is listed)
  std::vector<int> a0(K), b0(K);
  for (int t = 0, ra = 0, rb = 0; t < K; ++t) {
    a0[t] = ra;
    b0[t] = rb;
    ra += (int)rup(sh.m[t], BM);
    rb += rows_b_of(C, sh.m[t]);
  }
  int mmax = 0;
  for (int t : blocks) mmax = std::max(mmax, sh.m[t]);
  SplitInfo* dinfo = (SplitInfo*)w.info;
  auto split = [&](const S* x, bool wa, bool wb) -> int {
    std::vector<SplitInfo> inf(nl);
    for (int l = 0; l < nl; ++l) {
      const int t = blocks[l];
      inf[l] = SplitInfo{x_off[t], sh.m[t], wa ? a0[t] : -1, wb ? b0[t] : -1, 0, 0};
    }
    PD_CK(cudaMemcpyAsync(dinfo, inf.data(), sizeof(SplitInfo) * nl, cudaMemcpyHostToDevice, st));
    tc_colexp_kernel<S><<<dim3(mmax, nl), 256, 0, st>>>(n, dinfo, x, w.ea, w.eb);
    PD_CK_LAUNCH();
    tc_split_cols_kernel<S><<<dim3((unsigned)cdiv(n, 256), mmax, nl), 256, 0, st>>>(
        n, dinfo, x, w.ea, w.eb, w.da, w.rows_a * w.pitch_a, w.pitch_a, w.db, w.rows_b * w.pitch_b, w.pitch_b);
    PD_CK_LAUNCH();
    return 0;
  };
  if (same_ab) {
    PD_TRY(split(a, true, true));
  } else {
    if (!reuse_a) PD_TRY(split(a, true, false));
    PD_TRY(split(b, false, true));
  }
  // tiles and split-K
  const int k2 = (int)((C ? 2 : 1) * n);
  int64_t tiles = 0;
  auto tile_kept = [&](int m, int tm, int tn) {
    const int cw = C ? 32 : 64;
    return !triangle || (int64_t)cw * tn + cw - 1 >= (int64_t)BM * tm;
  };
  for (int t : blocks) {
    const int m = sh.m[t], tn_n = (int)(C ? cdiv(m, 32) : cdiv(m, 64));
    for (int tm = 0; tm < cdiv(m, BM); ++tm)
      for (int tn = 0; tn < tn_n; ++tn) tiles += tile_kept(m, tm, tn);
  }
  int nsplit = (int)std::max<int64_t>(1, cdiv(2 * 152, std::max<int64_t>(1, tiles)));
  nsplit = std::min(nsplit, (int)std::max<int64_t>(1, cdiv(k2, 512)));
  nsplit = std::max<int>(nsplit, (int)cdiv(k2, kMaxKSplit));
  nsplit = std::min(nsplit, w.max_split);
  const int ksplit = (int)rup(cdiv(k2, nsplit), kChunk * BK);
  nsplit = (int)cdiv(k2, ksplit);
  std::vector<TcDesc> hd(nl);
  std::vector<TcItem> hi;
  std::vector<int> lst(nl);
  int64_t poff = 0;
  for (int l = 0; l < nl; ++l) {
    const int t = blocks[l], m = sh.m[t];
    TcDesc& d = hd[l];
    d.a_row0 = a0[t];
    d.b_row0 = b0[t];
    d.m = m;
    d.ncols = m;
    d.k2 = k2;
    d.ksplit = ksplit;
    d.nsplit = nsplit;
    d.ldc = m;
    d.out_off = c_off[t];
    d.part_off = poff;
    poff += (int64_t)nsplit * m * m;
    lst[l] = l;
    const int tn_n = (int)(C ? cdiv(m, 32) : cdiv(m, 64));
    for (int tm = 0; tm < cdiv(m, BM); ++tm)
      for (int tn = 0; tn < tn_n; ++tn)
        if (tile_kept(m, tm, tn))
          for (int s = 0; s < nsplit; ++s) hi.push_back(TcItem{l, tm, tn, s});
  }
  if (poff > w.part_elems) {
    set_last_error_msg("tensor-core product: split partials exceed their scratch");
    return PDESHEP_WORKSPACE_TOO_SMALL;
  }
  CUtensorMap ma, mb;
  PD_TRY(make_map(&ma, w.da, k2, w.pitch_a, kTcDigits * w.rows_a, BM));
  PD_TRY(make_map(&mb, w.db, k2, w.pitch_b, kTcDigits * w.rows_b, BN));
  PD_TRY(launch_products<S>(w, ma, mb, (int)w.rows_a, (int)w.rows_b, hd, hi, w.ea, c, st));
  if (nsplit > 1 || triangle) PD_CK(cudaMemcpyAsync(w.list, lst.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, st));
  if (nsplit > 1) {
    const int g = (int)std::min<int64_t>(256, cdiv((int64_t)mmax * mmax, 256));
    tc_reduce_kernel<S><<<dim3(g, nl), 256, 0, st>>>(w.desc, w.list, c, (const S*)w.part, triangle ? 1 : 0);
    PD_CK_LAUNCH();
  }
  if (triangle) {
    const int g = (int)std::min<int64_t>(256, cdiv((int64_t)mmax * mmax, 256));
    tc_mirror_kernel<S><<<dim3(g, nl), 256, 0, st>>>(w.desc, w.list, c);
    PD_CK_LAUNCH();
  }
  return 0;
}

template <typename S>
int tc_gemm_update(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                   const std::vector<int64_t>& x_off, const std::vector<int64_t>& t_off, const S* a, const S* tm,
                   S* c, cudaStream_t st) {
  constexpr int C = tcs<S>::C;
  const int K = (int)sh.m.size();
  const int64_t n = sh.n, npad = rup(n, BM);
  const int nl = (int)blocks.size();
  if (!nl) return 0;
  std::vector<int> b0(K);
  for (int t = 0, rb = 0; t < K; ++t) {
    b0[t] = rb;
    rb += rows_b_of(C, sh.m[t]);
  }
  int mmax = 0, kmax = 0;
  for (int t : blocks) {
    mmax = std::max(mmax, sh.m[t]);
    kmax = std::max(kmax, k2_update(C, sh.m[t]));
  }
  SplitInfo* dinfo = (SplitInfo*)w.info;
  std::vector<int> c0(K);
  for (int t = 0, c = 0; t < K; ++t) {
    c0[t] = c;
    c += sh.m[t];
  }
  std::vector<SplitInfo> inf(nl);
  for (int l = 0; l < nl; ++l) {
    const int t = blocks[l];
    inf[l] = SplitInfo{x_off[t], sh.m[t], (int)(t * npad), b0[t], k2_update(C, sh.m[t]), c0[t]};
  }
  PD_CK(cudaMemcpyAsync(dinfo, inf.data(), sizeof(SplitInfo) * nl, cudaMemcpyHostToDevice, st));
  tc_colscale_kernel<S><<<dim3(mmax, nl), 256, 0, st>>>(n, dinfo, a, w.ec);
  PD_CK_LAUNCH();
  tc_rowexp_kernel<S><<<dim3((unsigned)cdiv(n, 256), nl), 256, 0, st>>>(n, dinfo, a, w.ec, w.eu);
  PD_CK_LAUNCH();
  const int mpmax = C ? kmax / 2 : kmax;
  tc_split_rows_kernel<S><<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(mpmax, 32), nl), 256, 0, st>>>(
      n, dinfo, a, w.ec, w.eu, w.du, w.rows_u * w.pitch_u, w.pitch_u);
  PD_CK_LAUNCH();
  // T digits: the SplitInfo offsets point into the small blocks
  std::vector<SplitInfo> tinf(inf);
  for (int l = 0; l < nl; ++l) tinf[l].x_off = t_off[blocks[l]];
  SplitInfo* dtinf = dinfo + nl;
  PD_CK(cudaMemcpyAsync(dtinf, tinf.data(), sizeof(SplitInfo) * nl, cudaMemcpyHostToDevice, st));
  tc_split_small_kernel<S><<<dim3(mmax, nl), 128, 0, st>>>(dtinf, tm, w.ec, w.eb, w.db, w.rows_b * w.pitch_u,
                                                           w.pitch_u);
  PD_CK_LAUNCH();
  std::vector<TcDesc> hd(nl);
  std::vector<TcItem> hi;
  for (int l = 0; l < nl; ++l) {
    const int t = blocks[l], m = sh.m[t];
    TcDesc& d = hd[l];
    d.a_row0 = (int)(t * npad);
    d.b_row0 = b0[t];
    d.m = (int)n;
    d.ncols = m;
    d.k2 = k2_update(C, m);
    d.ksplit = d.k2;
    d.nsplit = 1;
    d.ldc = (int)n;
    d.out_off = x_off[t];
    d.part_off = 0;
    const int tn_n = (int)(C ? cdiv(m, 32) : cdiv(m, 64));
    for (int tn = 0; tn < tn_n; ++tn)
      for (int tmi = 0; tmi < cdiv(n, BM); ++tmi) hi.push_back(TcItem{l, tmi, tn, 0});
  }
  CUtensorMap ma, mb;
  PD_TRY(make_map(&ma, w.du, w.pitch_u, w.pitch_u, kTcDigits * w.rows_u, BM));
  PD_TRY(make_map(&mb, w.db, w.pitch_u, w.pitch_u, kTcDigits * w.rows_b, BN));
  return launch_products<S>(w, ma, mb, (int)w.rows_u, (int)w.rows_b, hd, hi, w.eu, c, st);
}

template <typename S>
int tc_band_split(const TcScratch& w, int64_t n, int b, const void* band, int64_t ldab, cudaStream_t st) {
  if (!w.dband) {
    set_last_error_msg("tensor-core band product: scratch planned without the band");
    return PDESHEP_WORKSPACE_TOO_SMALL;
  }
  tc_band_rowexp_kernel<S><<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, b, (const S*)band, ldab, w.eband);
  PD_CK_LAUNCH();
  tc_band_digits_kernel<S><<<(unsigned)w.rows_band, 128, 0, st>>>(
      n, b, (const S*)band, ldab, w.eband, (int)w.band_lo, (int)w.band_w, w.dband, w.rows_band * w.pitch_band,
      w.pitch_band);
  PD_CK_LAUNCH();
  return 0;
}

template <typename S>
int tc_band_matmul(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                   const std::vector<int64_t>& x_off, const S* X, S* Y, cudaStream_t st) {
  constexpr int C = tcs<S>::C;
  const int K = (int)sh.m.size();
  const int64_t n = sh.n;
  const int nl = (int)blocks.size();
  if (!nl) return 0;
  std::vector<int> b0(K);
  for (int t = 0, rb = 0; t < K; ++t) {
    b0[t] = rb;
    rb += rows_b_of(C, sh.m[t]);
  }
  int mmax = 0;
  for (int t : blocks) mmax = std::max(mmax, sh.m[t]);
  const int64_t pitch = (C ? 2 : 1) * w.band_half;
  SplitInfo* dinfo = (SplitInfo*)w.info;
  std::vector<SplitInfo> inf(nl);
  for (int l = 0; l < nl; ++l) {
    const int t = blocks[l];
    inf[l] = SplitInfo{x_off[t], sh.m[t], -1, b0[t], 0, 0};
  }
  PD_CK(cudaMemcpyAsync(dinfo, inf.data(), sizeof(SplitInfo) * nl, cudaMemcpyHostToDevice, st));
  tc_colexp_kernel<S><<<dim3(mmax, nl), 256, 0, st>>>(n, dinfo, X, w.ea, w.eb);
  PD_CK_LAUNCH();
  tc_split_xcols_kernel<S><<<dim3((unsigned)cdiv(w.band_half, 256), mmax, nl), 256, 0, st>>>(
      n, w.band_half, dinfo, X, w.eb, w.db, w.rows_b * pitch, pitch);
  PD_CK_LAUNCH();
  std::vector<TcDesc> hd(nl);
  std::vector<TcItem> hi;
  const int k2 = (int)((C ? 2 : 1) * w.band_w);
  for (int l = 0; l < nl; ++l) {
    const int t = blocks[l], m = sh.m[t];
    TcDesc& d = hd[l];
    d = TcDesc{};
    d.a_row0 = 0;
    d.b_row0 = b0[t];
    d.m = (int)n;
    d.ncols = m;
    d.k2 = k2;
    d.ksplit = k2;
    d.nsplit = 1;
    d.ldc = (int)n;
    d.out_off = x_off[t];
    d.band = 1;
    d.band_lo = (int)w.band_lo;
    d.band_w = (int)w.band_w;
    d.band_half = (int)w.band_half;
    const int tn_n = (int)(C ? cdiv(m, 32) : cdiv(m, 64));
    for (int tn = 0; tn < tn_n; ++tn)
      for (int tmi = 0; tmi < cdiv(n, BM); ++tmi) hi.push_back(TcItem{l, tmi, tn, 0});
  }
  CUtensorMap ma, mb;
  PD_TRY(make_map(&ma, w.dband, k2, w.pitch_band, kTcDigits * w.rows_band, BM));
  PD_TRY(make_map(&mb, w.db, pitch, pitch, kTcDigits * w.rows_b, BN));
  return launch_products<S>(w, ma, mb, (int)w.rows_band, (int)w.rows_b, hd, hi, w.eband, Y, st);
}

int tc_set_wait_polls(unsigned polls) {
  const unsigned v = polls ? polls : kDrainPolls;
  PD_CK(cudaMemcpyToSymbol(g_tc_wait_polls, &v, sizeof(v)));
  return 0;
}

int tc_read_error(const TcScratch& w, cudaStream_t st) {
  int e = 0;
  PD_CK(cudaMemcpyAsync(&e, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  return e ? PDESHEP_DEVICE_TIMEOUT : 0;
}

int tc_clear_error(const TcScratch& w, cudaStream_t st) {
  PD_CK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  return 0;
}

template int tc_gemm_herm<double>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                  const std::vector<int64_t>&, const std::vector<int64_t>&, const double*,
                                  const double*, double*, bool, bool, bool, cudaStream_t);
template int tc_gemm_herm<double2>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                   const std::vector<int64_t>&, const std::vector<int64_t>&, const double2*,
                                   const double2*, double2*, bool, bool, bool, cudaStream_t);
template int tc_band_split<double>(const TcScratch&, int64_t, int, const void*, int64_t, cudaStream_t);
template int tc_band_split<double2>(const TcScratch&, int64_t, int, const void*, int64_t, cudaStream_t);
template int tc_band_matmul<double>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                    const std::vector<int64_t>&, const double*, double*, cudaStream_t);
template int tc_band_matmul<double2>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                     const std::vector<int64_t>&, const double2*, double2*, cudaStream_t);
template int tc_gemm_update<double>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                    const std::vector<int64_t>&, const std::vector<int64_t>&, const double*,
                                    const double*, double*, cudaStream_t);
template int tc_gemm_update<double2>(const TcScratch&, const TcShape&, const std::vector<int>&,
                                     const std::vector<int64_t>&, const std::vector<int64_t>&, const double2*,
                                     const double2*, double2*, cudaStream_t);


// ---------------------------------------------------------------------------
// C ABI: batched block products (FP64, float-float or tensor-core digits)
// ---------------------------------------------------------------------------
namespace {
struct BlockGemmWs {
  TcScratch tc;
  void* items;
  void* part;
  int64_t part_elems;
};
BlockGemmWs plan_block_gemm(Arena& a, int64_t n, int cplx, int nblk, const int32_t* m) {
  BlockGemmWs w;
  TcShape sh{n, cplx, std::vector<int>(m, m + nblk)};
  w.tc = plan_tc_scratch(a, sh);
  w.items = a.take<char>((size_t)nblk * sizeof(GemmItem<double2>));
  int64_t mm = 0;
  for (int t = 0; t < nblk; ++t) mm += (int64_t)m[t] * m[t];
  w.part_elems = 8 * mm;
  w.part = a.take<char>((size_t)w.part_elems * (cplx ? 16 : 8));
  return w;
}

template <typename S>
int block_gemm(int kind, int arith, int64_t n, int nblk, const int32_t* hm, const S* A, const S* B, S* Cm,
               void* work, size_t work_bytes, cudaStream_t st) {
  Arena a(work, work_bytes);
  BlockGemmWs w = plan_block_gemm(a, n, std::is_same<S, double2>::value ? 1 : 0, nblk, hm);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  std::vector<int64_t> xo(nblk), so(nblk);
  std::vector<int> blocks(nblk);
  int mmax = 0;
  for (int t = 0, c = 0; t < nblk; ++t) {
    xo[t] = (int64_t)c * n;
    so[t] = t ? so[t - 1] + (int64_t)hm[t - 1] * hm[t - 1] : 0;
    c += hm[t];
    blocks[t] = t;
    mmax = std::max(mmax, (int)hm[t]);
  }
  if (arith == PDESHEP_RR_TENSOR) {
    TcShape sh{n, std::is_same<S, double2>::value ? 1 : 0, std::vector<int>(hm, hm + nblk)};
    PD_TRY(tc_clear_error(w.tc, st));
    if (kind == PDESHEP_GEMM_UPDATE)
      PD_TRY(tc_gemm_update<S>(w.tc, sh, blocks, xo, so, A, B, Cm, st));
    else
      PD_TRY(tc_gemm_herm<S>(w.tc, sh, blocks, xo, so, A, kind == PDESHEP_GEMM_GRAM ? A : B, Cm,
                             kind == PDESHEP_GEMM_GRAM, false, kind == PDESHEP_GEMM_GRAM, st));
    return tc_read_error(w.tc, st);
  }
  std::vector<GemmItem<S>> it(nblk);
  for (int t = 0; t < nblk; ++t) {
    GemmItem<S>& x = it[t];
    const int m = hm[t];
    if (kind == PDESHEP_GEMM_UPDATE) {
      x = GemmItem<S>{A + xo[t], B + so[t], Cm + xo[t], (int)n, m, m, (int)n, m, (int)n, 0};
    } else {
      x = GemmItem<S>{A + xo[t], (kind == PDESHEP_GEMM_GRAM ? A : B) + xo[t], Cm + so[t], m, m, (int)n, (int)n,
                      (int)n, m, so[t]};
    }
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  S one{}, zero{};
  if constexpr (std::is_same<S, double>::value) one = 1.0; else one = make_double2(1.0, 0.0);
  const int ff = arith == PDESHEP_RR_FLOATFLOAT ? 1 : 0;
  if (kind == PDESHEP_GEMM_UPDATE)
    PD_TRY(launch_gemm<S>(false, nblk, (const GemmItem<S>*)w.items, (int)n, mmax, mmax, one, zero, 1, (S*)w.part,
                          0, st, 0, 0, ff));
  else
    PD_TRY(launch_gemm<S>(true, nblk, (const GemmItem<S>*)w.items, mmax, mmax, (int)n, one, zero, 8, (S*)w.part,
                          w.part_elems / 8, st, kind == PDESHEP_GEMM_GRAM ? 1 : 0, 0, ff));
  PD_CK(cudaStreamSynchronize(st));
  return 0;
}
}  // namespace

extern "C" size_t pdeshep_band_matmul_tc_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t ncols) {
  if (n <= 0 || b < 0 || ncols <= 0) return 0;
  Arena a;
  int32_t m = ncols;
  plan_tc_scratch(a, TcShape{n, is_complex ? 1 : 0, std::vector<int>(1, m)}, b);
  return a.used();
}

extern "C" int pdeshep_band_matmul_tc(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                      int32_t ncols, const void* d_x, void* d_y, void* d_work, size_t work_bytes,
                                      void* stream) {
  if (n <= 0 || n > (int64_t)1 << 30) return -1;
  if (b < 0 || b >= n) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (ncols < 1 || ncols > 4096 || ncols > n) return -6;
  if (!d_x) return -7;
  if (!d_y) return -8;
  if (!d_work) return -9;
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(d_work, work_bytes);
  const TcShape sh{n, is_complex ? 1 : 0, std::vector<int>(1, (int)ncols)};
  TcScratch w = plan_tc_scratch(a, sh, b);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  PD_TRY(tc_clear_error(w, st));
  const std::vector<int> blocks(1, 0);
  const std::vector<int64_t> xo(1, 0);
  if (is_complex) {
    PD_TRY(tc_band_split<double2>(w, n, b, d_band, ldab, st));
    PD_TRY(tc_band_matmul<double2>(w, sh, blocks, xo, (const double2*)d_x, (double2*)d_y, st));
  } else {
    PD_TRY(tc_band_split<double>(w, n, b, d_band, ldab, st));
    PD_TRY(tc_band_matmul<double>(w, sh, blocks, xo, (const double*)d_x, (double*)d_y, st));
  }
  return tc_read_error(w, st);
}

extern "C" size_t pdeshep_block_gemm_workspace_size(int64_t n, int32_t is_complex, int32_t nblk,
                                                    const int32_t* h_m) {
  if (n <= 0 || nblk <= 0 || !h_m) return 0;
  Arena a;
  plan_block_gemm(a, n, is_complex ? 1 : 0, nblk, h_m);
  return a.used();
}

extern "C" int pdeshep_block_gemm(int32_t kind, int32_t arith, int64_t n, int32_t is_complex, int32_t nblk,
                                  const int32_t* h_m, const void* d_a, const void* d_b, void* d_c, void* d_work,
                                  size_t work_bytes, void* stream) {
  if (kind < PDESHEP_GEMM_AHB || kind > PDESHEP_GEMM_UPDATE) return -1;
  if (arith < PDESHEP_RR_FLOATFLOAT || arith > PDESHEP_RR_TENSOR) return -2;
  if (n <= 0 || n > (int64_t)1 << 30) return -3;
  if (nblk <= 0) return -5;
  if (!h_m) return -6;
  for (int t = 0; t < nblk; ++t)
    if (h_m[t] < 1 || h_m[t] > n || h_m[t] > 4096) return -6;
  if (!d_a) return -7;
  if (kind != PDESHEP_GEMM_GRAM && !d_b) return -8;
  if (!d_c) return -9;
  if (!d_work) return -10;
  cudaStream_t st = (cudaStream_t)stream;
  if (is_complex)
    return block_gemm<double2>(kind, arith, n, nblk, h_m, (const double2*)d_a, (const double2*)d_b, (double2*)d_c,
                               d_work, work_bytes, st);
  return block_gemm<double>(kind, arith, n, nblk, h_m, (const double*)d_a, (const double*)d_b, (double*)d_c, d_work,
                            work_bytes, st);
}

}  // namespace pdeshep
