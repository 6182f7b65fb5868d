// tcgemm.cuh -- FP64-class tall products of the Rayleigh-Ritz step (Section 2.2
// of arXiv 2012.00506: the Gram matrix Q^H Q of CholQR, the projection
// Q^H (B Q) and the basis update Q W) on the tcgen05 tensor cores.
//
// Operands are split into six bf16 "digits" per FP64 value with one power-of-two
// scale per row of the reduction (an error-free splitting in the manner of
// Ozaki et al., 2012): with |x| < 2^e, V = round(x 2^(47-e)) is written in
// balanced base 256, V = sum_d D_d 256^(5-d) with |D_d| <= 128, and digit d is
// stored as the bf16 value D_d 2^(-8d) (exact: at most 8 significant bits).
// The product of rows a, b is then
//     a.b ~ 2^(ea+eb-14) sum_{d+d' <= 6} sum_k Da_d(k) Db_d'(k)
// (26 digit pairs; the pairs with d+d' > 6 are dropped, each below 2^-56 of
// |a||b|; stopping at d+d' <= 5 would leave a systematic 2^-48-level bias in
// Gram diagonals from the dropped squares of digit 3).  Every digit product is
// exact in the tensor core's FP32 accumulator, but the accumulation itself is
// not correctly rounded (measured: a bias that grows with the number of
// accumulations), so the five leading levels d+d' = 0..4 are kept in separate
// TMEM accumulators and moved to integer registers every 128 k, while their
// sums are still exact integers (below 2^24 units of the level); the
// accumulation order and rounding of the tensor core never touch them.  Only
// the levels 5 and 6 (2^-40 of the result) share one FP32 accumulator over the
// whole range.  The error is then set by the rounding of the digits (2^-48 of
// the row maximum per element): about 1e-15 |a| |b| per entry.
//
// Complex products are real products with twice the reduction length: a row
// of op(A) holds [Re | Im] of an A row and every complex output column j is
// two rows of the B digit array, [Re-coefficients | Im-coefficients], placed
// 32 rows apart in each 64-row tile, so that one thread ends up with the real
// and imaginary part of the same output entry.
#pragma once
#include <vector>

#include "common.cuh"

namespace pdeshep {

constexpr int kTcDigits = 6;

// One block product of the batch.
struct TcDesc {
  int a_row0;      // first row of this block in each digit plane of A
  int b_row0;      // first row in each digit plane of B
  int m;           // output rows
  int ncols;       // output columns (complex or real)
  int k2;          // reduction length in digit-array elements (2 k for complex)
  int ksplit;      // reduction elements per split (multiple of 128)
  int nsplit;
  int ldc;
  int64_t out_off; // element offset of the output block
  int64_t part_off;// element offset of split 0 in the partial buffer (nsplit > 1), layout as the output with ld m
  // band products: A rows hold the band of 128-row tile tm over the window of W columns starting
  // at 128 tm - band_lo ([Re | Im] windows for complex), B rows hold whole columns of X
  // ([Re | -Im] and [Im | Re] halves of band_half elements each); 0 for the other products
  int band, band_lo, band_w, band_half;
};
struct TcItem {
  int desc, tm, tn, split;
};

// Scratch of the tensor-core products: digit planes of the operands, row
// exponents, descriptors and split-K partials.
struct TcScratch {
  unsigned short* da = nullptr;  // A^H B: A digit rows (kTcDigits planes of rows_a x pitch_a bf16)
  unsigned short* du = nullptr;  // A T: A digit rows (planes of rows_u x pitch_u)
  unsigned short* db = nullptr;  // B digit rows of either product (planes of rows_b x pitch)
  unsigned short* dband = nullptr;  // band digit rows (planes of rows_band x pitch_band), see tc_band_split
  int* eband = nullptr;
  int* ea = nullptr;
  int* eu = nullptr;
  int* eb = nullptr;
  int* ec = nullptr;             // column exponents of the A operand of A T (equilibration)
  TcDesc* desc = nullptr;
  TcItem* items = nullptr;
  char* info = nullptr;          // per-block split descriptors
  int* list = nullptr;
  int* err = nullptr;            // set by a bounded wait that gave up
  void* part = nullptr;
  int64_t rows_a = 0, rows_b = 0, rows_u = 0, pitch_a = 0, pitch_b = 0, pitch_u = 0;
  int64_t rows_band = 0, pitch_band = 0, band_lo = 0, band_w = 0, band_half = 0;
  int64_t max_items = 0, max_blocks = 0, part_elems = 0;
  int max_split = 1;
};

// Sizes: n rows of the tall operands, blocks of m[t] columns, complex or real.
struct TcShape {
  int64_t n;
  int cplx;
  std::vector<int> m;
};
TcScratch plan_tc_scratch(Arena& a, const TcShape& sh, int band_b = -1);  // band_b >= 0: band products too

// C_t = A_t^H B_t (m_t x m_t, ld ldc[t], at c + c_off[t]) for the listed blocks; A_t, B_t are n x m_t
// column-major at a + x_off[t], b + x_off[t].  same_ab: B is A (the Gram matrix; one split pass).
// reuse_a: the A digits of the previous call with the same blocks and A are still valid.
// triangle: only tiles on or above the diagonal are computed (Hermitian output, lower part mirrored).
template <typename S>
int tc_gemm_herm(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                 const std::vector<int64_t>& x_off, const std::vector<int64_t>& c_off, const S* a, const S* b, S* c,
                 bool same_ab, bool reuse_a, bool triangle, cudaStream_t st);
// C_t = A_t T_t (n x m_t at c + x_off[t]) with A_t n x m_t at a + x_off[t] and T_t m_t x m_t (ld m_t)
// at t + t_off[t].
template <typename S>
int tc_gemm_update(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                   const std::vector<int64_t>& x_off, const std::vector<int64_t>& t_off, const S* a, const S* tm,
                   S* c, cudaStream_t st);

// Band products Y_t = B X_t (B Hermitian band, lower storage; X_t, Y_t n x m_t at x_off[t]):
// tc_band_split writes the digits of B once (rows of 128-row tiles over their band window),
// tc_band_matmul splits the columns of X and runs one tile per (128 rows, 32 or 64 columns).
template <typename S>
int tc_band_split(const TcScratch& w, int64_t n, int b, const void* band, int64_t ldab, cudaStream_t st);
template <typename S>
int tc_band_matmul(const TcScratch& w, const TcShape& sh, const std::vector<int>& blocks,
                   const std::vector<int64_t>& x_off, const S* X, S* Y, cudaStream_t st);
size_t tc_band_bytes(int64_t n, int b, int cplx);

// PDESHEP_DEVICE_TIMEOUT if a product kernel's bounded wait gave up since the last clear (synchronises)
int tc_read_error(const TcScratch& w, cudaStream_t st);
int tc_set_wait_polls(unsigned polls);  // 0: the default
int tc_clear_error(const TcScratch& w, cudaStream_t st);

}  // namespace pdeshep
