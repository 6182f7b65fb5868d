// dense.cuh -- FP64 building blocks of the Rayleigh-Ritz step (Section 2.2 of
// arXiv 2012.00506: A_q = Q^H A Q, A_q W_q = W_q Lambda_q, X = Q W_q) and of
// CholQR: batched GEMM, small Cholesky and triangular inverse, cluster
// parallel Jacobi eigensolver, band-times-block products, column norms.
#pragma once
#include "common.cuh"

namespace pdeshep {

// One product C = alpha op(A) B + beta C of a batch (column-major operands).
// op(A) = A (m x k) or A^H (A stored k x m).  part_off: element offset of this
// item's m x m... partial-sum block when split-K is used.
template <typename S>
struct GemmItem {
  const S* A;
  const S* B;
  S* C;
  int m, n, k;
  int lda, ldb, ldc;
  int64_t part_off;
};

// Launch a batch of products.  splits > 1 splits the k dimension; then `part`
// must hold splits * sum_i(m_i * n_i) elements (deterministic reduction).
template <typename S>
int launch_gemm(bool conjA, int nitems, const GemmItem<S>* d_items, int max_m, int max_n, int max_k,
                S alpha, S beta, int splits, S* part, int64_t part_stride, cudaStream_t st);

// Per-slice small dense kernels.  Blocks of slice t start at offset off[t]
// (elements) with order m[t]; one thread-block cluster per slice.
struct SmallDesc {
  int64_t off;   // element offset of the m x m block
  int64_t voff;  // element offset of the vector block (eigenvalues, m entries)
  int m;
  int pad;
};

// In-place upper Cholesky G = R^H R (upper triangle of G becomes R, lower
// cleared).  info[t] = j+1 if pivot j is not positive.
template <typename S>
int launch_cholesky(int nblk, const SmallDesc* d_desc, S* G, int* info, cudaStream_t st);

// Rinv = R^{-1} for upper triangular R (out of place, same layout).
template <typename S>
int launch_triinv(int nblk, const SmallDesc* d_desc, const S* R, S* Rinv, cudaStream_t st);

// Hermitian Jacobi: A (overwritten), eigenvalues ascending into lam (offset
// voff), eigenvectors into Vout (same layout as A).  Vwork: scratch like A.
// sweeps_out[t]: sweeps used or -1 if max_sweeps hit.
template <typename S>
int launch_jacobi(int nblk, const SmallDesc* d_desc, int max_m, S* A, S* Vwork, S* Vout, double* lam,
                  double tol, int max_sweeps, int* sweeps_out, double* scratch, cudaStream_t st);

// Y = B X for the Hermitian band (lower storage), X, Y n x ncols (ld n).
template <typename S>
int launch_band_matmul(int64_t n, int b, const void* band, int64_t ldab, int ncols, const S* X, S* Y,
                       cudaStream_t st);

}  // namespace pdeshep
