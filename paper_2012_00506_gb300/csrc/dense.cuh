// dense.cuh -- FP64 building blocks of the Rayleigh-Ritz step (Section 2.2 of
// arXiv 2012.00506: A_q = Q^H A Q, A_q W_q = W_q Lambda_q, X = Q W_q) and of
// CholQR: batched GEMM, small Cholesky and triangular inverse, cluster
// parallel Jacobi eigensolver, band-times-block products, column norms.
#pragma once
#include <vector>

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
// herm: output Hermitian (only upper tiles computed, lower mirrored); triB: B upper triangular.
// ff: float-float arithmetic on the FP32 pipes (about 48-bit products, FP32 exponent range)
// instead of FP64.
template <typename S>
int launch_gemm(bool conjA, int nitems, const GemmItem<S>* d_items, int max_m, int max_n, int max_k,
                S alpha, S beta, int splits, S* part, int64_t part_stride, cudaStream_t st, int herm = 0,
                int triB = 0, int ff = 0);

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
// diag0 (optional, vector layout voff) receives the diagonal of G before factorization and
// minratio[t] (optional) = min_c R(c,c)^2 / G(c,c): the squared sine of the smallest angle
// between a column and the span of the ones before it.
template <typename S>
int launch_cholesky(int nblk, const SmallDesc* d_desc, S* G, int* info, cudaStream_t st,
                    double* diag0 = nullptr, double* minratio = nullptr);

// Rinv = R^{-1} for upper triangular R (out of place, same layout).
int cluster_ctas_used();
template <typename S>
int launch_triinv(int nblk, const SmallDesc* d_desc, const S* R, S* Rinv, cudaStream_t st);

// Hermitian Jacobi: A and Aalt (scratch like A) are overwritten, eigenvalues
// ascending into lam (offset voff), eigenvectors into Vout (same layout as A).
// Vwork: scratch like A.  sweeps_out[t]: sweeps used or -1 if max_sweeps hit.
template <typename S>
int launch_jacobi(int nblk, const SmallDesc* d_desc, int max_m, S* A, S* Aalt, S* Vwork, S* Vout, double* lam,
                  double tol, int max_sweeps, int* sweeps_out, double* scratch, cudaStream_t st);

// Mixed-precision small Hermitian eigensolver: FP32 Jacobi gives V32 (blocks
// already close to diagonal start from I instead), FP64 Ogita-Aishima
// refinement steps (batched GEMMs over all SMs) bring V to FP64 accuracy, and
// blocks left with an unresolved cluster finish with FP64 Jacobi sweeps on
// V^H A V.  Same layout and outputs as launch_jacobi.
template <typename S>
struct EighScratch {
  typename lowp<S>::type* A32;
  typename lowp<S>::type* A32b;
  typename lowp<S>::type* V32w;
  typename lowp<S>::type* V32;
  S* Vd;
  S* T;
  S* Vw;
  S* W64;
  double* lam32;
  int* sweeps;
  double* jscratch;
  GemmItem<S>* items;
  SmallDesc* dsub;
  double* delta;
  double* shift;
  S* A64;
  double* reach;            // per column: reach of the refinement's unseparated couplings
  double* reach_sorted;     // the same in ascending eigenvalue order
  int ccap;                 // capacity of the cluster arrays below
  GemmItem<S>* citems;
  SmallDesc* cdesc;
  int* csweeps;
  double* cjscratch;
  int ff = 0;               // float-float products in the refinement (set by the caller)
};
// columns i0..i0+c-1 of the m x m block at element offset off (eigenvalues at voff)
struct ClusterRef {
  int64_t off, voff;
  int m, i0, c;
};
constexpr int kMaxCluster = 64;
constexpr int kRefineSteps = 10;
constexpr double kRefineTol = 1e-8;
constexpr int kOaSplit = 16;  // CTAs per block in one refinement step
template <typename S>
EighScratch<S> plan_eigh_scratch(Arena& a, int64_t msq, int64_t mtot, int nblk);
// C_t = op(A_t) B_t for m x m blocks at each block's offset (abc = {A, B, C} bases).
template <typename S>
int small_gemm(bool conjA, const std::vector<SmallDesc>& blk, int max_m, S* const* abc, int herm, int triB,
               GemmItem<S>* d_items, cudaStream_t st, int ff = 0);

// h_fp32[t] (optional, default all): run the FP32 pre-rotation on block t; blocks that are
// already nearly diagonal skip it and go straight to the FP64 sweeps.
// what the mixed eigensolver did (accumulated by the caller)
struct EighReport {
  int refine_steps = 0, clusters = 0, max_cluster = 0, fallback_unconverged = 0, fallback_wide = 0;
};
template <typename S>
int eigh_mixed(int nblk, const SmallDesc* d_desc, const SmallDesc* h_desc, int max_m, S* A, double* lam, S* W,
               const EighScratch<S>& w, cudaStream_t st, int* fp64_sweeps_out = nullptr,
               const unsigned char* h_fp32 = nullptr, int* fp32_sweeps_out = nullptr, EighReport* rep = nullptr);

// Y = B X for the Hermitian band (lower storage), X, Y n x ncols (ld n).
// Float-float band product: the band is split once (launch_band_split into
// band_split_bytes of scratch), then Y = B X runs on the FP32 pipes.
size_t band_split_bytes(int64_t n, int b, int cplx);
template <typename S>
int launch_band_split(int64_t n, int b, const void* band, int64_t ldab, void* out, cudaStream_t st);
template <typename S>
int launch_band_matmul_ff(int64_t n, int b, const void* band_split, int ncols, const S* X, S* Y, cudaStream_t st);
template <typename S>
int launch_band_matmul(int64_t n, int b, const void* band, int64_t ldab, int ncols, const S* X, S* Y,
                       cudaStream_t st);

}  // namespace pdeshep
