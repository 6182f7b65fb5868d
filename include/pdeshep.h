/*
 * pdeshep.h -- C ABI of the GB300 (sm_103a) banded FEAST spectrum-slicing
 * library: the data-parallel core of step (II) of PDESHEP (arXiv 2012.00506,
 * "A Parallel Direct Eigensolver for Sequences of Hermitian Eigenvalue
 * Problems with No Tridiagonalization").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Band storage.  The Hermitian (or real symmetric) band matrix B of order n
 *    and semi-bandwidth b is given in LAPACK lower compact band form,
 *    column-major: B(i,j) for j <= i <= min(n-1, j+b) at band[(i-j) + j*ldab],
 *    ldab >= b+1.  Real input is double; complex input is interleaved
 *    pdeshep_c128.  The diagonal of a complex band must have zero imaginary
 *    part (it is ignored).  This is the compact storage the paper keeps on
 *    every process (Section 3, "stored compactly as in LAPACK").
 *  * Dense blocks (start vectors, eigenvectors) are column-major n x m with
 *    leading dimension n, of the same scalar type as the band.
 *  * Pointers prefixed d_ are device pointers, h_ host pointers.  The caller
 *    owns every buffer; the library never allocates device memory.  Scratch
 *    memory is a caller-provided device workspace whose size is returned by
 *    the matching *_workspace_size query (256-byte aligned base required).
 *  * Work is issued on the CUDA stream passed as `stream` (a cudaStream_t;
 *    NULL = legacy default stream).  Entry points that return host outputs
 *    synchronise that stream before returning.
 *  * Status: 0 = success; -i = the i-th argument (1-based) is invalid
 *    (LAPACK `info` convention); positive = a PDESHEP_* outcome below.
 *    CUDA runtime failures return PDESHEP_CUDA_ERROR and leave the message
 *    in pdeshep_last_error().
 */
#ifndef PDESHEP_H
#define PDESHEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double re, im;
} pdeshep_c128;

/* ---- status codes --------------------------------------------------------- */
#define PDESHEP_OK 0
#define PDESHEP_NOT_CONVERGED 1      /* max_iter reached before every slice converged */
#define PDESHEP_COUNT_MISMATCH 2     /* m0 of a slice is below its exact count (Section 3.2) */
#define PDESHEP_CHOLQR_BREAKDOWN 3   /* Gram matrix not numerically positive definite */
#define PDESHEP_NONFINITE_INPUT 4    /* NaN/Inf in the band or start vectors */
#define PDESHEP_WORKSPACE_TOO_SMALL 5
#define PDESHEP_DEVICE_TIMEOUT 6     /* a bounded device-side wait gave up */
#define PDESHEP_SINGULAR 7           /* exactly zero pivot in a shifted factorization */
#define PDESHEP_CUDA_ERROR 8
#define PDESHEP_EIG_NOT_CONVERGED 9  /* small dense eigensolver did not converge */

/* ---- precision of the shifted factorizations and solves ----------------- */
#define PDESHEP_FP64 0   /* complex128 LU and solves (plain FEAST, Algorithm 1) */
#define PDESHEP_MIXED 1  /* complex64 LU and solves with FP32 accumulation + FP64 refinement */

/* ---- refinement policy for PDESHEP_MIXED --------------------------------- */
#define PDESHEP_REFINE_NONE 0      /* plain filter in complex64 (FP32-class accuracy) */
#define PDESHEP_REFINE_RESIDUAL 1  /* filter applied to FP64 Ritz residuals (default):
                                      r(B) x = r(lambda) x + sum_j w_j/(z_j-lambda) (z_j I-B)^{-1} (Bx - lambda x) */

typedef struct {
  double tol;              /* relative residual ||Bx - lambda x|| / (bnorm ||x||); default 1e-10 */
  int32_t max_iter;        /* FEAST iterations per slice; default 20 */
  int32_t precision;       /* PDESHEP_FP64 or PDESHEP_MIXED; default PDESHEP_MIXED */
  int32_t refine_policy;   /* PDESHEP_REFINE_*; default PDESHEP_REFINE_RESIDUAL */
  int32_t rhs_chunk;       /* right-hand sides per solve work item: 16, 32 or 64 (a thread per
                              row of a 32-row tile, the window in shared memory), 128 (complex64
                              factors only: a thread per right-hand side, the window in tensor
                              memory, b <= 128) or 256 (complex64 factors only: the tile products
                              on the tensor cores as bf16x6 MMAs into tensor memory, items of 128
                              right-hand sides, b <= 128; the tensor core truncates its FP32
                              accumulator, so these solves carry 2-3x the error of the FP32-FMA
                              ones); a nonzero value serves every filter pass.  0 = the first four
                              passes on the tensor cores where they apply and are not measured
                              slower, the later passes on the fastest FP32-FMA width (measured when
                              autotune is on, else 128 where it applies or 32) */
  double ellipse_ratio;    /* vertical / horizontal semi-axis of the contour; default 0.3 */
  double bnorm;            /* ||B||_2 for the residual; <= 0: computed by the library */
  uint64_t seed;           /* start vectors drawn by the library when d_x0 is NULL (see
                              pdeshep_random_start); default 0 */
  size_t hbm_cap_bytes;    /* cap on the factor storage (factors and per-system solve outputs) of
                              one group of slices; 0 = whatever the workspace holds.  Slices run
                              in consecutive groups whose factors all stay resident within the
                              cap and the workspace, each group iterating to convergence on
                              factors computed once (a call that fits is one group); a single
                              slice whose factors exceed it streams them in waves every
                              iteration */
  int32_t autotune;        /* 0 off; 1 use the tuned choice for this problem shape, measuring
                              it on first use; 2 measure again.  Tuned: the solve column block
                              (16/32/64/128 and whether 256 serves the first passes, unless
                              rhs_chunk is set) and the split count of the tall Gram products
                              (2/4/8) */
  int32_t verbose;         /* 0 quiet */
  void* stream;            /* cudaStream_t */
  int32_t rr_arith;        /* PDESHEP_MIXED only: arithmetic of the Rayleigh-Ritz products.
                              PDESHEP_RR_TENSOR (default): tall products (Gram, projection, basis
                              update) as bf16 digit products on the tensor cores, FP64-class; band
                              and small products float-float.  PDESHEP_RR_FLOATFLOAT: all products
                              float-float.  In both, iterations after the third run the
                              float-float products in FP64.  PDESHEP_RR_FP64: all products FP64 */
  int32_t m0_resize;       /* 1: the subspace rule of Section 3.2 in the library.  The exact counts
                              m_i are taken first; a slice whose h_m0[i] is below m_i + 10 runs
                              with max(ceil(1.3 m_i), m_i + 10) columns, at most m0_cap.  The
                              blocks of d_x0 / d_evals / d_evecs are then m0_cap columns each
                              (slice i at column i * m0_cap; its start vectors are the first m0
                              columns of its block).  COUNT_MISMATCH only if m_i > m0_cap.
                              0 (default): h_m0 as given, COUNT_MISMATCH if below m_i */
  const char* tune_cache;  /* file that keeps tuned choices across processes; NULL = in-process */
  int32_t graphs;          /* 1: with resident factors, each filter pass (right-hand sides,
                              weights, both solves, accumulation) is captured once per set of
                              active slices as a CUDA graph and replayed; needs a stream other
                              than the legacy default stream.  0 (default): direct launches */
  int32_t m0_cap;          /* column capacity of each slice's block when m0_resize = 1 */
  int32_t* h_m0_used;      /* optional host output (nslices): the m0 each slice ran with */
} pdeshep_opts;

/* Arithmetic of the Rayleigh-Ritz products (Gram, projection, basis update,   */
/* band product, eigenvector refinement) in mixed precision.  FLOATFLOAT runs  */
/* them as float-float (FP32 pairs, ~48-bit products, FP32 exponent range) on  */
/* the FP32 pipes, which GB300 has 64x more of than FP64; FP64 keeps them in   */
/* FP64 arithmetic.  Counts and residual tests are the same either way.       */
#define PDESHEP_RR_FLOATFLOAT 0
#define PDESHEP_RR_FP64 1
#define PDESHEP_RR_TENSOR 2   /* bf16 digit products on the tensor cores (FP64-class) */

/* Kernel groups timed separately (CUDA events around each launch). */
#define PDESHEP_KG_INERTIA 0     /* LDL^T inertia (and the band amax reduction) */
#define PDESHEP_KG_FACTOR 1      /* shifted band LU (tile init + factorization) */
#define PDESHEP_KG_SOLVE 2       /* multi-RHS band solves (forward + backward sweeps) */
#define PDESHEP_KG_ACCUM 3       /* right-hand-side preparation and weighted accumulation of Q */
#define PDESHEP_KG_GEMM 4        /* tall products (Gram, projection, basis update): FP64 or float-float */
#define PDESHEP_KG_SMALL 5       /* FP64 Cholesky and triangular inverse, small m0 x m0 products */
#define PDESHEP_KG_BANDMM 6      /* band times block (B Q, B X; FP64 or float-float) and residual norms */
#define PDESHEP_KG_EIG 7         /* small eigensolver: FP32 Jacobi, FP64-class refinement, clusters */
#define PDESHEP_KG_COUNT 8

typedef struct {
  int32_t iterations;      /* FEAST iterations of the slowest slice */
  int32_t waves;           /* factorization waves issued */
  int64_t factorizations;  /* shifted band LU factorizations */
  int64_t rhs_sweeps;      /* (system, column-block) forward+backward solve sweeps */
  double ms_inertia;       /* wall time per phase (CUDA events on the stream) */
  double ms_factor;
  double ms_solve;
  double ms_rr;
  double ms_total;
  double max_residual;     /* over the converged in-slice pairs */
  double min_rel_error_est;/* reserved */
  /* per kernel group (PDESHEP_KG_*): summed device time of its launches, launch
     count, and algorithmic work (real flops, complex multiply-add = 8) */
  double kg_ms[PDESHEP_KG_COUNT];
  int64_t kg_launches[PDESHEP_KG_COUNT];
  double kg_flops[PDESHEP_KG_COUNT];
  int64_t rhs_columns;     /* sum over solve sweeps of the right-hand sides swept */
  int32_t cluster_ctas;    /* thread blocks per slice in the small dense kernels */
  int32_t jacobi_sweeps64; /* FP64 Jacobi sweeps, summed over Rayleigh-Ritz calls (max over slices) */
  int32_t jacobi_sweeps32; /* FP32 Jacobi sweeps, same accounting */
  int32_t rr_calls;        /* Rayleigh-Ritz calls */
  /* small dense eigensolver, summed over Rayleigh-Ritz calls: FP64 refinement
     steps, clusters resolved by their own Rayleigh-Ritz step (and the widest),
     and blocks sent to the FP64 Jacobi path because the refinement had not
     converged or left a cluster wider than 64 */
  int32_t eig_refine_steps;
  int32_t eig_clusters;
  int32_t eig_max_cluster;
  int32_t eig_fallback_unconverged;
  int32_t eig_fallback_wide;
  int32_t rhs_chunk_used;  /* solve column block of the last filter pass */
  int32_t gram_splits_used;/* split count of the last tall Gram product */
  int32_t tuned;           /* number of choices measured by the autotuner in this call */
  int32_t graph_launches;  /* filter passes replayed from CUDA graphs */
  int32_t cholqr_shifted;  /* slices whose Gram matrix needed a shifted Cholesky */
  int32_t gram_fp64;       /* float-float mode: slices whose Gram matrices were redone in FP64 */
  int32_t rr_fp64_from;    /* float-float mode: iteration from which the Rayleigh-Ritz products ran in
                              FP64 because slices were still unconverged after 3 iterations (0: never) */
  int32_t rhs_chunk_early; /* solve column block of the first four filter passes when it differs from
                              the later passes' (256: the tensor-core solve, chosen when measured faster;
                              passes after the fourth take the round-to-nearest FP32-FMA solves); 0: none */
} pdeshep_stats;

/* Forget every tuned choice held in this process (cache files are kept). */
void pdeshep_tune_reset(void);

/* Testing hook: the number of polls after which a bounded mbarrier wait of the tensor-core kernels */
/* (tall and band products, complex64 solves) gives up; polls <= 0 restores the defaults (2^24     */
/* and 2^22 polls with back-off, about a second).  A wait that gives up ends its CTA's work, the   */
/* call returns PDESHEP_DEVICE_TIMEOUT, and the GPU context stays usable: before a CTA exits it    */
/* still waits, with the default limit, for every copy and product it issued.  Process-wide for    */
/* the current device; do not change it while calls are in flight.  Returns 0 or                   */
/* PDESHEP_CUDA_ERROR.                                                                             */
int pdeshep_debug_wait_limit(int64_t polls);

/* Fill *o with the defaults listed above. */
void pdeshep_opts_default(pdeshep_opts* o);

/* Human-readable name of a status code (static string). */
const char* pdeshep_status_string(int status);

/* Last CUDA error message recorded by this thread (static per-thread buffer). */
const char* pdeshep_last_error(void);

/* Library version string. */
const char* pdeshep_version(void);

/* Number of CUDA kernels this library has launched in this process so far. */
uint64_t pdeshep_kernel_launches(void);

/* Measured ALU throughput of the current GPU (the roofline denominator of    */
/* kernels bound by the FP32 or FP64 pipes; not part of the paper's method):  */
/* a launch of SMs x 2048 threads, each running 8 independent FMA chains of   */
/* 16 x iters steps; best of three launches timed with CUDA events on        */
/* `stream`.  fp64 = 0: FP32 FMAs, 1: FP64 FMAs.  *h_tflops = 2 x FMAs /      */
/* time in TFLOP/s.  d_scratch: any device buffer of SMs x 2048 doubles      */
/* (never written in practice).  Synchronous.                                */
int pdeshep_alu_peak(int32_t fp64, int64_t iters, double* h_tflops, void* d_scratch, void* stream);

/* ------------------------------------------------------------------------ */
/* Sylvester inertia (Section 3.2; Section 3.1): for every sigma_s counts the  */
/* eigenvalues of B below sigma_s as the number of negative pivots of the     */
/* pivot-free LDL^T (real) / LDL^H (complex) factorization of B - sigma_s I,  */
/* computed in FP64 without fused multiply-add, in a fixed operation order.   */
/* An exactly zero pivot is replaced by -pivmin, pivmin = DBL_MIN *           */
/* max(1, amax^2), amax = max over stored band entries of max(|Re|,|Im|).     */
/*  h_sigma[nsigma] (host) -> h_neg[nsigma] (host, synchronous).              */
/*  d_pivots: optional device output (NULL to skip) of the nsigma x n pivots  */
/*  D (row s holds the pivots for sigma_s).                                   */
/* Workspace: pdeshep_inertia_workspace_size(n, b, is_complex, nsigma).      */
/* ------------------------------------------------------------------------ */
size_t pdeshep_inertia_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nsigma);
int pdeshep_inertia(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                    int32_t nsigma, const double* h_sigma, int64_t* h_neg, double* d_pivots,
                    void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Allocation-free inertia.  The paper has no counterpart: this entry point   */
/* exists for callers that cannot hand the library any device memory -- for  */
/* example code whose device memory is wholly owned by another allocator, or */
/* a callback that may only run kernels on buffers it is given -- and so      */
/* cannot supply the workspace of pdeshep_inertia.  It computes the same      */
/* counts as pdeshep_inertia (same kernel, same arithmetic) but keeps its     */
/* scratch (a few words plus the shifts and counts) in one fixed 20 KiB       */
/* device array inside the library; every GPU that loads the library holds   */
/* that array until the process exits.  It never allocates or frees device  */
/* memory.                                                                   */
/*  Limits: nsigma <= 1024 (else -6) and the LDL^T window must fit in shared */
/*  memory: real b <= 194, complex b <= 149 (else -2); the reason is then in */
/*  pdeshep_last_error().                                                    */
/*  Every call looks up the array's device address on the current device    */
/*  (cudaGetSymbolAddress); the first call on a device may load the library's */
/*  device code there, so make that first call before any stream capture.    */
/*  A negative b is refused with -2 as well.  All calls share the one array  */
/*  and it keeps the last call's                                             */
/*  contents (each call clears and rewrites what it uses): calls that may    */
/*  overlap on the GPU -- concurrent streams, or host threads on the same    */
/*  device -- race on it and must be serialised by the caller.  Synchronous: */
/*  returns after h_neg is written.                                          */
/* ------------------------------------------------------------------------ */
int pdeshep_inertia_noalloc(int64_t n, int32_t b, int32_t is_complex, const void* d_band,
                            int64_t ldab, int32_t nsigma, const double* h_sigma, int64_t* h_neg,
                            void* stream);

/* ------------------------------------------------------------------------ */
/* Eigenvalue enclosures by bisection on inertia (slice boundaries with exact */
/* counts; the fall-back of the slice proposer).  For each requested index   */
/* k_t (0-based, ascending order of eigenvalues) returns h_lo[t] < h_hi[t]    */
/* with count(h_lo[t]) <= k_t < count(h_hi[t]), i.e. lambda_{k_t} in          */
/* [h_lo, h_hi), and h_hi - h_lo <= rtol * max(1, |h_lo|, |h_hi|).  All       */
/* enclosures are refined together: each round evaluates `fanout` points per  */
/* enclosure in one batched inertia launch.                                  */
/* ------------------------------------------------------------------------ */
size_t pdeshep_bisect_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nidx,
                                     int32_t fanout);
int pdeshep_bisect(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                   int32_t nidx, const int64_t* h_idx, double rtol, int32_t fanout,
                   double* h_lo, double* h_hi, void* d_work, size_t work_bytes, void* stream);

/* Gershgorin interval [lo, hi] of the band (device reduction, synchronous). */
int pdeshep_gershgorin(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                       double* h_lo, double* h_hi, void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Quadrature rule (Section 2.2, eqs. (8)-(9)): ne Gauss-Legendre nodes on the */
/* upper half of the ellipse around [lo, hi] with vertical/horizontal ratio  */
/* rho: z_k = c + r(cos t_k + i rho sin t_k), w_k = (omega_k r/4)(rho cos t_k */
/* + i sin t_k), t_k = (pi/2)(1 - x_k), c = (lo+hi)/2, r = (hi-lo)/2, so that  */
/* the filter is r(x) = 2 Re sum_k w_k/(z_k - x) (the lower half follows by   */
/* conjugate symmetry).  Host only.                                          */
/* ------------------------------------------------------------------------ */
int pdeshep_contour_rule(int32_t ne, double lo, double hi, double rho, pdeshep_c128* h_z,
                         pdeshep_c128* h_w);
/* The midpoint trapezoid rule on the same half ellipse (Section 2.2 cites it beside Gauss         */
/* quadrature): t_k = pi (k + 1/2)/ne, w_k = (r/(2 ne))(rho cos t_k + i sin t_k), same filter      */
/* convention; for rho = 1 the filter is 1/(1 + ((x-c)/r)^(2 ne)).  Pass the nodes and weights to */
/* pdeshep_band_slice through h_nodes / h_weights.  Host only.                                    */
int pdeshep_contour_rule_trapezoid(int32_t ne, double lo, double hi, double rho, pdeshep_c128* h_z,
                                   pdeshep_c128* h_w);
/* The Zolotarev rule (the improved rational filter Section 2.2 cites after eq. (10)): ne nodes   */
/* on the upper half of the circle with diameter [lo, hi] and weights in the same convention,      */
/* whose filter 2 Re sum_k w_k/(z_k - x) is within E of the indicator of [lo, hi] at every real x  */
/* at least gap*(hi - lo) away from both lo and hi, E being the equioscillation error of           */
/* Zolotarev's best type (2ne-1, 2ne) approximation of sign(x) on [-1,-ell] U [ell,1] with         */
/* sqrt(ell) = gap/(1 + gap); r(lo) = r(hi) = 1/2 - f_inf with |f_inf| = E/2 (the constant term of */
/* the rational function, which a rule of nodes and weights cannot carry, is left out).            */
/* Arguments: 1 <= ne <= 256, finite lo < hi, finite gap >= 1e-8; h_z, h_w hold ne entries each   */
/* (caller-owned host memory); h_err receives E (may be NULL).  Returns 0, or -1 (ne), -2 (lo/hi), */
/* -4 (gap), -5 (h_z NULL), -6 (h_w NULL).  Rounding amplified by the partial fractions adds to E: */
/* the filter is within E + 1e-12 of the indicator for gap >= 1e-4, E + 1e-10 for gap >= 1e-6 and */
/* E + 1e-9 down to gap = 1e-8 (ne <= 256).  Host only; pass the rule to pdeshep_band_slice        */
/* through h_nodes / h_weights.                                                                    */
int pdeshep_contour_rule_zolotarev(int32_t ne, double lo, double hi, double gap, pdeshep_c128* h_z,
                                   pdeshep_c128* h_w, double* h_err);

/* ------------------------------------------------------------------------ */
/* Shifted band solves of eq. (10): for each shift z_s, factor z_s I - B by   */
/* LU with partial pivoting inside the band (fill to 2b superdiagonals) and   */
/* solve for nrhs right-hand sides:                                          */
/*   trans = 0: X_s = (z_s I - B)^{-1} Y;  trans = 1: X_s = (z_s I - B)^{-H} Y */
/* d_rhs: n x nrhs complex128 (device); d_x: nshift blocks of n x nrhs        */
/* complex128 (device), block s at d_x + s*n*nrhs.                            */
/* precision: PDESHEP_FP64 (complex128 arithmetic) or PDESHEP_MIXED (complex64 */
/* factors and solves, FP32 accumulation; inputs/outputs stay complex128).    */
/* d_ipiv: optional (NULL to skip) nshift x n int32 pivot rows, 0-based,      */
/* LAPACK gbtrf meaning: at step k rows k and d_ipiv[k] were interchanged.   */
/* Returns PDESHEP_SINGULAR if some pivot was exactly zero.                   */
/* ------------------------------------------------------------------------ */
size_t pdeshep_shifted_solve_workspace_size(int64_t n, int32_t b, int32_t nshift, int32_t nrhs,
                                            int32_t precision);
int pdeshep_shifted_solve(int64_t n, int32_t b, int32_t is_complex, const void* d_band,
                          int64_t ldab, int32_t nshift, const pdeshep_c128* h_shifts, int32_t nrhs,
                          const pdeshep_c128* d_rhs, int32_t trans, int32_t precision,
                          pdeshep_c128* d_x, int32_t* d_ipiv, void* d_work, size_t work_bytes,
                          void* stream);

/* ------------------------------------------------------------------------ */
/* Band times dense block: d_y = B d_x for nrhs columns (FP64).               */
/* ------------------------------------------------------------------------ */
int pdeshep_band_matmul(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                        int32_t nrhs, const void* d_x, void* d_y, void* stream);

/* ------------------------------------------------------------------------ */
/* CholQR (orthonormal basis for the Rayleigh-Ritz step of Section 2.2) on a  */
/* batch of column blocks, FP64: for block t (n x m_t, starting at column     */
/* col_off[t] of d_q), G = Q^H Q = R^H R (R upper, positive diagonal),        */
/* Q <- Q R^{-1}; `passes` = 1 (CholQR) or 2 (CholQR2).  d_r: optional        */
/* output of the last pass's R factors, block t at d_r + sum_{u<t} m_u^2,     */
/* column-major.  Returns PDESHEP_CHOLQR_BREAKDOWN if a Cholesky pivot is not */
/* positive.                                                                 */
/* ------------------------------------------------------------------------ */
size_t pdeshep_cholqr_workspace_size(int64_t n, int32_t nblk, const int32_t* h_m, int32_t is_complex);
int pdeshep_cholqr(int64_t n, int32_t is_complex, int32_t nblk, const int32_t* h_m, void* d_q,
                   int32_t passes, void* d_r, void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Re-slicing from the previous step's eigenvalues (Section 3.1).  Host only  */
/* (no GPU work): h_d[n] ascending (the previous eigenvalues), b0 <= h_d[0],  */
/* h_d[n-1] < bK.  Groups are taken by value, G_i = [b_{i-1}, b_i).           */
/*   PDESHEP_PART_KMEANS       the simplified 1-D k-means of Algorithm 3:     */
/*                             from equal counts, each inner boundary moves   */
/*                             to the gap after the midpoint of its groups'   */
/*                             centroids (mean of a group's extreme points)   */
/*                             until none moves (at most max_sweeps sweeps);  */
/*                             empty groups are merged away (K may shrink)    */
/*   PDESHEP_PART_EQUAL_COUNT  "Approach-1": equal counts (the first n mod K  */
/*                             groups one more), boundaries at gap midpoints  */
/*   PDESHEP_PART_EQUAL_WIDTH  "Approach-2": K equal pieces of [b0, bK]       */
/* Out: h_bounds[K_out + 1], h_counts[K_out] (capacities K + 1 and K),        */
/* *h_k_out = K_out <= K, *h_sweeps (optional) = k-means sweeps.              */
/* ------------------------------------------------------------------------ */
#define PDESHEP_PART_KMEANS 0
#define PDESHEP_PART_EQUAL_COUNT 1
#define PDESHEP_PART_EQUAL_WIDTH 2
int pdeshep_partition(int32_t method, int64_t n, const double* h_d, int32_t K, double b0, double bK,
                      int32_t max_sweeps, double* h_bounds, int32_t* h_counts, int32_t* h_k_out,
                      int32_t* h_sweeps);

/* Start vectors after a re-slicing (Section 3.1: when a slice grows the     */
/* previous vectors are interlaced with random ones, when it shrinks some are */
/* removed).  h_prev_vals[nprev]: Ritz value of each previous column.  For    */
/* new slice i the block of h_m0[i] entries of h_src (blocks in slice order)  */
/* lists the previous columns with values in [b_i, b_{i+1}) -- the h_m0[i]    */
/* nearest to the slice centre if there are more -- in ascending value (ties  */
/* by column), then (mode 1) the nearest columns outside the slice, and -1    */
/* for each remaining column (a random start vector).  Offer the previous    */
/* call's converged pairs (distinct eigenvectors): its unconverged extra      */
/* columns approximate the neighbouring slices' vectors, and mixing both can  */
/* make a start block numerically rank-deficient.  Host only.                */
/* ------------------------------------------------------------------------ */
int pdeshep_restart_plan(int64_t nprev, const double* h_prev_vals, int32_t K, const double* h_bounds,
                         const int32_t* h_m0, int32_t mode, int64_t* h_src);

/* ------------------------------------------------------------------------ */
/* The start block of a re-sliced call from a restart plan (the device side  */
/* of pdeshep_restart_plan, Section 3.1): column j of d_dst (n x ncols,       */
/* column-major, the band's type) is column h_src[j] of d_prev (n x nprev)    */
/* when h_src[j] >= 0, else column col0 + j of the library's start-vector    */
/* stream with this seed (pdeshep_random_start's columns: the random vectors */
/* interlaced with the previous ones).  h_src[j] < nprev (else -6).          */
/* d_work: pdeshep_gather_columns_workspace_size(ncols) bytes.  Asynchronous. */
/* ------------------------------------------------------------------------ */
size_t pdeshep_gather_columns_workspace_size(int32_t ncols);
int pdeshep_gather_columns(int64_t n, int32_t is_complex, const void* d_prev, int64_t nprev, int32_t ncols,
                           const int64_t* h_src, uint64_t seed, int64_t col0, void* d_dst, void* d_work,
                           size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Outer bounds of the wanted eigenvalues i0 .. i0+nev-1 of the band from the */
/* previous matrix's eigenvalues h_prev[nprev] (ascending) (Section 3.2,      */
/* Algorithm 4 and the lower-bound search described beside it): bK starts at  */
/* d = h_prev[i0+nev-1] plus step = max(|alpha d|, m_hat (d - h_prev[i0+nev-2]))*/
/* and grows by step until the inertia count below it is >= i0 + nev; b0     */
/* starts at h_prev[i0] minus max(|alpha d'|, m_hat (h_prev[i0+1] - d')) and  */
/* shrinks until the count below it is <= i0 (a zero step becomes 2^-40 of   */
/* the value).  At most max_it counts each; h_iters[2] (optional) = the       */
/* counts taken for b0 and bK.  Returns PDESHEP_NOT_CONVERGED (outputs still  */
/* written) when a search spent its max_it counts without reaching its       */
/* target, i.e. the bounds do not enclose the wanted eigenvalues.            */
/* Synchronous.  Workspace:                                                  */
/* pdeshep_outer_bounds_workspace_size(n, b, is_complex).                     */
/* ------------------------------------------------------------------------ */
size_t pdeshep_outer_bounds_workspace_size(int64_t n, int32_t b, int32_t is_complex);
int pdeshep_outer_bounds(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                         int64_t nprev, const double* h_prev, int64_t i0, int64_t nev, double alpha,
                         double m_hat, int32_t max_it, double* h_b0, double* h_bK, int32_t* h_iters,
                         void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Tall block products of the Rayleigh-Ritz step (Section 2.2: the Gram      */
/* matrix Q^H Q of the orthonormalisation, the projection Q^H (B Q) and the  */
/* basis update Q W) on a batch of column blocks of n rows.  Block t of d_a   */
/* (and d_b for kind 0) is n x m_t, column-major (ld n), at column           */
/* sum_{u<t} m_u; the m_t x m_t blocks (output of kinds 0 and 1, second      */
/* operand of kind 2) sit at element offset sum_{u<t} m_u^2, column-major.   */
/*   kind PDESHEP_GEMM_AHB    C_t = A_t^H B_t                                 */
/*   kind PDESHEP_GEMM_GRAM   C_t = A_t^H A_t (Hermitian; d_b unused)         */
/*   kind PDESHEP_GEMM_UPDATE C_t = A_t B_t, n x m_t in the layout of d_a     */
/* arith: PDESHEP_RR_FP64 (FP64 pipes), PDESHEP_RR_FLOATFLOAT (float-float   */
/* on the FP32 pipes) or PDESHEP_RR_TENSOR (bf16 digit products on the       */
/* tcgen05 tensor cores, FP64-class accuracy: a few units of 2^-48 |a| |b|  */
/* per entry).  Returns PDESHEP_DEVICE_TIMEOUT (after synchronising) if a    */
/* tensor-core kernel's bounded wait gave up.                                */
/* ------------------------------------------------------------------------ */
/* Y = B X for the Hermitian band (lower storage, as pdeshep_band_matmul) and X, Y n x ncols     */
/* column-major (ld n), on the tensor cores with the same bf16 digit products: each 128-row tile */
/* of B over its (128 + 2 b)-column window times the digit rows of X.  FP64-class accuracy (a   */
/* few units of 2^-48 |B(i,:)| max|X(:,j)| per entry).                                          */
size_t pdeshep_band_matmul_tc_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t ncols);
int pdeshep_band_matmul_tc(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                           int32_t ncols, const void* d_x, void* d_y, void* d_work, size_t work_bytes,
                           void* stream);
#define PDESHEP_GEMM_AHB 0
#define PDESHEP_GEMM_GRAM 1
#define PDESHEP_GEMM_UPDATE 2
size_t pdeshep_block_gemm_workspace_size(int64_t n, int32_t is_complex, int32_t nblk, const int32_t* h_m);
int pdeshep_block_gemm(int32_t kind, int32_t arith, int64_t n, int32_t is_complex, int32_t nblk,
                       const int32_t* h_m, const void* d_a, const void* d_b, void* d_c, void* d_work,
                       size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched small dense Hermitian eigensolver for A_q W_q = W_q Lambda_q       */
/* (Section 2.2): block t is an m_t x m_t column-major matrix at offset       */
/* sum_{u<t} m_u^2 of d_a (overwritten), eigenvalues ascending into d_lam     */
/* (offset sum_{u<t} m_u), eigenvectors into d_v (same layout as d_a), each   */
/* scaled so its first largest-magnitude component is real positive.         */
/* Cyclic Jacobi in parallel (round-robin) order on a thread-block cluster    */
/* per block: FP32 sweeps give V32, then H = V32^H A V32 (FP64) is nearly     */
/* diagonal and FP64 sweeps finish it (off(H) <= 1e-14 ||H||_F); the          */
/* eigenvectors are V32 W.                                                    */
/* ------------------------------------------------------------------------ */
size_t pdeshep_eigh_workspace_size(int32_t nblk, const int32_t* h_m, int32_t is_complex);
int pdeshep_eigh(int32_t is_complex, int32_t nblk, const int32_t* h_m, void* d_a, double* d_lam,
                 void* d_v, void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* FEAST spectrum slicing on the band (Algorithm 1 per slice; slices are     */
/* level-L1 and quadrature nodes level-L2 of the paper's parallelism, here a  */
/* batch on one GPU).  Slice i is [h_bounds[i], h_bounds[i+1]).               */
/*  h_nodes/h_weights: ne complex nodes/weights per slice (slice-major), or   */
/*    NULL for the Gauss-Legendre ellipse rule of pdeshep_contour_rule.       */
/*  h_m0[i]: subspace size of slice i (must be >= the slice's exact count;    */
/*    Section 3.2 suggests max(1.3 m_i, m_i + 10)).                            */
/*  d_x0: n x sum(m0) start vectors (slice-major column blocks), same type as */
/*    the band; e.g. random vectors or the previous SCF step's eigenvectors;  */
/*    NULL: drawn by the library from opts.seed (pdeshep_random_start's       */
/*    columns, numbered by the output column of each slice block).          */
/*  Outputs: d_evals[sum(m0)], d_evecs n x sum(m0) (same type as the band);   */
/*    in slice block i the first h_nfound[i] pairs are the converged in-slice  */
/*    eigenpairs (ascending), then the other Ritz pairs (ascending).          */
/*    h_counts[i] = exact inertia count of slice i.  h_stats optional.         */
/* Returns PDESHEP_NOT_CONVERGED if some slice did not converge (its outputs  */
/* are the last Ritz pairs; converged slices are valid).                     */
/* Workspace: pdeshep_workspace_size with the same opts (its plan of slice   */
/* groups depends on hbm_cap_bytes, m0_resize and m0_cap).  Statistics of a  */
/* grouped call are summed over the groups (iterations: the maximum).        */
/* ------------------------------------------------------------------------ */
size_t pdeshep_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nslices,
                              const int32_t* h_m0, int32_t ne, const pdeshep_opts* opts);
int pdeshep_band_slice(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                       int32_t nslices, const double* h_bounds, int32_t ne,
                       const pdeshep_c128* h_nodes, const pdeshep_c128* h_weights,
                       const int32_t* h_m0, const void* d_x0, void* d_work, size_t work_bytes,
                       const pdeshep_opts* opts, double* d_evals, void* d_evecs, int32_t* h_counts,
                       int32_t* h_nfound, pdeshep_stats* h_stats);

/* ------------------------------------------------------------------------ */
/* Start vectors drawn by the library (the "random vectors" of Algorithm 1's */
/* first iteration, for callers that pass d_x0 = NULL): columns col0 ..      */
/* col0+ncols-1 of a counter-based stream, n x ncols column-major into d_x.  */
/* Entry (i, c) uses word k = (col0 + c) n + i: real bands x = u(seed + k),  */
/* complex bands x = u(seed + 2k) + i u(seed + 2k + 1), u(w) = (top 53 bits  */
/* of splitmix64(w)) 2^-52 - 1, uniform in [-1, 1) (splitmix64: Vigna's     */
/* generator, golden-ratio increment 0x9e3779b97f4a7c15, then the mixer).    */
/* Asynchronous.                                                             */
/* ------------------------------------------------------------------------ */
int pdeshep_random_start(int64_t n, int32_t is_complex, int64_t col0, int32_t ncols, uint64_t seed, void* d_x,
                         void* stream);

/* ======================================================================== */
/* Slice proposal.  The paper slices the spectrum by inertia counts          */
/* (Section 3.2) and, with no earlier spectrum to go by, points to density- */
/* of-states estimates (Section 3.1); one of its partition objectives is an  */
/* equal eigenvalue count per slice (Section 3.1).  The network below is not */
/* in the paper: it predicts equal-count boundaries from cheap statistics of */
/* the band, and every count the proposer returns is an exact inertia count. */
/* ======================================================================== */

/* Number of FP32 parameters of the proposal network 98 -> 256 -> 256 -> 256  */
/* -> 64 (ReLU hidden layers, softmax head).  Parameter vector layout: for   */
/* each of the four layers W (out x in, row-major) then its bias (out).      */
int64_t pdeshep_mlp_param_count(void);

/* ------------------------------------------------------------------------ */
/* 98 FP32 features of one band into d_features[98] (asynchronous):         */
/*  [0,64)  histogram of diag(B) over the Gershgorin interval [lo, hi]: bin  */
/*          k = clamp(floor((d - lo) / ((hi - lo)/64)), 0, 63) computed in   */
/*          FP64, as fractions of n;                                        */
/*  64, 65  (lo + hi)/2 / s and (hi - lo)/2 / s with s = max(|lo|, |hi|);    */
/*  [66,98) Chebyshev moments mu_k = (1/(8n)) sum_p z_p^H T_k(Bs) z_p,       */
/*          k = 0..31, of Bs = (B - c I)/r (c, r the interval's centre and   */
/*          half-width), accumulated in FP64 (kernel polynomial method).     */
/* Probe p (p = 0..7), entry i: +1 if splitmix64(seed + p*n + i) is even,    */
/* else -1 (splitmix64: Vigna's 64-bit mixer with increment                 */
/* 0x9e3779b97f4a7c15).  d_work: pdeshep_slice_features_workspace_size      */
/* bytes (5 * 8 * n scalars of the band's type plus a few KiB).             */
/* ------------------------------------------------------------------------ */
size_t pdeshep_slice_features_workspace_size(int64_t n, int32_t is_complex);
int pdeshep_slice_features(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                           uint64_t seed, float* d_features, void* d_work, size_t work_bytes,
                           void* stream);

/* ------------------------------------------------------------------------ */
/* Network evaluation on a batch (asynchronous, FP32).  d_x: batch x 98      */
/* row-major features; d_bounds: batch x 63 row-major outputs, the cumulative */
/* sums of the softmax of the 64 logits = predicted equal-count boundaries   */
/* k/64 (k = 1..63) in normalised [0, 1] coordinates of the Gershgorin       */
/* interval.  pdeshep_mlp_grad also takes targets (batch x 63) and writes    */
/* the loss L = mean over batch and the 63 boundaries of the squared error  */
/* to d_loss[0] and dL/dparams to d_grad (param_count floats).              */
/* pdeshep_mlp_train_step does that and one Adam step (beta1 0.9, beta2      */
/* 0.999, eps 1e-8, bias correction with the 1-based `step`) on d_params,    */
/* d_adam_m, d_adam_v (param_count floats each, moments start at zero).      */
/* batch in [1, 65535]; d_work: pdeshep_mlp_workspace_size(batch) bytes.     */
/* ------------------------------------------------------------------------ */
size_t pdeshep_mlp_workspace_size(int32_t batch);
int pdeshep_mlp_forward(const float* d_params, int32_t batch, const float* d_x, float* d_bounds,
                        void* d_work, size_t work_bytes, void* stream);
int pdeshep_mlp_grad(const float* d_params, int32_t batch, const float* d_x, const float* d_target,
                     float* d_grad, float* d_loss, void* d_work, size_t work_bytes, void* stream);
int pdeshep_mlp_train_step(float* d_params, float* d_adam_m, float* d_adam_v, int32_t step, float lr,
                           int32_t batch, const float* d_x, const float* d_target, float* d_loss,
                           void* d_work, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Training labels of the proposal network (its regression targets): for k =  */
/* 1..nslices-1, t_k = floor(k n / nslices + 1/2) clipped to [1, n-1]; the    */
/* eigenvalues t_k - 1 and t_k (0-based, ascending) are enclosed by bisection */
/* on inertia to relative width rtol (pdeshep_bisect, `fanout` points per    */
/* enclosure per launch), and h_targets[k-1] = clip((s_k - lo)/(hi - lo), 0,  */
/* 1) in FP32, s_k the midpoint of the two enclosures' midpoints and [lo, hi] */
/* the Gershgorin interval (pdeshep_gershgorin).  The equal-count partition   */
/* is one of the paper's partition objectives (Section 3.1); counts by        */
/* inertia (Section 3.2).  Synchronous.                                       */
/* ------------------------------------------------------------------------ */
size_t pdeshep_equal_count_targets_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nslices,
                                                  int32_t fanout);
int pdeshep_equal_count_targets(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                int32_t nslices, double rtol, int32_t fanout, float* h_targets, void* d_work,
                                size_t work_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Propose nslices slices holding equal shares of the eigenvalues with       */
/* ascending indices in [frac_lo n, frac_hi n):  target count of boundary k  */
/* is t_k = floor(n (frac_lo + (frac_hi - frac_lo) k / nslices) + 1/2).     */
/*  1. Proposal: with d_params, features -> network -> the predicted         */
/*     counting function, inverted piecewise linearly at t_k / n; with       */
/*     d_params == NULL, equal widths over the Gershgorin interval (uniform  */
/*     density; the "no network" baseline).  Boundaries with t_k = 0 or n sit */
/*     just outside the Gershgorin interval (exact counts 0 and n).          */
/*  2. Validation: exact inertia counts at every other boundary, all in one  */
/*     batched launch; a boundary is accepted if |count - t_k| <= count_tol. */
/*  3. Fall-back: the rejected boundaries are re-placed together by          */
/*     multisection on inertia (`fanout` points per boundary per launch)     */
/*     inside brackets taken from every count evaluated so far, until each   */
/*     count is within count_tol (or the bracket is a cluster narrower than  */
/*     rounding, where the closest count is kept).                          */
/* Outputs: h_bounds[nslices+1] ascending, h_counts[nslices] exact inertia   */
/* counts of [h_bounds[k], h_bounds[k+1]); optional h_used_fallback = number */
/* of boundaries rejected in step 2, h_inertia_evals = shifts evaluated,     */
/* h_proposed_counts[nslices+1] = exact count below each boundary of step 1 */
/* (before the fall-back; it measures the proposal's quality).  In step 3    */
/* one point per boundary and launch is the regula-falsi estimate on the     */
/* counting function, the other fanout-1 split the bracket evenly (fanout 1: */
/* plain bisection).                                                         */
/* n >= 1, nslices in [1, 1024], fanout in [1, 64].  Synchronous.            */
/* d_work: pdeshep_propose_workspace_size bytes.  NONFINITE_INPUT if the     */
/* band holds NaN/Inf.                                                       */
/* ------------------------------------------------------------------------ */
size_t pdeshep_propose_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nslices,
                                      int32_t fanout);
int pdeshep_propose_slices(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                           const float* d_params, uint64_t seed, double frac_lo, double frac_hi,
                           int32_t nslices, int32_t count_tol, int32_t fanout, double* h_bounds,
                           int32_t* h_counts, int32_t* h_used_fallback, int64_t* h_inertia_evals,
                           int64_t* h_proposed_counts, void* d_work, size_t work_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PDESHEP_H */
