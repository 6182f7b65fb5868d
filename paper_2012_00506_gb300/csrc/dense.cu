// dense.cu -- FP64 kernels of the Rayleigh-Ritz step and CholQR.
//
// FP64 is the scarce resource on sm_103a (about 1.2 TFLOP/s for the whole
// GPU), so these kernels aim at keeping every SM's FP64 pipe busy: the tall
// products (Gram matrices Q^H Q, projections Q^H (BQ), basis updates Q W) are
// a batched split-K GEMM over all slices, and the small per-slice factorizations
// (Cholesky, triangular inverse, Jacobi) run on a thread-block cluster per
// slice with the matrix in L2 and cluster barriers between phases.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "dense.cuh"

namespace cg = cooperative_groups;

namespace pdeshep {

// ---------------------------------------------------------------------------
// batched GEMM, 32 x 32 output tiles, 32-deep k tiles, 256 threads (2 x 2 each).
// FP64 runs at about 2 FMA per clock per SM on this part, so shared-memory
// bandwidth is never the limit and small tiles cost nothing; they cut the
// padding of m0 x m0 outputs (m0 = 267 pads to 288 instead of 320).
// herm: the product is Hermitian (Gram, projection): only tiles with
//   ti <= tj are computed and the lower triangle is filled by conjugation.
// triB: B is upper triangular (R^{-1}): the k loop stops at the tile's last
//   column.
// ---------------------------------------------------------------------------
constexpr int GBM = 32, GBN = 32, GBK = 32;

template <typename S, bool CA>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmItem<S>* items, S alpha, S beta, int splits,
                                                  S* part, int64_t part_stride, int herm, int triB) {
  __shared__ S As[GBK][GBM + 1];
  __shared__ S Bs[GBK][GBN + 1];
  const GemmItem<S> it = items[blockIdx.y];
  const int tm = (it.m + GBM - 1) / GBM, tn = (it.n + GBN - 1) / GBN;
  if ((int)blockIdx.x >= tm * tn) return;
  const int ti = blockIdx.x % tm, tj = blockIdx.x / tm;
  if (herm && ti > tj) return;
  const int i0 = ti * GBM, j0 = tj * GBN;
  const int split = blockIdx.z;
  const int klim = triB ? min(it.k, j0 + GBN) : it.k;
  const int kper = ((klim + splits - 1) / splits + GBK - 1) / GBK * GBK;
  const int kb = split * kper, ke = min(klim, kb + kper);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  S acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) acc[a][c] = sc<S>::zero();
  for (int k0 = kb; k0 < ke; k0 += GBK) {
    for (int e = tid; e < GBM * GBK; e += 256) {
      int i, kk;
      S v = sc<S>::zero();
      if (CA) {
        kk = e % GBK;
        i = e / GBK;
        if (i0 + i < it.m && k0 + kk < ke) v = sc<S>::conj(it.A[(k0 + kk) + (int64_t)(i0 + i) * it.lda]);
      } else {
        i = e % GBM;
        kk = e / GBM;
        if (i0 + i < it.m && k0 + kk < ke) v = it.A[(i0 + i) + (int64_t)(k0 + kk) * it.lda];
      }
      As[kk][i] = v;
    }
    for (int e = tid; e < GBN * GBK; e += 256) {
      const int kk = e % GBK, j = e / GBK;
      S v = sc<S>::zero();
      if (j0 + j < it.n && k0 + kk < ke) v = it.B[(k0 + kk) + (int64_t)(j0 + j) * it.ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GBK; ++kk) {
      const S a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const S b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      sc<S>::fma_(acc[0][0], a0, b0);
      sc<S>::fma_(acc[0][1], a0, b1);
      sc<S>::fma_(acc[1][0], a1, b0);
      sc<S>::fma_(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = i0 + ty + 16 * q, j = j0 + tx + 16 * r;
      if (i >= it.m || j >= it.n) continue;
      if (splits > 1) {
        part[split * part_stride + it.part_off + i + (int64_t)j * it.m] = acc[q][r];
      } else {
        S* cp = it.C + i + (int64_t)j * it.ldc;
        S v = sc<S>::mul(alpha, acc[q][r]);
        if (sc<S>::re(beta) != 0.0 || sc<S>::abs2(beta) != 0.0) v = sc<S>::add(v, sc<S>::mul(beta, *cp));
        *cp = v;
        if (herm && ti < tj) it.C[j + (int64_t)i * it.ldc] = sc<S>::conj(v);
      }
    }
}

template <typename S>
__global__ void gemm_reduce_kernel(const GemmItem<S>* items, S alpha, S beta, int splits, const S* part,
                                   int64_t part_stride, int herm) {
  const GemmItem<S> it = items[blockIdx.y];
  const int64_t total = (int64_t)it.m * it.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % it.m), j = (int)(e / it.m);
    const int ti = i / GBM, tj = j / GBN;
    if (herm && ti > tj) continue;
    S s = sc<S>::zero();
    for (int p = 0; p < splits; ++p) s = sc<S>::add(s, part[p * part_stride + it.part_off + e]);
    S* cp = it.C + i + (int64_t)j * it.ldc;
    S v = sc<S>::mul(alpha, s);
    if (sc<S>::re(beta) != 0.0 || sc<S>::abs2(beta) != 0.0) v = sc<S>::add(v, sc<S>::mul(beta, *cp));
    *cp = v;
    if (herm && ti < tj) it.C[j + (int64_t)i * it.ldc] = sc<S>::conj(v);
  }
}

template <typename S>
int launch_gemm(bool conjA, int nitems, const GemmItem<S>* d_items, int max_m, int max_n, int max_k, S alpha,
                S beta, int splits, S* part, int64_t part_stride, cudaStream_t st, int herm, int triB) {
  if (nitems <= 0 || max_m <= 0 || max_n <= 0) return 0;
  if (max_k <= 0) splits = 1;
  if (splits < 1) splits = 1;
  dim3 grid((unsigned)(ceil_div(max_m, GBM) * ceil_div(max_n, GBN)), (unsigned)nitems, (unsigned)splits);
  if (conjA)
    gemm_kernel<S, true><<<grid, 256, 0, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
  else
    gemm_kernel<S, false><<<grid, 256, 0, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
  PD_CK_LAUNCH();
  if (splits > 1) {
    int blocks = (int)ceil_div((int64_t)max_m * max_n, 256);
    if (blocks > 1024) blocks = 1024;
    gemm_reduce_kernel<S><<<dim3(blocks, nitems), 256, 0, st>>>(d_items, alpha, beta, splits, part, part_stride,
                                                               herm);
    PD_CK_LAUNCH();
  }
  return 0;
}

// ---------------------------------------------------------------------------
// cluster helpers
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 256;
static int g_cluster_ctas = 16;  // CTAs per slice; falls back to the portable 8 if 16 cannot launch

__device__ __forceinline__ int cl_rank() { return (int)cg::this_cluster().block_rank(); }
__device__ __forceinline__ int cl_size() { return (int)cg::this_cluster().num_blocks(); }
__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
__device__ __forceinline__ int cl_slice() { return blockIdx.x / cl_size(); }

template <typename K, typename... Args>
static int launch_cluster(K kernel, int nblk, size_t smem, cudaStream_t st, Args... args) {
  for (;;) {
    const int G = g_cluster_ctas;
    if (G > 8) PD_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nblk * G));
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (G > 8) {
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        g_cluster_ctas = 8;
        continue;
      }
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess && G > 8) {
      cudaGetLastError();
      g_cluster_ctas = 8;
      continue;
    }
    PD_CK(e);
    count_launch();
    return 0;
  }
}

// ---------------------------------------------------------------------------
// Cholesky G = R^H R, upper, in place; one cluster per block
// ---------------------------------------------------------------------------
template <typename S>
__global__ void cholesky_kernel(const SmallDesc* desc, S* Gall, int* info, double* diag0, double* minratio) {
  const int t = cl_slice();
  const SmallDesc d = desc[t];
  const int m = d.m;
  S* G = Gall + d.off;
  const int gid = cl_rank() * blockDim.x + threadIdx.x, gsz = cl_size() * blockDim.x;
  if (diag0) {
    for (int i = gid; i < m; i += gsz) diag0[d.voff + i] = sc<S>::re(G[i + (int64_t)i * m]);
    cl_sync();
  }
  int bad = 0;
  for (int j = 0; j < m; ++j) {
    const double dj = sc<S>::re(G[j + (int64_t)j * m]);
    if (!(dj > 0.0) || !isfinite(dj)) {
      bad = j + 1;
      break;
    }
    const double r = sqrt(dj);
    const double ri = 1.0 / r;
    for (int i = j + 1 + gid; i < m; i += gsz) G[j + (int64_t)i * m] = sc<S>::scale(G[j + (int64_t)i * m], ri);
    cl_sync();
    const int tt = m - j - 1;
    for (int64_t e = gid; e < (int64_t)tt * tt; e += gsz) {
      const int i = j + 1 + (int)(e % tt), k = j + 1 + (int)(e / tt);
      if (i > k) continue;
      // G(i,k) -= conj(R(j,i)) R(j,k)
      S v = G[i + (int64_t)k * m];
      const S a = sc<S>::conj(G[j + (int64_t)i * m]);
      const S b = G[j + (int64_t)k * m];
      v = sc<S>::sub(v, sc<S>::mul(a, b));
      G[i + (int64_t)k * m] = v;
    }
    if (gid == 0) G[j + (int64_t)j * m] = sc<S>::from_re(r);
    cl_sync();
  }
  // clear the strict lower triangle
  for (int64_t e = gid; e < (int64_t)m * m; e += gsz) {
    const int i = (int)(e % m), k = (int)(e / m);
    if (i > k) G[e] = sc<S>::zero();
  }
  if (gid == 0) info[t] = bad;
  // min over columns of r_cc^2 / G_cc: the squared sine of the angle between column c
  // and the span of the previous ones (small => ill-conditioned, repeat the pass)
  if (diag0 && minratio && cl_rank() == 0) {
    __shared__ double red[32];
    double mn = bad ? 0.0 : 1.0;
    if (!bad)
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        const double r = sc<S>::re(G[c + (int64_t)c * m]);
        const double g0 = diag0[d.voff + c];
        mn = fmin(mn, g0 > 0.0 ? r * r / g0 : 0.0);
      }
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mn = fmin(mn, red[w]);
      minratio[t] = mn;
    }
  }
}

template <typename S>
int launch_cholesky(int nblk, const SmallDesc* d_desc, S* G, int* info, cudaStream_t st, double* diag0,
                    double* minratio) {
  if (nblk <= 0) return 0;
  return launch_cluster(cholesky_kernel<S>, nblk, 0, st, d_desc, G, info, diag0, minratio);
}

// ---------------------------------------------------------------------------
// upper triangular inverse, column per thread
// ---------------------------------------------------------------------------
template <typename S>
__global__ void triinv_kernel(const SmallDesc* desc, const S* Rall, S* Iall) {
  const int t = cl_slice();
  const SmallDesc d = desc[t];
  const int m = d.m;
  const S* R = Rall + d.off;
  S* X = Iall + d.off;
  const int gid = cl_rank() * blockDim.x + threadIdx.x, gsz = cl_size() * blockDim.x;
  for (int j = gid; j < m; j += gsz) {
    S* x = X + (int64_t)j * m;
    for (int i = j + 1; i < m; ++i) x[i] = sc<S>::zero();
    const double rjj = sc<S>::re(R[j + (int64_t)j * m]);
    x[j] = sc<S>::from_re(1.0 / rjj);
    for (int i = j - 1; i >= 0; --i) {
      S s = sc<S>::zero();
      for (int k = i + 1; k <= j; ++k) sc<S>::fma_(s, R[i + (int64_t)k * m], x[k]);
      const double rii = sc<S>::re(R[i + (int64_t)i * m]);
      x[i] = sc<S>::scale(s, -1.0 / rii);
    }
  }
}

template <typename S>
int launch_triinv(int nblk, const SmallDesc* d_desc, const S* R, S* Rinv, cudaStream_t st) {
  if (nblk <= 0) return 0;
  return launch_cluster(triinv_kernel<S>, nblk, 0, st, d_desc, R, Rinv);
}

// ---------------------------------------------------------------------------
// Jacobi eigensolver, parallel (round-robin) ordering, one cluster per block.
// Pairs of round r among M players (M = m rounded up to even; player m is a
// dummy when m is odd): (r mod (M-1), M-1) and ((r+i) mod (M-1),
// (r-i+M-1) mod (M-1)), i = 1..M/2-1; every pair meets once per sweep.
// ---------------------------------------------------------------------------
template <typename S>
struct Rot {
  typename real_t<S>::type c, s;
  S u;  // phase of A(p,q)
  int p, q;
};

template <typename S>
__device__ __forceinline__ void make_rot(const S* A, int m, int p, int q, Rot<S>& r) {
  using R = typename real_t<S>::type;
  r.p = p;
  r.q = q;
  r.c = R(1);
  r.s = R(0);
  r.u = sc<S>::from_re(R(1));
  if (p >= m || q >= m) {
    r.p = -1;
    return;
  }
  const S apq = A[p + (int64_t)q * m];
  const R g = sqrt(sc<S>::abs2(apq));
  const R tiny = sizeof(R) == 8 ? R(1e-300) : R(1e-35);
  if (!(g > tiny)) {
    r.p = -1;
    return;
  }
  r.u = sc<S>::scale(apq, R(1) / g);
  const R app = sc<S>::re(A[p + (int64_t)p * m]), aqq = sc<S>::re(A[q + (int64_t)q * m]);
  const R th = (aqq - app) / (R(2) * g);
  const R t = (th >= R(0) ? R(1) : R(-1)) / (fabs(th) + sqrt(th * th + R(1)));
  r.c = R(1) / sqrt(t * t + R(1));
  r.s = t * r.c;
}

template <typename S>
__global__ void jacobi_kernel(const SmallDesc* desc, S* Aall, S* Vall, S* Vout, double* lamall,
                              double tol, int max_sweeps, int* sweeps_out, double* scratch) {
  using R = typename real_t<S>::type;
  extern __shared__ __align__(16) char smem[];
  Rot<S>* rot = (Rot<S>*)smem;
  __shared__ double red[2][kSmallThreads / 32];
  const int t = cl_slice();
  const SmallDesc d = desc[t];
  const int m = d.m;
  S* A = Aall + d.off;
  S* V = Vall + d.off;
  const int cr = cl_rank(), G = cl_size();
  const int gid = cr * blockDim.x + threadIdx.x, gsz = G * blockDim.x;
  const int M = m + (m & 1);
  const int np = M / 2;
  double* part = scratch + (int64_t)t * 2 * G;

  for (int64_t e = gid; e < (int64_t)m * m; e += gsz) {
    const int i = (int)(e % m), k = (int)(e / m);
    V[e] = sc<S>::from_re(i == k ? R(1) : R(0));
  }
  cl_sync();
  int sweeps = 0, converged = 0;
  for (;; ++sweeps) {
    // off-norm and Frobenius norm (deterministic: per-CTA partials summed in order)
    double off = 0.0, fro = 0.0;
    for (int64_t e = gid; e < (int64_t)m * m; e += gsz) {
      const int i = (int)(e % m), k = (int)(e / m);
      const double a2 = (double)sc<S>::abs2(A[e]);
      fro += a2;
      if (i != k) off += a2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      fro += __shfl_down_sync(0xffffffffu, fro, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = off;
      red[1][threadIdx.x >> 5] = fro;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, sf = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        so += red[0][w];
        sf += red[1][w];
      }
      part[2 * cr] = so;
      part[2 * cr + 1] = sf;
    }
    cl_sync();
    double so = 0.0, sf = 0.0;
    for (int c = 0; c < G; ++c) {
      so += part[2 * c];
      sf += part[2 * c + 1];
    }
    cl_sync();  // partials may be overwritten next sweep only after everyone read them
    if (sqrt(so) <= tol * sqrt(sf) || sf == 0.0) {
      converged = 1;
      break;
    }
    if (sweeps >= max_sweeps) break;
    for (int r = 0; r < M - 1; ++r) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = r % (M - 1);
          q = M - 1;
        } else {
          p = (r + i) % (M - 1);
          q = (r - i + M - 1) % (M - 1);
        }
        make_rot<S>(A, m, p, q, rot[i]);
      }
      // every CTA must have read the pivots of this round before any column changes
      cl_sync();
      // columns of A and V: A <- A J, V <- V J
      for (int64_t e = gid; e < (int64_t)np * m; e += gsz) {
        const int i = (int)(e / m), k = (int)(e % m);
        const Rot<S> ro = rot[i];
        if (ro.p < 0) continue;
        const S uc = sc<S>::scale(ro.u, ro.c), us = sc<S>::scale(ro.u, ro.s);
        S* ap = A + (int64_t)ro.p * m;
        S* aq = A + (int64_t)ro.q * m;
        S akp = ap[k], akq = aq[k];
        ap[k] = sc<S>::sub(sc<S>::mul(akp, uc), sc<S>::scale(akq, ro.s));
        aq[k] = sc<S>::add(sc<S>::mul(akp, us), sc<S>::scale(akq, ro.c));
        S* vp = V + (int64_t)ro.p * m;
        S* vq = V + (int64_t)ro.q * m;
        S vkp = vp[k], vkq = vq[k];
        vp[k] = sc<S>::sub(sc<S>::mul(vkp, uc), sc<S>::scale(vkq, ro.s));
        vq[k] = sc<S>::add(sc<S>::mul(vkp, us), sc<S>::scale(vkq, ro.c));
      }
      cl_sync();
      // rows of A: A <- J^H A
      for (int64_t e = gid; e < (int64_t)np * m; e += gsz) {
        const int i = (int)(e % np), k = (int)(e / np);
        const Rot<S> ro = rot[i];
        if (ro.p < 0) continue;
        const S ucc = sc<S>::conj(sc<S>::scale(ro.u, ro.c)), usc = sc<S>::conj(sc<S>::scale(ro.u, ro.s));
        S* col = A + (int64_t)k * m;
        const S apk = col[ro.p], aqk = col[ro.q];
        S np_ = sc<S>::sub(sc<S>::mul(ucc, apk), sc<S>::scale(aqk, ro.s));
        S nq_ = sc<S>::add(sc<S>::mul(usc, apk), sc<S>::scale(aqk, ro.c));
        if (k == ro.q) np_ = sc<S>::zero();
        if (k == ro.p) {
          nq_ = sc<S>::zero();
          np_ = sc<S>::from_re(sc<S>::re(np_));
        }
        if (k == ro.q) nq_ = sc<S>::from_re(sc<S>::re(nq_));
        col[ro.p] = np_;
        col[ro.q] = nq_;
      }
      cl_sync();
    }
  }
  // sort ascending by eigenvalue (rank sort, ties by index), phase-normalise
  double* lam = lamall + d.voff;
  for (int i = gid; i < m; i += gsz) {
    const R li = sc<S>::re(A[i + (int64_t)i * m]);
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      const R lj = sc<S>::re(A[j + (int64_t)j * m]);
      rank += (lj < li) || (lj == li && j < i);
    }
    lam[rank] = li;
    // phase of the first largest-magnitude component
    const S* v = V + (int64_t)i * m;
    int kb = 0;
    R best = R(-1);
    for (int k = 0; k < m; ++k) {
      const R a = sc<S>::abs2(v[k]);
      if (a > best) {
        best = a;
        kb = k;
      }
    }
    const R nb = sqrt(best);
    S ph = sc<S>::from_re(R(1));
    if (nb > R(0)) ph = sc<S>::scale(sc<S>::conj(v[kb]), R(1) / nb);
    S* vo = Vout + d.off + (int64_t)rank * m;
    for (int k = 0; k < m; ++k) vo[k] = sc<S>::mul(v[k], ph);
    vo[kb] = sc<S>::from_re(nb);
  }
  if (gid == 0) sweeps_out[t] = converged ? sweeps : -1;
}

template <typename S>
int launch_jacobi(int nblk, const SmallDesc* d_desc, int max_m, S* A, S* Vwork, S* Vout, double* lam,
                  double tol, int max_sweeps, int* sweeps_out, double* scratch, cudaStream_t st) {
  if (nblk <= 0) return 0;
  const size_t smem = sizeof(Rot<S>) * (size_t)((max_m + 2) / 2);
  if (smem > 48 * 1024) PD_CK(cudaFuncSetAttribute(jacobi_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return launch_cluster(jacobi_kernel<S>, nblk, smem, st, d_desc, A, Vwork, Vout, lam, tol, max_sweeps,
                        sweeps_out, scratch);
}

// ---------------------------------------------------------------------------
// Y = B X for the Hermitian band.  Block: 32 rows x 8 columns (one warp per
// column); band entries of the 32 rows are reused by the 8 warps through L1.
// ---------------------------------------------------------------------------
template <typename S, bool CPLXB>
__global__ void __launch_bounds__(256) band_matmul_kernel(int64_t n, int b, const double* __restrict__ band,
                                                         int64_t ldab, int ncols, const S* __restrict__ X,
                                                         S* __restrict__ Y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const int c = blockIdx.y * 8 + warp;
  if (i >= n || c >= ncols) return;
  const S* x = X + (int64_t)c * n;
  S acc = sc<S>::zero();
  const int64_t j0 = i - b < 0 ? 0 : i - b, j1 = i + b > n - 1 ? n - 1 : i + b;
  for (int64_t j = j0; j <= j1; ++j) {
    S bij;
    if constexpr (CPLXB) {
      double re, im;
      if (j <= i) {
        const double* p = band + 2 * ((i - j) + j * ldab);
        re = p[0];
        im = (j == i) ? 0.0 : p[1];
      } else {
        const double* p = band + 2 * ((j - i) + i * ldab);
        re = p[0];
        im = -p[1];
      }
      bij = make_double2(re, im);
      sc<double2>::fma_(acc, bij, x[j]);
    } else {
      const double v = j <= i ? band[(i - j) + j * ldab] : band[(j - i) + i * ldab];
      sc<S>::fma_(acc, sc<S>::from_re(v), x[j]);
    }
  }
  Y[i + (int64_t)c * n] = acc;
}

template <typename S>
int launch_band_matmul(int64_t n, int b, const void* band, int64_t ldab, int ncols, const S* X, S* Y,
                       cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return 0;
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(ncols, 8));
  if constexpr (std::is_same<S, double2>::value)
    band_matmul_kernel<double2, true><<<grid, 256, 0, st>>>(n, b, (const double*)band, ldab, ncols, X, Y);
  else
    band_matmul_kernel<double, false><<<grid, 256, 0, st>>>(n, b, (const double*)band, ldab, ncols, X, Y);
  PD_CK_LAUNCH();
  return 0;
}

// ---------------------------------------------------------------------------
// mixed-precision small eigensolver
// ---------------------------------------------------------------------------
template <typename A, typename Bt>
__global__ void small_cast_kernel(const SmallDesc* desc, const A* __restrict__ src, Bt* __restrict__ dst) {
  const SmallDesc d = desc[blockIdx.y];
  const int64_t total = (int64_t)d.m * d.m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const A v = src[d.off + e];
    Bt w;
    if constexpr (std::is_same<A, double>::value || std::is_same<A, float>::value) {
      w = (Bt)v;
    } else {
      w.x = (typename real_t<Bt>::type)v.x;
      w.y = (typename real_t<Bt>::type)v.y;
    }
    dst[d.off + e] = w;
  }
}

// first largest-magnitude component of each column real and positive
template <typename S>
__global__ void phase_kernel(const SmallDesc* desc, S* Wall) {
  const SmallDesc d = desc[blockIdx.y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = blockIdx.x * nw + warp; c < d.m; c += gridDim.x * nw) {
    S* v = Wall + d.off + (int64_t)c * d.m;
    double best = -1.0;
    int kb = d.m;
    for (int k = lane; k < d.m; k += 32) {
      const double a = sc<S>::abs2(v[k]);
      if (a > best) {
        best = a;
        kb = k;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int ok = __shfl_down_sync(0xffffffffu, kb, o);
      if (ob > best || (ob == best && ok < kb)) {
        best = ob;
        kb = ok;
      }
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    kb = __shfl_sync(0xffffffffu, kb, 0);
    const double nb = sqrt(best);
    if (!(nb > 0.0)) continue;
    const S ph = sc<S>::scale(sc<S>::conj(v[kb]), 1.0 / nb);
    for (int k = lane; k < d.m; k += 32) v[k] = (k == kb) ? sc<S>::from_re(nb) : sc<S>::mul(v[k], ph);
  }
}

template <typename S>
EighScratch<S> plan_eigh_scratch(Arena& a, int64_t msq, int64_t mtot, int nblk) {
  using L = typename lowp<S>::type;
  EighScratch<S> w;
  w.A32 = a.take<L>(msq);
  w.V32w = a.take<L>(msq);
  w.V32 = a.take<L>(msq);
  w.Vd = a.take<S>(msq);
  w.T = a.take<S>(msq);
  w.Vw = a.take<S>(msq);
  w.W64 = a.take<S>(msq);
  w.lam32 = a.take<double>(mtot);
  w.sweeps = a.take<int>(nblk);
  w.jscratch = a.take<double>((size_t)nblk * 2 * 16);
  w.items = a.take<GemmItem<S>>(nblk);
  return w;
}

template <typename S>
int eigh_mixed(int nblk, const SmallDesc* d_desc, const SmallDesc* h_desc, int max_m, S* A, double* lam, S* W,
               const EighScratch<S>& w, cudaStream_t st, int* fp64_sweeps_out) {
  using L = typename lowp<S>::type;
  if (nblk <= 0) return 0;
  const dim3 g((unsigned)std::min<int64_t>(ceil_div((int64_t)max_m * max_m, 256), 512), (unsigned)nblk);
  small_cast_kernel<S, L><<<g, 256, 0, st>>>(d_desc, A, w.A32);
  PD_CK_LAUNCH();
  PD_TRY(launch_jacobi<L>(nblk, d_desc, max_m, w.A32, w.V32w, w.V32, w.lam32, 2e-6, 20, w.sweeps, w.jscratch, st));
  small_cast_kernel<L, S><<<g, 256, 0, st>>>(d_desc, w.V32, w.Vd);
  PD_CK_LAUNCH();
  S one, zero;
  if constexpr (std::is_same<S, double>::value) {
    one = 1.0;
    zero = 0.0;
  } else {
    one = make_double2(1.0, 0.0);
    zero = make_double2(0.0, 0.0);
  }
  std::vector<GemmItem<S>> it(nblk);
  // V32 is unitary only to FP32 accuracy: orthonormalise it in FP64 (one CholQR
  // pass, its Gram matrix is I + O(1e-7)) so that V^H A V is a similarity.
  for (int t = 0; t < nblk; ++t) {
    const int m = h_desc[t].m;
    const int64_t o = h_desc[t].off;
    it[t] = GemmItem<S>{w.Vd + o, w.Vd + o, w.T + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(true, nblk, w.items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, 1, 0));
  PD_TRY(launch_cholesky<S>(nblk, d_desc, w.T, w.sweeps, st));
  PD_TRY(launch_triinv<S>(nblk, d_desc, w.T, w.Vw, st));
  for (int t = 0; t < nblk; ++t) {
    const int m = h_desc[t].m;
    const int64_t o = h_desc[t].off;
    it[t] = GemmItem<S>{w.Vd + o, w.Vw + o, w.W64 + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(false, nblk, w.items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, 0, 1));
  PD_CK(cudaMemcpyAsync(w.Vd, w.W64, sizeof(S) * (size_t)(h_desc[nblk - 1].off + (int64_t)h_desc[nblk - 1].m *
                                                                                       h_desc[nblk - 1].m),
                        cudaMemcpyDeviceToDevice, st));
  // T = A Vd
  for (int t = 0; t < nblk; ++t) {
    const int m = h_desc[t].m;
    const int64_t o = h_desc[t].off;
    it[t] = GemmItem<S>{A + o, w.Vd + o, w.T + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(false, nblk, w.items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, 0, 0));
  // H = Vd^H T (into A)
  for (int t = 0; t < nblk; ++t) {
    const int m = h_desc[t].m;
    const int64_t o = h_desc[t].off;
    it[t] = GemmItem<S>{w.Vd + o, w.T + o, A + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(true, nblk, w.items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, 1, 0));
  PD_TRY(launch_jacobi<S>(nblk, d_desc, max_m, A, w.Vw, w.W64, lam, 1e-14, 60, w.sweeps, w.jscratch, st));
  if (fp64_sweeps_out) PD_CK(cudaMemcpyAsync(fp64_sweeps_out, w.sweeps, sizeof(int) * nblk, cudaMemcpyDeviceToDevice, st));
  // W = Vd W64
  for (int t = 0; t < nblk; ++t) {
    const int m = h_desc[t].m;
    const int64_t o = h_desc[t].off;
    it[t] = GemmItem<S>{w.Vd + o, w.W64 + o, W + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.items, it.data(), sizeof(GemmItem<S>) * nblk, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(false, nblk, w.items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, 0, 0));
  phase_kernel<S><<<dim3((unsigned)ceil_div(max_m, 8), nblk), 256, 0, st>>>(d_desc, W);
  PD_CK_LAUNCH();
  return 0;
}

// explicit instantiations
template EighScratch<double> plan_eigh_scratch<double>(Arena&, int64_t, int64_t, int);
template EighScratch<double2> plan_eigh_scratch<double2>(Arena&, int64_t, int64_t, int);
template int eigh_mixed<double>(int, const SmallDesc*, const SmallDesc*, int, double*, double*, double*,
                                const EighScratch<double>&, cudaStream_t, int*);
template int eigh_mixed<double2>(int, const SmallDesc*, const SmallDesc*, int, double2*, double*, double2*,
                                 const EighScratch<double2>&, cudaStream_t, int*);
template int launch_gemm<double>(bool, int, const GemmItem<double>*, int, int, int, double, double, int,
                                 double*, int64_t, cudaStream_t, int, int);
template int launch_gemm<double2>(bool, int, const GemmItem<double2>*, int, int, int, double2, double2, int,
                                  double2*, int64_t, cudaStream_t, int, int);
template int launch_cholesky<double>(int, const SmallDesc*, double*, int*, cudaStream_t, double*, double*);
template int launch_cholesky<double2>(int, const SmallDesc*, double2*, int*, cudaStream_t, double*, double*);
template int launch_triinv<double>(int, const SmallDesc*, const double*, double*, cudaStream_t);
template int launch_triinv<double2>(int, const SmallDesc*, const double2*, double2*, cudaStream_t);
template int launch_jacobi<double>(int, const SmallDesc*, int, double*, double*, double*, double*, double,
                                   int, int*, double*, cudaStream_t);
template int launch_jacobi<double2>(int, const SmallDesc*, int, double2*, double2*, double2*, double*,
                                    double, int, int*, double*, cudaStream_t);
template int launch_jacobi<float>(int, const SmallDesc*, int, float*, float*, float*, double*, double, int,
                                  int*, double*, cudaStream_t);
template int launch_jacobi<float2>(int, const SmallDesc*, int, float2*, float2*, float2*, double*, double,
                                   int, int*, double*, cudaStream_t);
template int launch_band_matmul<double>(int64_t, int, const void*, int64_t, int, const double*, double*,
                                        cudaStream_t);
template int launch_band_matmul<double2>(int64_t, int, const void*, int64_t, int, const double2*,
                                         double2*, cudaStream_t);

}  // namespace pdeshep
