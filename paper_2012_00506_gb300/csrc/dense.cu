// dense.cu -- FP64 kernels of the Rayleigh-Ritz step and CholQR.
//
// FP64 is the scarce resource on sm_103a (about 1.2 TFLOP/s for the whole
// GPU), so these kernels aim at keeping every SM's FP64 pipe busy: the tall
// products (Gram matrices Q^H Q, projections Q^H (BQ), basis updates Q W) are
// a batched split-K GEMM over all slices, and the small per-slice factorizations
// (Cholesky, triangular inverse, Jacobi) run on a thread-block cluster per
// slice with the matrix in L2 and cluster barriers between phases.
#include <cooperative_groups.h>

#include <stdlib.h>

#include <algorithm>
#include <map>
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

// ---------------------------------------------------------------------------
// The same products in float-float arithmetic on the FP32 pipes.  GB300 runs
// FP32 at 64 times its FP64 rate, so an FP64 operand is split into a pair of
// floats (hi = fl(v), lo = fl(v - hi): about 48 significant bits) and every
// product is accumulated error-free (exact product by an FMA, exact sum by
// Knuth's two-sum) into a (hi, lo) accumulator; the cross terms hi*lo enter
// the low word and lo*lo is dropped.  Relative accuracy of a length-K dot
// product is about 2^-48 sqrt(K) in practice, far inside the 1e-10 residual
// target; the exponent range is FP32's (operands above ~1e-19 in magnitude
// keep full precision).  Tiles: 64 x 64 outputs per CTA of 512 threads, 4 x 2
// per thread, k-steps of 16 staged in shared memory as (hi, lo) pairs.
// ---------------------------------------------------------------------------
constexpr int FBM = 64, FBN = 64, FBK = 16, FFT = 512;

template <typename S>
struct ffv;  // a split operand in shared memory
template <>
struct ffv<double> {
  using type = float2;  // (hi, lo)
};
template <>
struct ffv<double2> {
  using type = float4;  // (re hi, re lo, im hi, im lo)
};

__device__ __forceinline__ float2 ff_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ void ff_load(double v, bool conj, float2& o) {
  (void)conj;
  o = ff_split(v);
}
__device__ __forceinline__ void ff_load(double2 v, bool conj, float4& o) {
  const float2 a = ff_split(v.x), b = ff_split(conj ? -v.y : v.y);
  o = make_float4(a.x, a.y, b.x, b.y);
}

// (h, l) += x * y exactly up to the dropped x_lo * y_lo and the rounding of l
__device__ __forceinline__ void ff_mac(float& h, float& l, float xh, float xl, float yh, float yl) {
  const float p = xh * yh;
  const float e = fmaf(xh, yh, -p);
  const float c = fmaf(xh, yl, xl * yh);
  const float s = h + p;
  const float bb = s - h;
  const float t = (h - (s - bb)) + (p - bb);
  h = s;
  l += t + (e + c);
}

struct ffacc1 {
  float h, l;
};
struct ffacc2 {
  float rh, rl, ih, il;
};
__device__ __forceinline__ void ff_fma(ffacc1& a, float2 x, float2 y) { ff_mac(a.h, a.l, x.x, x.y, y.x, y.y); }
__device__ __forceinline__ void ff_fma(ffacc2& a, float4 x, float4 y) {
  // (xr + i xi)(yr + i yi) = (xr yr - xi yi) + i (xr yi + xi yr)
  ff_mac(a.rh, a.rl, x.x, x.y, y.x, y.y);
  ff_mac(a.rh, a.rl, -x.z, -x.w, y.z, y.w);
  ff_mac(a.ih, a.il, x.x, x.y, y.z, y.w);
  ff_mac(a.ih, a.il, x.z, x.w, y.x, y.y);
}
__device__ __forceinline__ double ff_val(const ffacc1& a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double2 ff_val(const ffacc2& a) {
  return make_double2((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il);
}

template <typename S, bool CA>
__global__ void __launch_bounds__(FFT) ffgemm_kernel(const GemmItem<S>* items, S alpha, S beta, int splits,
                                                    S* part, int64_t part_stride, int herm, int triB) {
  using V = typename ffv<S>::type;
  using ACC = typename std::conditional<std::is_same<S, double2>::value, ffacc2, ffacc1>::type;
  // two stages of the (hi, lo) tiles: the next k-step's operands are fetched
  // into registers before the current step's products and split into the other
  // stage after them, so the FP64-pipe splitting overlaps other warps' FMAs
  extern __shared__ __align__(16) unsigned char ffsm[];
  V(*As)[FBK][FBM] = reinterpret_cast<V(*)[FBK][FBM]>(ffsm);
  V(*Bs)[FBK][FBN] = reinterpret_cast<V(*)[FBK][FBN]>(ffsm + 2 * sizeof(V) * FBK * FBM);
  const GemmItem<S> it = items[blockIdx.y];
  const int tm = (it.m + FBM - 1) / FBM, tn = (it.n + FBN - 1) / FBN;
  if ((int)blockIdx.x >= tm * tn) return;
  const int ti = blockIdx.x % tm, tj = blockIdx.x / tm;
  if (herm && ti > tj) return;
  const int i0 = ti * FBM, j0 = tj * FBN;
  const int split = blockIdx.z;
  const int klim = triB ? min(it.k, j0 + FBN) : it.k;
  const int kper = ((klim + splits - 1) / splits + FBK - 1) / FBK * FBK;
  const int kb = split * kper, ke = min(klim, kb + kper);
  // 512 threads: thread (tx, ty) owns rows ty + 16 q (q < 4) and columns tx + 32 r (r < 2)
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  constexpr int NA = (FBM * FBK) / FFT, NB = (FBN * FBK) / FFT;
  S ra[NA], rb[NB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + q * FFT;
      ra[q] = sc<S>::zero();
      if (CA) {  // A stored k x m: read along k
        const int kk = e % FBK, i = e / FBK;
        if (i0 + i < it.m && k0 + kk < ke) ra[q] = it.A[(k0 + kk) + (int64_t)(i0 + i) * it.lda];
      } else {   // A stored m x k: read along m
        const int i = e % FBM, kk = e / FBM;
        if (i0 + i < it.m && k0 + kk < ke) ra[q] = it.A[(i0 + i) + (int64_t)(k0 + kk) * it.lda];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * FFT;
      const int kk = e % FBK, j = e / FBK;
      rb[q] = sc<S>::zero();
      if (j0 + j < it.n && k0 + kk < ke) rb[q] = it.B[(k0 + kk) + (int64_t)(j0 + j) * it.ldb];
    }
  };
  auto stash = [&](int stg) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + q * FFT;
      const int kk = CA ? e % FBK : e / FBM, i = CA ? e / FBK : e % FBM;
      ff_load(ra[q], CA, As[stg][kk][i]);
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * FFT;
      ff_load(rb[q], false, Bs[stg][e % FBK][e / FBK]);
    }
  };
  ACC acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) acc[a][c] = ACC{};
  int stg = 0;
  if (kb < ke) {
    fetch(kb);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += FBK) {
    const bool more = k0 + FBK < ke;
    if (more) fetch(k0 + FBK);
#pragma unroll 4
    for (int kk = 0; kk < FBK; ++kk) {
      V a[4], b[2];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[stg][kk][ty + 16 * q];
#pragma unroll
      for (int r = 0; r < 2; ++r) b[r] = Bs[stg][kk][tx + 32 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 2; ++r) ff_fma(acc[q][r], a[q], b[r]);
    }
    if (more) stash(stg ^ 1);
    __syncthreads();
    stg ^= 1;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = i0 + ty + 16 * q, j = j0 + tx + 32 * r;
      if (i >= it.m || j >= it.n) continue;
      const S val = ff_val(acc[q][r]);
      if (splits > 1) {
        part[split * part_stride + it.part_off + i + (int64_t)j * it.m] = val;
      } else {
        S* cp = it.C + i + (int64_t)j * it.ldc;
        S v = sc<S>::mul(alpha, val);
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
                S beta, int splits, S* part, int64_t part_stride, cudaStream_t st, int herm, int triB, int ff) {
  if (nitems <= 0 || max_m <= 0 || max_n <= 0) return 0;
  if (max_k <= 0) splits = 1;
  if (splits < 1) splits = 1;
  if (ff) {
    dim3 grid((unsigned)(ceil_div(max_m, FBM) * ceil_div(max_n, FBN)), (unsigned)nitems, (unsigned)splits);
    const size_t smem = 2 * sizeof(typename ffv<S>::type) * FBK * (FBM + FBN);
    if (conjA) {
      PD_CK(cudaFuncSetAttribute(ffgemm_kernel<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ffgemm_kernel<S, true><<<grid, FFT, smem, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
    } else {
      PD_CK(cudaFuncSetAttribute(ffgemm_kernel<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      ffgemm_kernel<S, false><<<grid, FFT, smem, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
    }
  } else {
    dim3 grid((unsigned)(ceil_div(max_m, GBM) * ceil_div(max_n, GBN)), (unsigned)nitems, (unsigned)splits);
    if (conjA)
      gemm_kernel<S, true><<<grid, 256, 0, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
    else
      gemm_kernel<S, false><<<grid, 256, 0, st>>>(d_items, alpha, beta, splits, part, part_stride, herm, triB);
  }
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
// Cluster shape of the per-slice kernels: 16 CTAs (non-portable) with one CTA
// per SM (forced by a large dynamic shared-memory request, since these kernels
// are FP64-pipe bound and two CTAs on one SM would share it); falls back to
// 8 CTAs, then to 8 CTAs without the SM-spreading request.
struct ClusterShape {
  int ctas;
  size_t spread_smem;
};
static const ClusterShape kShapes[] = {{16, 120 * 1024}, {8, 120 * 1024}, {8, 0}};
static int g_shape = 0;
static int g_last_ctas = 0;  // cluster size of the last cluster launch

int cluster_ctas_used() { return g_last_ctas ? g_last_ctas : kShapes[g_shape].ctas; }

__device__ __forceinline__ int cl_rank() { return (int)cg::this_cluster().block_rank(); }
__device__ __forceinline__ int cl_size() { return (int)cg::this_cluster().num_blocks(); }
__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }
__device__ __forceinline__ int cl_slice() { return blockIdx.x / cl_size(); }

// Per launch, with `resident`, the widest shape whose nblk clusters are all
// resident at once (a 16-CTA cluster needs 16 SMs of one GPC, so only a few
// fit); otherwise, or if none fits, the widest usable shape.  Occupancy answers
// are cached per kernel and shape.
static std::map<std::pair<const void*, int>, int> g_cluster_fit;

template <typename K, typename... Args>
static int launch_cluster_t(bool resident, K kernel, int nblk, size_t smem, int threads, cudaStream_t st,
                            Args... args) {
  const int nshapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));
  for (;;) {
    int pick = -1;
    for (int sidx = g_shape; sidx < nshapes; ++sidx) {
      const ClusterShape sh = kShapes[sidx];
      const size_t dyn = std::max(smem, sh.spread_smem);
      const auto key = std::make_pair((const void*)kernel, sidx * 4096 + (int)(dyn >> 10));
      auto it = g_cluster_fit.find(key);
      int nc = 0;
      if (it != g_cluster_fit.end()) {
        nc = it->second;
      } else {
        cudaError_t e = cudaSuccess;
        if (sh.ctas > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess && dyn > 48 * 1024)
          e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nblk * sh.ctas));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = dyn;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = sh.ctas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&nc, kernel, &cfg);
        if (e != cudaSuccess) {
          cudaGetLastError();
          nc = 0;
        }
        g_cluster_fit[key] = nc;
      }
      if (nc < 1) continue;
      if (pick < 0) pick = sidx;          // widest usable
      if (!resident) break;
      if (nc >= nblk) {                   // widest with every cluster resident
        pick = sidx;
        break;
      }
    }
    if (pick < 0) pick = nshapes - 1;
    const ClusterShape sh = kShapes[pick];
    const size_t dyn = std::max(smem, sh.spread_smem);
    cudaError_t e = cudaSuccess;
    if (sh.ctas > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess && dyn > 48 * 1024)
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nblk * sh.ctas));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sh.ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess && pick < nshapes - 1) {
      cudaGetLastError();
      g_shape = pick + 1;  // this shape is not usable here
      continue;
    }
    PD_CK(e);
    count_launch();
    g_last_ctas = sh.ctas;
    return 0;
  }
}

template <typename K, typename... Args>
static int launch_cluster(K kernel, int nblk, size_t smem, cudaStream_t st, Args... args) {
  return launch_cluster_t(false, kernel, nblk, smem, kSmallThreads, st, args...);
}

// ---------------------------------------------------------------------------
// Cholesky G = R^H R, upper, in place; one cluster per block
// ---------------------------------------------------------------------------
__device__ __forceinline__ double shfl_s(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double2 shfl_s(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <typename S>
__global__ void __launch_bounds__(1024) cholesky_kernel(const SmallDesc* desc, S* Gall, int* info, double* diag0,
                                                        double* minratio) {
  const int t = cl_slice();
  const SmallDesc d = desc[t];
  const int m = d.m;
  S* G = Gall + d.off;
  const int gid = cl_rank() * blockDim.x + threadIdx.x, gsz = cl_size() * blockDim.x;
  if (diag0) {
    for (int i = gid; i < m; i += gsz) diag0[d.voff + i] = sc<S>::re(G[i + (int64_t)i * m]);
    cl_sync();
  }
  // Blocked right-looking factorization in panels of CB columns, three cluster
  // barriers per panel: (1) CTA 0 factors the diagonal block in shared memory,
  // (2) every CTA solves R_JJ^H R_JK = G_JK for its columns right of the panel,
  // (3) the trailing upper triangle gets G_KK -= R_JK^H R_JK.
  constexpr int CB = 32;
  __shared__ S Rjj[CB][CB + 1];  // R_JJ (row, col)
  __shared__ int sh_bad;
  int bad = 0;
  for (int j0 = 0; j0 < m && !bad; j0 += CB) {
    const int nb = min(CB, m - j0);
    if (cl_rank() == 0) {
      for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        Rjj[r][c] = G[(j0 + r) + (int64_t)(j0 + c) * m];
      }
      if (threadIdx.x == 0) sh_bad = 0;
      __syncthreads();
      if (threadIdx.x < 32) {  // one warp factors the diagonal block; lane c owns column c
        const int lane = threadIdx.x;
        for (int j = 0; j < nb; ++j) {
          const double dj = sc<S>::re(Rjj[j][j]);
          if (!((dj > 0.0) && isfinite(dj))) {
            if (lane == 0) sh_bad = j0 + j + 1;
            break;
          }
          const double r = sqrt(dj);
          __syncwarp();
          if (lane > j && lane < nb) Rjj[j][lane] = sc<S>::scale(Rjj[j][lane], 1.0 / r);
          __syncwarp();
          if (lane > j && lane < nb)
            for (int i = j + 1; i <= lane; ++i)
              Rjj[i][lane] = sc<S>::sub(Rjj[i][lane], sc<S>::mul(sc<S>::conj(Rjj[j][i]), Rjj[j][lane]));
          __syncwarp();
          if (lane == j) Rjj[j][j] = sc<S>::from_re(r);
          __syncwarp();
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int r = e % nb, c = e / nb;
        if (r <= c) G[(j0 + r) + (int64_t)(j0 + c) * m] = Rjj[r][c];
      }
      if (threadIdx.x == 0) info[t] = sh_bad;  // provisional; rewritten below
    }
    cl_sync();
    bad = info[t];
    if (bad) break;
    // every CTA: R_JJ into shared memory, then one warp per column k of the row panel
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int r = e % nb, c = e / nb;
      Rjj[r][c] = r <= c ? G[(j0 + r) + (int64_t)(j0 + c) * m] : sc<S>::zero();
    }
    __syncthreads();
    const int k0 = j0 + nb;
    {
      const int lane = threadIdx.x & 31;
      const int gw = gid >> 5, nw = gsz >> 5;
      for (int k = k0 + gw; k < m; k += nw) {
        // forward substitution R_JJ^H x = g, column-oriented: once x_i is final
        // (lane i), the rows below subtract conj(R(i, row)) x_i
        S g = lane < nb ? G[(j0 + lane) + (int64_t)k * m] : sc<S>::zero();
        for (int i = 0; i < nb; ++i) {
          S xi = shfl_s(g, i);
          xi = sc<S>::scale(xi, 1.0 / sc<S>::re(Rjj[i][i]));
          if (lane == i) g = xi;
          if (lane > i && lane < nb) g = sc<S>::sub(g, sc<S>::mul(sc<S>::conj(Rjj[i][lane]), xi));
        }
        if (lane < nb) {
          G[(j0 + lane) + (int64_t)k * m] = g;
          // transposed copy into the (unused) strict lower triangle of the panel
          // columns: R(j0+l, k) at G(k, j0+l), read with unit stride below
          G[k + (int64_t)(j0 + lane) * m] = g;
        }
      }
    }
    cl_sync();
    // trailing update of the upper triangle: G(i,k) -= sum_l conj(R(l,i)) R(l,k), k0 <= i <= k
    const int tt = m - k0;
    for (int64_t e = gid; e < (int64_t)tt * tt; e += gsz) {
      const int i = k0 + (int)(e % tt), k = k0 + (int)(e / tt);
      if (i > k) continue;
      S v = G[i + (int64_t)k * m];
      for (int l = 0; l < nb; ++l) {
        const S* pl = G + (int64_t)(j0 + l) * m;
        v = sc<S>::sub(v, sc<S>::mul(sc<S>::conj(pl[i]), pl[k]));
      }
      G[i + (int64_t)k * m] = v;
    }
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
  return launch_cluster_t(true, cholesky_kernel<S>, nblk, 0, 1024, st, d_desc, G, info, diag0, minratio);
}

// ---------------------------------------------------------------------------
// upper triangular inverse X = R^{-1}, blocked in 32 x 32 tiles: invert the
// diagonal tiles (one thread per column), then for tile distance d = 1, 2, ...
// T_ij = sum_{k=i+1..j} R_ik X_kj (kept transposed in the still-unused lower
// tile (j,i), so every index stays inside the m x m block even when the last
// tile is partial) and X_ij = -X_ii T_ij; two cluster barriers per distance.
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(1024) triinv_kernel(const SmallDesc* desc, const S* Rall, S* Xall) {
  const int t = cl_slice();
  const SmallDesc dsc = desc[t];
  const int m = dsc.m;
  const S* R = Rall + dsc.off;
  S* X = Xall + dsc.off;
  const int gid = cl_rank() * blockDim.x + threadIdx.x, gsz = cl_size() * blockDim.x;
  const int nb = (m + 31) / 32;
  for (int64_t e = gid; e < (int64_t)m * m; e += gsz) X[e] = sc<S>::zero();
  cl_sync();
  for (int it = gid; it < nb * 32; it += gsz) {
    const int i = it / 32, c = it % 32;
    const int j = 32 * i + c;
    if (j >= m) continue;
    X[j + (int64_t)j * m] = sc<S>::from_re(1.0 / sc<S>::re(R[j + (int64_t)j * m]));
    for (int r = c - 1; r >= 0; --r) {
      const int row = 32 * i + r;
      S acc = sc<S>::zero();
      for (int k = r + 1; k <= c; ++k) sc<S>::fma_(acc, R[row + (int64_t)(32 * i + k) * m], X[32 * i + k + (int64_t)j * m]);
      X[row + (int64_t)j * m] = sc<S>::scale(acc, -1.0 / sc<S>::re(R[row + (int64_t)row * m]));
    }
  }
  cl_sync();
  for (int d = 1; d < nb; ++d) {
    const int nblkd = nb - d;
    for (int it = gid; it < nblkd * 1024; it += gsz) {
      const int i = it / 1024, r = (it % 1024) % 32, c = (it % 1024) / 32;
      const int j = i + d;
      const int row = 32 * i + r, col = 32 * j + c;
      if (row >= m || col >= m) continue;
      S acc = sc<S>::zero();
      const int qend = min(32 * (j + 1), m);
      for (int q = 32 * (i + 1); q < qend; ++q) sc<S>::fma_(acc, R[row + (int64_t)q * m], X[q + (int64_t)col * m]);
      X[(32 * j + c) + (int64_t)(32 * i + r) * m] = acc;  // T_ij(r,c), transposed into the lower tile (j,i)
    }
    cl_sync();
    for (int it = gid; it < nblkd * 1024; it += gsz) {
      const int i = it / 1024, r = (it % 1024) % 32, c = (it % 1024) / 32;
      const int j = i + d;
      const int row = 32 * i + r, col = 32 * j + c;
      if (row >= m || col >= m) continue;
      S acc = sc<S>::zero();
      const int send = min(32, m - 32 * i);
      for (int q = r; q < send; ++q)
        sc<S>::fma_(acc, X[row + (int64_t)(32 * i + q) * m], X[(32 * j + c) + (int64_t)(32 * i + q) * m]);
      X[row + (int64_t)col * m] = sc<S>::scale(acc, -1.0);
    }
    cl_sync();
  }
  for (int64_t e = gid; e < (int64_t)m * m; e += gsz) {
    const int row = (int)(e % m), col = (int)(e / m);
    if (row / 32 > col / 32) X[e] = sc<S>::zero();
  }
}

template <typename S>
int launch_triinv(int nblk, const SmallDesc* d_desc, const S* R, S* Rinv, cudaStream_t st) {
  if (nblk <= 0) return 0;
  return launch_cluster_t(true, triinv_kernel<S>, nblk, 0, 1024, st, d_desc, R, Rinv);
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

// Rotation of the pair (p, q) of one round.  Indices >= m (the dummy player of
// an odd m) are stored as -1; a pair without rotation keeps c = 1, s = 0, u = 1.
template <typename S>
__device__ __forceinline__ void make_rot(const S* A, int m, int p, int q, Rot<S>& r) {
  using R = typename real_t<S>::type;
  r.p = p < m ? p : -1;
  r.q = q < m ? q : -1;
  r.c = R(1);
  r.s = R(0);
  r.u = sc<S>::from_re(R(1));
  if (p >= m || q >= m) return;
  const S apq = A[p + (int64_t)q * m];
  // |A(p,q)| without squaring: in FP32 the square of an element below ~1e-19
  // is subnormal, and a modulus taken from it makes the rotation non-unitary
  const R g = sc<S>::absv(apq);
  const R tiny = sizeof(R) == 8 ? R(1e-290) : R(1e-30);
  if (!(g > tiny)) return;
  r.u = sc<S>::scale(apq, R(1) / g);
  const R app = sc<S>::re(A[p + (int64_t)p * m]), aqq = sc<S>::re(A[q + (int64_t)q * m]);
  const R th = (aqq - app) / (R(2) * g);
  const R t = (th >= R(0) ? R(1) : R(-1)) / (fabs(th) + sqrt(th * th + R(1)));
  r.c = R(1) / sqrt(t * t + R(1));
  r.s = t * r.c;
}

template <typename S>
__global__ void __launch_bounds__(512) jacobi_kernel(const SmallDesc* desc, S* Aall, S* Aalt, S* Vall, S* Vout,
                                                     double* lamall, double tol, int max_sweeps, int* sweeps_out,
                                                     double* scratch) {
  using R = typename real_t<S>::type;
  extern __shared__ __align__(16) char smem[];
  Rot<S>* rot = (Rot<S>*)smem;
  __shared__ double red[2][32];
  const int t = cl_slice();
  const SmallDesc d = desc[t];
  const int m = d.m;
  // A is updated out of place, alternating between the two buffers: a round
  // reads its pivots and blocks from one and writes the other, so no CTA can see
  // a half-updated round and one cluster barrier per round suffices
  S* A = Aall + d.off;
  S* Anext = Aalt + d.off;
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
      // every CTA derives the round's rotations from the same A
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
      __syncthreads();
      // A <- J^H A J in one pass: the 2 x 2 block of A in rows (p_i, q_i) and columns
      // (p_k, q_k) needs only the rotations of pairs i and k, so the blocks are
      // independent; V <- V J likewise per (row, pair).  One cluster barrier per round.
      const int64_t nb = (int64_t)np * np;
      for (int64_t e = gid; e < nb; e += gsz) {
        const int i = (int)(e % np), k = (int)(e / np);
        const Rot<S> ri = rot[i], rk = rot[k];
        const int ra[2] = {ri.p, ri.q}, cb[2] = {rk.p, rk.q};
        S x[2][2];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 2; ++b2)
            x[a][b2] = (ra[a] >= 0 && cb[b2] >= 0) ? A[ra[a] + (int64_t)cb[b2] * m] : sc<S>::zero();
        // columns: [x_p, x_q] <- [x_p u c - x_q s, x_p u s + x_q c] (pair k)
        const S uck = sc<S>::scale(rk.u, rk.c), usk = sc<S>::scale(rk.u, rk.s);
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const S xp = x[a][0], xq = x[a][1];
          x[a][0] = sc<S>::sub(sc<S>::mul(xp, uck), sc<S>::scale(xq, rk.s));
          x[a][1] = sc<S>::add(sc<S>::mul(xp, usk), sc<S>::scale(xq, rk.c));
        }
        // rows: [x_p; x_q] <- [conj(u c) x_p - s x_q; conj(u s) x_p + c x_q] (pair i)
        const S ucc = sc<S>::conj(sc<S>::scale(ri.u, ri.c)), usc = sc<S>::conj(sc<S>::scale(ri.u, ri.s));
#pragma unroll
        for (int b2 = 0; b2 < 2; ++b2) {
          const S xp = x[0][b2], xq = x[1][b2];
          x[0][b2] = sc<S>::sub(sc<S>::mul(ucc, xp), sc<S>::scale(xq, ri.s));
          x[1][b2] = sc<S>::add(sc<S>::mul(usc, xp), sc<S>::scale(xq, ri.c));
        }
        if (i == k && ri.p >= 0 && ri.q >= 0) {  // the rotated pivot block: exact zeros, real diagonal
          x[0][1] = sc<S>::zero();
          x[1][0] = sc<S>::zero();
          x[0][0] = sc<S>::from_re(sc<S>::re(x[0][0]));
          x[1][1] = sc<S>::from_re(sc<S>::re(x[1][1]));
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 2; ++b2)
            if (ra[a] >= 0 && cb[b2] >= 0) Anext[ra[a] + (int64_t)cb[b2] * m] = x[a][b2];
      }
      const int64_t nv = (int64_t)np * m;
      for (int64_t e = gid; e < nv; e += gsz) {
        const int k = (int)(e / m), row = (int)(e % m);
        const Rot<S> rk = rot[k];
        if (rk.p < 0 || rk.q < 0) continue;
        const S vp = V[row + (int64_t)rk.p * m], vq = V[row + (int64_t)rk.q * m];
        const S uc = sc<S>::scale(rk.u, rk.c), us = sc<S>::scale(rk.u, rk.s);
        V[row + (int64_t)rk.p * m] = sc<S>::sub(sc<S>::mul(vp, uc), sc<S>::scale(vq, rk.s));
        V[row + (int64_t)rk.q * m] = sc<S>::add(sc<S>::mul(vp, us), sc<S>::scale(vq, rk.c));
      }
      // (every row and column index is in exactly one pair, so the blocks cover all of A;
      // the partner of the dummy player of an odd m is rotated by the identity)
      cl_sync();
      S* tmp = A;
      A = Anext;
      Anext = tmp;
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
int launch_jacobi(int nblk, const SmallDesc* d_desc, int max_m, S* A, S* Aalt, S* Vwork, S* Vout, double* lam,
                  double tol, int max_sweeps, int* sweeps_out, double* scratch, cudaStream_t st) {
  if (nblk <= 0) return 0;
  const size_t smem = sizeof(Rot<S>) * (size_t)((max_m + 2) / 2);
  if (smem > 48 * 1024) PD_CK(cudaFuncSetAttribute(jacobi_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return launch_cluster_t(false, jacobi_kernel<S>, nblk, smem, 512, st, d_desc, A, Aalt, Vwork, Vout, lam, tol, max_sweeps,
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

// Band entries split once into float-float pairs, layout [j * (b+1) + d] for
// B(j+d, j) (the compact lower band, leading dimension b+1).
template <typename S>
__global__ void band_split_kernel(int64_t n, int b, const double* __restrict__ band, int64_t ldab,
                                  typename ffv<S>::type* __restrict__ out) {
  const int64_t total = n * (int64_t)(b + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / (b + 1);
    const int d = (int)(e % (b + 1));
    if constexpr (std::is_same<S, double2>::value) {
      const double* p = band + 2 * (d + j * ldab);
      const double im = d == 0 ? 0.0 : p[1];
      ff_load(make_double2(p[0], im), false, out[e]);
    } else {
      ff_load(band[d + j * ldab], false, out[e]);
    }
  }
}

// Y = B X in float-float arithmetic.  Block: 32 rows x 8 columns, one warp per
// column; the warp stages the column's x(i0-b .. i0+31+b) in shared memory as
// float-float pairs (each x entry is split once for its 2b+1 uses), the band
// comes pre-split and is shared by the 8 warps through L1.
template <typename S>
__global__ void __launch_bounds__(256) band_matmul_ff_kernel(int64_t n, int b,
                                                            const typename ffv<S>::type* __restrict__ bs,
                                                            int ncols, const S* __restrict__ X, S* __restrict__ Y) {
  using V = typename ffv<S>::type;
  using ACC = typename std::conditional<std::is_same<S, double2>::value, ffacc2, ffacc1>::type;
  extern __shared__ __align__(16) unsigned char ffsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int W = 32 + 2 * b;
  V* xs = (V*)ffsm + (size_t)warp * W;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int c = blockIdx.y * 8 + warp;
  if (c >= ncols) return;  // whole warp leaves; no block-wide barrier follows
  const S* x = X + (int64_t)c * n;
  for (int t = lane; t < W; t += 32) {
    const int64_t j = i0 - b + t;
    S v = sc<S>::zero();
    if (j >= 0 && j < n) v = x[j];
    ff_load(v, false, xs[t]);
  }
  __syncwarp();
  const int64_t i = i0 + lane;
  if (i >= n) return;
  ACC acc{};
  const int64_t j0 = i - b < 0 ? 0 : i - b, j1 = i + b > n - 1 ? n - 1 : i + b;
  for (int64_t j = j0; j <= j1; ++j) {
    V bij;
    if (j <= i) {
      bij = bs[(i - j) + j * (int64_t)(b + 1)];
    } else {
      bij = bs[(j - i) + i * (int64_t)(b + 1)];
      if constexpr (std::is_same<S, double2>::value) {
        bij.z = -bij.z;
        bij.w = -bij.w;
      }
    }
    ff_fma(acc, bij, xs[j - (i0 - b)]);
  }
  Y[i + (int64_t)c * n] = ff_val(acc);
}

template <typename S>
int launch_band_split(int64_t n, int b, const void* band, int64_t ldab, void* out, cudaStream_t st) {
  band_split_kernel<S><<<1024, 256, 0, st>>>(n, b, (const double*)band, ldab, (typename ffv<S>::type*)out);
  PD_CK_LAUNCH();
  return 0;
}

size_t band_split_bytes(int64_t n, int b, int cplx) {
  return (size_t)n * (size_t)(b + 1) * (cplx ? sizeof(float4) : sizeof(float2));
}

template <typename S>
int launch_band_matmul_ff(int64_t n, int b, const void* band_split, int ncols, const S* X, S* Y, cudaStream_t st) {
  if (n <= 0 || ncols <= 0) return 0;
  using V = typename ffv<S>::type;
  const size_t smem = (size_t)8 * (32 + 2 * b) * sizeof(V);
  if (smem > 48 * 1024)
    PD_CK(cudaFuncSetAttribute(band_matmul_ff_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(ncols, 8));
  band_matmul_ff_kernel<S><<<grid, 256, smem, st>>>(n, b, (const V*)band_split, ncols, X, Y);
  PD_CK_LAUNCH();
  return 0;
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

// A <- A - mu I with mu = mean of Re diag(A), per block; mu saved in shift[t]
template <typename S>
__global__ void shift_kernel(const SmallDesc* desc, S* Aall, double* shift) {
  const SmallDesc d = desc[blockIdx.x];
  S* A = Aall + d.off;
  __shared__ double red[32];
  __shared__ double mu;
  double sum = 0.0;
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) sum += sc<S>::re(A[i + (int64_t)i * d.m]);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    mu = d.m > 0 ? t / d.m : 0.0;
    shift[blockIdx.x] = mu;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
    S* a = A + i + (int64_t)i * d.m;
    *a = sc<S>::from_re(sc<S>::re(*a) - mu);
  }
}

__global__ void unshift_kernel(const SmallDesc* desc, double* lam, const double* shift) {
  const SmallDesc d = desc[blockIdx.x];
  for (int i = threadIdx.x; i < d.m; i += blockDim.x) lam[d.voff + i] += shift[blockIdx.x];
}

template <typename S>
__global__ void identity_kernel(S* V, int m) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) V[i + (int64_t)i * m] = sc<S>::from_re(1.0);
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
  w.A32b = a.take<L>(msq);
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
  w.dsub = a.take<SmallDesc>(2 * (size_t)nblk);
  w.delta = a.take<double>((size_t)nblk * kOaSplit);
  w.shift = a.take<double>(nblk);
  w.A64 = a.take<S>(msq);
  w.reach = a.take<double>(mtot);
  w.reach_sorted = a.take<double>(mtot);
  w.ccap = (int)(mtot / 2 + 1);
  w.citems = a.take<GemmItem<S>>(w.ccap);
  w.cdesc = a.take<SmallDesc>(w.ccap);
  w.csweeps = a.take<int>(w.ccap);
  w.cjscratch = a.take<double>((size_t)w.ccap * 2 * 16);
  return w;
}

template <typename S>
int small_gemm(bool conjA, const std::vector<SmallDesc>& blk, int max_m, S* const* abc, int herm, int triB,
               GemmItem<S>* d_items, cudaStream_t st, int ff) {
  // abc = {A base, B base, C base}; every block is m x m at the block's offset
  const int nb = (int)blk.size();
  if (!nb) return 0;
  std::vector<GemmItem<S>> it(nb);
  for (int t = 0; t < nb; ++t) {
    const int m = blk[t].m;
    const int64_t o = blk[t].off;
    it[t] = GemmItem<S>{abc[0] + o, abc[1] + o, abc[2] + o, m, m, m, m, m, m, 0};
  }
  PD_CK(cudaMemcpyAsync(d_items, it.data(), sizeof(GemmItem<S>) * nb, cudaMemcpyHostToDevice, st));
  S one, zero;
  if constexpr (std::is_same<S, double>::value) {
    one = 1.0;
    zero = 0.0;
  } else {
    one = make_double2(1.0, 0.0);
    zero = make_double2(0.0, 0.0);
  }
  return launch_gemm<S>(conjA, nb, d_items, max_m, max_m, max_m, one, zero, 1, nullptr, 0, st, herm, triB, ff);
}

// One refinement step of an approximate eigenvector matrix V of a Hermitian A
// (Ogita & Aishima, "Iterative refinement for symmetric eigenvalue
// decomposition", 2018); E overwrites S.  Their separation test uses one
// Frobenius-norm bound for all pairs; here each pair is tested on its own
// coupling, which keeps the step quadratic on the separated pairs while the
// others are left to the cluster treatment.
template <typename S>
__global__ void __launch_bounds__(256) oa_kernel(const SmallDesc* desc, S* Sall, const S* Pall, double* lamall,
                                                  double* est_out, double* reach_all) {
  // One refinement step (Ogita and Aishima, 2018) for block t, given S = V^H A V
  // and P = V^H V of the current approximate eigenvectors V:
  //   lambda_i = S_ii / P_ii, R = I - P, c_ij = S_ij + lambda_j R_ij,
  //   E_ij = c_ij / (lambda_j - lambda_i)   for a separated pair (|gap| > 4 max(|c_ij|, |c_ji|)),
  //   E_ij = R_ij / 2                       otherwise (and on the diagonal),
  // and V <- V (I + E) (done by the caller).  A separated pair gets |E_ij| < 1/4
  // and converges quadratically.  A pair that is not separated although it is
  // coupled (|c_ij| > 1e-14 max|lambda|) belongs to a cluster: its coupling is
  // left alone here and resolved by the caller.  Outputs: est = max(|E_ij| over
  // separated pairs, |R_ij|), the size of the correction, and per column j
  // reach_j = the largest lambda_i >= lambda_j (i != j) coupled to j without
  // being separated, or -inf.  Grid (blocks, kOaSplit): CTA y of a block handles
  // columns y*nw + warp (stride kOaSplit*nw); est_out[block * kOaSplit + y] is its
  // partial maximum.  Every CTA computes the (identical) lambda itself.
  const SmallDesc d = desc[blockIdx.x];
  const int m = d.m;
  S* Sm = Sall + d.off;
  const S* P = Pall + d.off;
  double* lam = lamall + d.voff;
  double* reach = reach_all + d.voff;
  __shared__ double red[2][32];
  __shared__ double sh_l;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double lmax = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double l = sc<S>::re(Sm[i + (int64_t)i * m]) / sc<S>::re(P[i + (int64_t)i * m]);
    lam[i] = l;
    lmax = fmax(lmax, fabs(l));
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_down_sync(0xffffffffu, lmax, o));
  if (lane == 0) red[0][warp] = lmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a = fmax(a, red[0][w]);
    sh_l = a;
  }
  __syncthreads();
  const double tiny = 1e-14 * sh_l;
  double emax = 0.0, rmax = 0.0;
  for (int j = blockIdx.y * nw + warp; j < m; j += gridDim.y * nw) {
    const double lj = lam[j];
    double rj = -INFINITY;
    for (int i = lane; i < m; i += 32) {
      const int64_t e = i + (int64_t)j * m;
      S r = sc<S>::scale(P[e], -1.0);
      if (i == j) r = sc<S>::add(r, sc<S>::from_re(1.0));
      rmax = fmax(rmax, sqrt(sc<S>::abs2(r)));
      S ev = sc<S>::scale(r, 0.5);
      if (i != j) {
        // c_ij and |c_ji| = |S_ij + lambda_i R_ij|: the pair is classified on the
        // larger of the two so that (i,j) and (j,i) always get the same treatment
        // (E + E^H then equals R, which keeps the orthogonality correction exact)
        const double li = lam[i];
        const S c = sc<S>::add(Sm[e], sc<S>::scale(r, lj));
        const double ca = fmax(sc<S>::absv(c), sc<S>::absv(sc<S>::add(Sm[e], sc<S>::scale(r, li))));
        const double gap = lj - li;
        if (ca > tiny) {
          if (fabs(gap) > 4.0 * ca) {
            ev = sc<S>::scale(c, 1.0 / gap);
            emax = fmax(emax, sqrt(sc<S>::abs2(ev)));
          } else if (li >= lj) {
            rj = fmax(rj, li);
          }
        }
      }
      Sm[e] = ev;
    }
    for (int o = 16; o > 0; o >>= 1) rj = fmax(rj, __shfl_down_sync(0xffffffffu, rj, o));
    if (lane == 0) reach[j] = rj;
  }
  for (int o = 16; o > 0; o >>= 1) {
    emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
    rmax = fmax(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
  }
  __syncthreads();
  if (lane == 0) {
    red[0][warp] = emax;
    red[1][warp] = rmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) {
      a = fmax(a, red[0][w]);
      b = fmax(b, red[1][w]);
    }
    est_out[blockIdx.x * gridDim.y + blockIdx.y] = fmax(a, b);
  }
}

// W[:, rank(i)] = V[:, i] * phase, eigenvalues sorted ascending (rank sort, ties by index).
template <typename S>
__global__ void __launch_bounds__(1024) sort_phase_kernel(const SmallDesc* desc, const S* Vall, const double* lam_in,
                                                          double* lam_out, S* Wall, const double* aux_in = nullptr,
                                                          double* aux_out = nullptr) {
  const SmallDesc d = desc[blockIdx.x];
  const int m = d.m;
  const S* V = Vall + d.off;
  S* Wm = Wall + d.off;
  const double* li = lam_in + d.voff;
  double* lo = lam_out + d.voff;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < m; i += nw) {
    int rank = 0;
    for (int j = lane; j < m; j += 32) rank += (li[j] < li[i]) || (li[j] == li[i] && j < i);
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_down_sync(0xffffffffu, rank, o);
    rank = __shfl_sync(0xffffffffu, rank, 0);
    const S* v = V + (int64_t)i * m;
    double best = -1.0;
    int kb = m;
    for (int k = lane; k < m; k += 32) {
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
    S ph = sc<S>::from_re(1.0);
    if (nb > 0.0) ph = sc<S>::scale(sc<S>::conj(v[kb]), 1.0 / nb);
    S* w = Wm + (int64_t)rank * m;
    for (int k = lane; k < m; k += 32) w[k] = (k == kb) ? sc<S>::from_re(nb) : sc<S>::mul(v[k], ph);
    if (lane == 0) {
      lo[rank] = li[i];
      if (aux_in) aux_out[d.voff + rank] = aux_in[d.voff + i];
    }
  }
}

// Rayleigh-Ritz on clusters of eigenvector columns.  Cluster q covers the c
// columns i0..i0+c-1 of an m x m block at element offset `off` (eigenvalues at
// voff): H = Vc^H A Vc (c x c, FP64), FP64 Jacobi H = Wc diag(mu) Wc^H,
// Vc <- Vc Wc, lambda(i0..) <- mu (ascending).  All clusters are batched.
template <typename S>
static int resolve_clusters(const std::vector<ClusterRef>& cl, const S* A, double* lam, S* W,
                            const EighScratch<S>& w, cudaStream_t st) {
  const int nq = (int)cl.size();
  if (nq > w.ccap) return PDESHEP_WORKSPACE_TOO_SMALL;
  S one, zero;
  if constexpr (std::is_same<S, double>::value) {
    one = 1.0;
    zero = 0.0;
  } else {
    one = make_double2(1.0, 0.0);
    zero = make_double2(0.0, 0.0);
  }
  int mx_m = 0, mx_c = 0;
  for (const ClusterRef& q : cl) {
    mx_m = std::max(mx_m, q.m);
    mx_c = std::max(mx_c, q.c);
  }
  std::vector<GemmItem<S>> it(nq);
  auto col = [&](const ClusterRef& q) { return q.off + (int64_t)q.i0 * q.m; };
  // T = A Vc  (m x c at the cluster's columns of T)
  for (int q = 0; q < nq; ++q) {
    const ClusterRef& c = cl[q];
    it[q] = GemmItem<S>{A + c.off, W + col(c), w.T + col(c), c.m, c.c, c.m, c.m, c.m, c.m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.citems, it.data(), sizeof(GemmItem<S>) * nq, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(false, nq, w.citems, mx_m, mx_c, mx_m, one, zero, 1, nullptr, 0, st, 0, 0));
  // H = Vc^H T  (c x c, leading dimension c, in A64 at the cluster's offset)
  for (int q = 0; q < nq; ++q) {
    const ClusterRef& c = cl[q];
    it[q] = GemmItem<S>{W + col(c), w.T + col(c), w.A64 + col(c), c.c, c.c, c.m, c.m, c.m, c.c, 0};
  }
  PD_CK(cudaMemcpyAsync(w.citems, it.data(), sizeof(GemmItem<S>) * nq, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(true, nq, w.citems, mx_c, mx_c, mx_m, one, zero, 1, nullptr, 0, st, 1, 0));
  std::vector<SmallDesc> cd(nq);
  for (int q = 0; q < nq; ++q) cd[q] = SmallDesc{col(cl[q]), cl[q].voff + cl[q].i0, cl[q].c, 0};
  PD_CK(cudaMemcpyAsync(w.cdesc, cd.data(), sizeof(SmallDesc) * nq, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_jacobi<S>(nq, w.cdesc, mx_c, w.A64, w.T, w.Vw, w.W64, w.lam32, 1e-14, 60, w.csweeps, w.cjscratch,
                          st));
  // Vc Wc -> Vd, then back into W; eigenvalues back into lam
  for (int q = 0; q < nq; ++q) {
    const ClusterRef& c = cl[q];
    it[q] = GemmItem<S>{W + col(c), w.W64 + col(c), w.Vd + col(c), c.m, c.c, c.c, c.m, c.c, c.m, 0};
  }
  PD_CK(cudaMemcpyAsync(w.citems, it.data(), sizeof(GemmItem<S>) * nq, cudaMemcpyHostToDevice, st));
  PD_TRY(launch_gemm<S>(false, nq, w.citems, mx_m, mx_c, mx_c, one, zero, 1, nullptr, 0, st, 0, 0));
  for (const ClusterRef& c : cl) {
    PD_CK(cudaMemcpyAsync(W + col(c), w.Vd + col(c), sizeof(S) * (size_t)c.m * c.c, cudaMemcpyDeviceToDevice, st));
    PD_CK(cudaMemcpyAsync(lam + c.voff + c.i0, w.lam32 + c.voff + c.i0, sizeof(double) * c.c,
                          cudaMemcpyDeviceToDevice, st));
  }
  std::vector<int> sw(nq);
  PD_CK(cudaMemcpyAsync(sw.data(), w.csweeps, sizeof(int) * nq, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  for (int v : sw)
    if (v < 0) return PDESHEP_EIG_NOT_CONVERGED;
  return 0;
}

template <typename S>
int eigh_mixed(int nblk, const SmallDesc* d_desc, const SmallDesc* h_desc, int max_m, S* A, double* lam, S* W,
               const EighScratch<S>& w, cudaStream_t st, int* fp64_sweeps_out, const unsigned char* h_fp32,
               int* fp32_sweeps_out, EighReport* rep) {
  using L = typename lowp<S>::type;
  if (nblk <= 0) return 0;
  std::vector<SmallDesc> all(h_desc, h_desc + nblk), sub, rest;
  for (int t = 0; t < nblk; ++t) (h_fp32 == nullptr || h_fp32[t] ? sub : rest).push_back(h_desc[t]);
  const int ns = (int)sub.size();
  S one, zero;
  if constexpr (std::is_same<S, double>::value) {
    one = 1.0;
    zero = 0.0;
  } else {
    one = make_double2(1.0, 0.0);
    zero = make_double2(0.0, 0.0);
  }
  const dim3 gcast((unsigned)std::min<int64_t>(ceil_div((int64_t)max_m * max_m, 256), 512), (unsigned)nblk);
  // Shift every block by the mean of its diagonal: the projected matrices of a slice
  // have eigenvalues clustered around an offset much larger than their spread, and
  // the FP32 stage, the refinement's cluster threshold and the Jacobi stopping test
  // must resolve the spread, not the offset.  The shift is added back at the end.
  shift_kernel<S><<<nblk, 256, 0, st>>>(d_desc, A, w.shift);
  PD_CK_LAUNCH();
  if (ns) {
    // FP32 Jacobi on the blocks far from diagonal gives the starting eigenvectors
    PD_CK(cudaMemcpyAsync(w.dsub, sub.data(), sizeof(SmallDesc) * ns, cudaMemcpyHostToDevice, st));
    const dim3 g((unsigned)gcast.x, (unsigned)ns);
    small_cast_kernel<S, L><<<g, 256, 0, st>>>(w.dsub, A, w.A32);
    PD_CK_LAUNCH();
    PD_TRY(launch_jacobi<L>(ns, w.dsub, max_m, w.A32, w.A32b, w.V32w, w.V32, w.lam32, 1e-6, 30, w.sweeps,
                            w.jscratch, st));
    if (fp32_sweeps_out)
      PD_CK(cudaMemcpyAsync(fp32_sweeps_out, w.sweeps, sizeof(int) * ns, cudaMemcpyDeviceToDevice, st));
    small_cast_kernel<L, S><<<g, 256, 0, st>>>(w.dsub, w.V32, w.Vd);
    PD_CK_LAUNCH();
  }
  for (auto& b : rest) {  // nearly diagonal blocks start from the identity
    PD_CK(cudaMemsetAsync(w.Vd + b.off, 0, sizeof(S) * (size_t)b.m * b.m, st));
    identity_kernel<S><<<1, 256, 0, st>>>(w.Vd + b.off, b.m);
    PD_CK_LAUNCH();
  }
  // FP64 refinement of V (kept in Vd): each step roughly squares the error of the
  // separated pairs.  A block leaves the batch after the step whose correction was
  // below kRefineTol (what remains is of the order of its square); at most
  // kRefineSteps steps.
  S* V = w.Vd;
  S* Vn = w.Vw;
  std::vector<double> drel(nblk, 1.0), est(nblk), estp((size_t)nblk * kOaSplit);
  std::vector<int> act(nblk);
  for (int t = 0; t < nblk; ++t) act[t] = t;
  for (int it = 0; it < kRefineSteps && !act.empty(); ++it) {
    const int na = (int)act.size();
    std::vector<SmallDesc> sub_d(na);
    for (int q = 0; q < na; ++q) sub_d[q] = all[act[q]];
    const SmallDesc* dd = d_desc;
    if (na != nblk) {
      PD_CK(cudaMemcpyAsync(w.dsub, sub_d.data(), sizeof(SmallDesc) * na, cudaMemcpyHostToDevice, st));
      dd = w.dsub;
    }
    {
      S* abc[3] = {A, V, w.T};  // T = A V
      PD_TRY(small_gemm<S>(false, sub_d, max_m, abc, 0, 0, w.items, st, w.ff));
    }
    {
      S* abc[3] = {V, w.T, w.W64};  // S = V^H A V  (in W64)
      PD_TRY(small_gemm<S>(true, sub_d, max_m, abc, 1, 0, w.items, st, w.ff));
    }
    {
      S* abc[3] = {V, V, w.T};  // P = V^H V  (in T)
      PD_TRY(small_gemm<S>(true, sub_d, max_m, abc, 1, 0, w.items, st, w.ff));
    }
    oa_kernel<S><<<dim3(na, kOaSplit), 256, 0, st>>>(dd, w.W64, w.T, w.lam32, w.delta, w.reach);
    PD_CK_LAUNCH();
    for (auto& b : sub_d)
      PD_CK(cudaMemcpyAsync(Vn + b.off, V + b.off, sizeof(S) * (size_t)b.m * b.m, cudaMemcpyDeviceToDevice, st));
    {
      // Vn = V + V E, then back into V
      std::vector<GemmItem<S>> it2(na);
      for (int q = 0; q < na; ++q) {
        const int m = sub_d[q].m;
        const int64_t o = sub_d[q].off;
        it2[q] = GemmItem<S>{V + o, w.W64 + o, Vn + o, m, m, m, m, m, m, 0};
      }
      PD_CK(cudaMemcpyAsync(w.items, it2.data(), sizeof(GemmItem<S>) * na, cudaMemcpyHostToDevice, st));
      PD_TRY(launch_gemm<S>(false, na, w.items, max_m, max_m, max_m, one, one, 1, nullptr, 0, st, 0, 0, w.ff));
    }
    for (auto& b : sub_d)
      PD_CK(cudaMemcpyAsync(V + b.off, Vn + b.off, sizeof(S) * (size_t)b.m * b.m, cudaMemcpyDeviceToDevice, st));
    PD_CK(cudaMemcpyAsync(estp.data(), w.delta, sizeof(double) * na * kOaSplit, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    for (int q = 0; q < na; ++q) {
      est[q] = 0.0;
      for (int c = 0; c < kOaSplit; ++c) est[q] = std::max(est[q], estp[(size_t)q * kOaSplit + c]);
    }
    if (rep) rep->refine_steps += 1;
    std::vector<int> next;
    for (int q = 0; q < na; ++q) {
      drel[act[q]] = est[q];
      if (!(est[q] < kRefineTol)) next.push_back(act[q]);
    }
    act.swap(next);
  }
  sort_phase_kernel<S><<<nblk, 1024, 0, st>>>(d_desc, V, w.lam32, lam, W, w.reach, w.reach_sorted);
  PD_CK_LAUNCH();
  // Clusters: runs of sorted eigenvalues tied together by pairs that the
  // refinement could not separate (a run extends while the next eigenvalue is
  // within the reach of the run).  Their mutual couplings were left alone; a
  // Rayleigh-Ritz step on each run's own columns resolves them (the cluster
  // treatment of Ogita and Aishima's refinement for clustered eigenvalues):
  // H = Vc^H A Vc, H = Wc diag(mu) Wc^H by FP64 Jacobi, Vc <- Vc Wc, lambda <- mu.
  // Blocks whose refinement did not converge, or with a run wider than
  // kMaxCluster columns, are redone by the robust path below.
  int64_t lam_len = 0;
  for (auto& b : all) lam_len = std::max<int64_t>(lam_len, b.voff + b.m);
  std::vector<double> lam_h(lam_len), reach_h(lam_len);
  PD_CK(cudaMemcpyAsync(lam_h.data(), lam, sizeof(double) * lam_len, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaMemcpyAsync(reach_h.data(), w.reach_sorted, sizeof(double) * lam_len, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  struct Cl {
    int t, i0, c;
  };
  std::vector<Cl> cl;
  std::vector<SmallDesc> fb, fb32;
  std::vector<int> fbidx;
  for (int t = 0; t < nblk; ++t) {
    const SmallDesc& b = all[t];
    bool bad = !(drel[t] < kRefineTol);
    if (bad && rep) rep->fallback_unconverged += 1;
    std::vector<Cl> mine;
    for (int i = 0; i < b.m && !bad;) {
      int j = i + 1;
      double r = reach_h[b.voff + i];
      while (j < b.m && lam_h[b.voff + j] <= r) {
        r = std::max(r, reach_h[b.voff + j]);
        ++j;
      }
      if (j - i > kMaxCluster) {
        bad = true;
        if (rep) rep->fallback_wide += 1;
      } else if (j - i > 1) {
        mine.push_back({t, i, j - i});
      }
      i = j;
    }
    if (!bad && rep)
      for (const Cl& q : mine) {
        rep->clusters += 1;
        rep->max_cluster = std::max(rep->max_cluster, q.c);
      }
    if (bad) {
      fb.push_back(b);
      fbidx.push_back(t);
    } else {
      cl.insert(cl.end(), mine.begin(), mine.end());
    }
  }
  if (!cl.empty()) {
    std::vector<ClusterRef> refs;
    for (const Cl& q : cl) refs.push_back({all[q.t].off, all[q.t].voff, all[q.t].m, q.i0, q.c});
    PD_TRY(resolve_clusters<S>(refs, A, lam, W, w, st));
  }
  const int nfb = (int)fb.size();
  if (nfb) {
    PD_CK(cudaMemcpyAsync(w.dsub, fb.data(), sizeof(SmallDesc) * nfb, cudaMemcpyHostToDevice, st));
    for (int q = 0; q < nfb; ++q) {
      const SmallDesc b = fb[q];
      const bool had32 = h_fp32 == nullptr || h_fp32[fbidx[q]];
      if (had32) {
        fb32.push_back(b);
      } else {
        PD_CK(cudaMemsetAsync(w.Vd + b.off, 0, sizeof(S) * (size_t)b.m * b.m, st));
        identity_kernel<S><<<1, 256, 0, st>>>(w.Vd + b.off, b.m);
        PD_CK_LAUNCH();
      }
    }
    if (!fb32.empty()) {
      const int n32 = (int)fb32.size();
      SmallDesc* d32 = w.dsub + nfb;  // second half of the descriptor scratch
      PD_CK(cudaMemcpyAsync(d32, fb32.data(), sizeof(SmallDesc) * n32, cudaMemcpyHostToDevice, st));
      small_cast_kernel<L, S><<<dim3((unsigned)gcast.x, (unsigned)n32), 256, 0, st>>>(d32, w.V32, w.Vd);
      PD_CK_LAUNCH();
      {
        S* abc[3] = {w.Vd, w.Vd, w.T};
        PD_TRY(small_gemm<S>(true, fb32, max_m, abc, 1, 0, w.items, st));
      }
      PD_TRY(launch_cholesky<S>(n32, d32, w.T, w.sweeps, st));
      PD_TRY(launch_triinv<S>(n32, d32, w.T, w.Vw, st));
      {
        S* abc[3] = {w.Vd, w.Vw, w.W64};
        PD_TRY(small_gemm<S>(false, fb32, max_m, abc, 0, 1, w.items, st));
      }
      for (auto& b : fb32)
        PD_CK(cudaMemcpyAsync(w.Vd + b.off, w.W64 + b.off, sizeof(S) * (size_t)b.m * b.m, cudaMemcpyDeviceToDevice, st));
    }
    {
      S* abc[3] = {A, w.Vd, w.T};  // T = A V
      PD_TRY(small_gemm<S>(false, fb, max_m, abc, 0, 0, w.items, st));
    }
    {
      S* abc[3] = {w.Vd, w.T, w.A64};  // H = V^H A V
      PD_TRY(small_gemm<S>(true, fb, max_m, abc, 1, 0, w.items, st));
    }
    PD_TRY(launch_jacobi<S>(nfb, w.dsub, max_m, w.A64, w.T, w.Vw, w.W64, lam, 1e-13, 60, w.sweeps, w.jscratch, st));
    {
      S* abc[3] = {w.Vd, w.W64, W};
      PD_TRY(small_gemm<S>(false, fb, max_m, abc, 0, 0, w.items, st));
    }
    phase_kernel<S><<<dim3((unsigned)ceil_div(max_m, 8), nfb), 256, 0, st>>>(w.dsub, W);
    PD_CK_LAUNCH();
  }
  unshift_kernel<<<nblk, 256, 0, st>>>(d_desc, lam, w.shift);
  PD_CK_LAUNCH();
  if (fp64_sweeps_out) {
    // report the fallback Jacobi's sweeps (0 for blocks that did not need it)
    std::vector<int> sw(nblk, 0);
    if (nfb) {
      std::vector<int> swf(nfb);
      PD_CK(cudaMemcpyAsync(swf.data(), w.sweeps, sizeof(int) * nfb, cudaMemcpyDeviceToHost, st));
      PD_CK(cudaStreamSynchronize(st));
      for (int q = 0; q < nfb; ++q) sw[fbidx[q]] = swf[q];
    }
    PD_CK(cudaMemcpyAsync(fp64_sweeps_out, sw.data(), sizeof(int) * nblk, cudaMemcpyHostToDevice, st));
  }
  return 0;
}

// explicit instantiations
template int small_gemm<double>(bool, const std::vector<SmallDesc>&, int, double* const*, int, int,
                                GemmItem<double>*, cudaStream_t, int);
template int small_gemm<double2>(bool, const std::vector<SmallDesc>&, int, double2* const*, int, int,
                                 GemmItem<double2>*, cudaStream_t, int);
template EighScratch<double> plan_eigh_scratch<double>(Arena&, int64_t, int64_t, int);
template EighScratch<double2> plan_eigh_scratch<double2>(Arena&, int64_t, int64_t, int);
template int eigh_mixed<double>(int, const SmallDesc*, const SmallDesc*, int, double*, double*, double*,
                                const EighScratch<double>&, cudaStream_t, int*, const unsigned char*, int*,
                                EighReport*);
template int eigh_mixed<double2>(int, const SmallDesc*, const SmallDesc*, int, double2*, double*, double2*,
                                 const EighScratch<double2>&, cudaStream_t, int*, const unsigned char*, int*,
                                 EighReport*);
template int launch_gemm<double>(bool, int, const GemmItem<double>*, int, int, int, double, double, int,
                                 double*, int64_t, cudaStream_t, int, int, int);
template int launch_gemm<double2>(bool, int, const GemmItem<double2>*, int, int, int, double2, double2, int,
                                  double2*, int64_t, cudaStream_t, int, int, int);
template int launch_cholesky<double>(int, const SmallDesc*, double*, int*, cudaStream_t, double*, double*);
template int launch_cholesky<double2>(int, const SmallDesc*, double2*, int*, cudaStream_t, double*, double*);
template int launch_triinv<double>(int, const SmallDesc*, const double*, double*, cudaStream_t);
template int launch_triinv<double2>(int, const SmallDesc*, const double2*, double2*, cudaStream_t);
template int launch_jacobi<double>(int, const SmallDesc*, int, double*, double*, double*, double*, double*,
                                   double, int, int*, double*, cudaStream_t);
template int launch_jacobi<double2>(int, const SmallDesc*, int, double2*, double2*, double2*, double2*, double*,
                                    double, int, int*, double*, cudaStream_t);
template int launch_jacobi<float>(int, const SmallDesc*, int, float*, float*, float*, float*, double*, double, int,
                                  int*, double*, cudaStream_t);
template int launch_jacobi<float2>(int, const SmallDesc*, int, float2*, float2*, float2*, float2*, double*, double,
                                   int, int*, double*, cudaStream_t);
template int launch_band_split<double>(int64_t, int, const void*, int64_t, void*, cudaStream_t);
template int launch_band_split<double2>(int64_t, int, const void*, int64_t, void*, cudaStream_t);
template int launch_band_matmul_ff<double>(int64_t, int, const void*, int, const double*, double*, cudaStream_t);
template int launch_band_matmul_ff<double2>(int64_t, int, const void*, int, const double2*, double2*,
                                            cudaStream_t);
template int launch_band_matmul<double>(int64_t, int, const void*, int64_t, int, const double*, double*,
                                        cudaStream_t);
template int launch_band_matmul<double2>(int64_t, int, const void*, int64_t, int, const double2*,
                                         double2*, cudaStream_t);

}  // namespace pdeshep
