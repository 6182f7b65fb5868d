// slicer.cu -- learned slice proposal.  Cheap statistics of the band feed a
// small FP32 network that predicts where the equal-count slice boundaries lie;
// exact LDL^T inertia counts then validate every proposed boundary and a
// multisection on inertia re-places the ones that miss their target count.
//
// The paper partitions the spectrum by inertia counts (Section 3.2) and names
// density-of-states estimates as the tool when no earlier spectrum is known
// (Section 3.1); equal eigenvalue counts per slice is one of its partition
// objectives (Section 3.1).  The network only proposes: every count returned
// comes from the inertia kernel.
//
// Features (98 per band):
//   [0, 64)   histogram of diag(B) over the Gershgorin interval [lo, hi]
//             (64 equal bins, fractions of n; bin k = floor((d - lo)/w), w =
//             (hi - lo)/64, clamped to [0, 63], evaluated in FP64)
//   64, 65    Gershgorin centre c = (lo+hi)/2 and radius r = (hi-lo)/2, both
//             divided by s = max(|lo|, |hi|) (scale-free)
//   [66, 98)  Chebyshev moments mu_k = z^H T_k(Bs) z / (n P), k = 0..31, of
//             Bs = (B - c I)/r, averaged over P = 8 Rademacher probes z
//             (kernel polynomial method; mu_0 = 1), accumulated in FP64
// Probe entry i of probe p: +1 if bit 0 of splitmix64(seed + p n + i) is 0,
// else -1, where splitmix64 is Vigna's generator (golden-ratio increment
// 0x9e3779b97f4a7c15, then xor-shift-multiply by 0xbf58476d1ce4e5b9 and
// 0x94d049bb133111eb with shifts 30, 27, 31).
//
// Network: 98 -> 256 -> 256 -> 256 -> 64, ReLU after the hidden layers,
// softmax over 64 slice-mass fractions, cumulative sums = 63 boundaries in
// normalised [0, 1] coordinates of the Gershgorin interval, i.e. the inverse
// of the normalised eigenvalue counting function at the fractions j/64.
// Loss: mean over the batch and the 63 boundaries of the squared error.
// Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
// Parameter vector: for each layer, W (out x in, row-major) then bias (out).
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dense.cuh"

namespace pdeshep {

// from inertia.cu
int gershgorin_device(int64_t n, int b, int cplx, const void* band, int64_t ldab, double* d_lo, double* d_hi,
                      cudaStream_t st);
size_t gershgorin_ws_doubles();
size_t inertia_ws_bytes(int b, int cplx, int nsigma);
int inertia_counts(int64_t n, int b, int cplx, const void* band, int64_t ldab, int nsigma, const double* h_sigma,
                   int64_t* h_neg, double* d_piv, void* work, size_t wbytes, cudaStream_t st, bool* nonfinite_out);

constexpr int kFeat = 98, kHid = 256, kOut = 64, kBins = 64, kMoments = 32, kProbes = 8;
constexpr int kNParams =
    kHid * kFeat + kHid + kHid * kHid + kHid + kHid * kHid + kHid + kOut * kHid + kOut;
constexpr int kChebBlocks = 64;
constexpr int kMaxSlices = 1024;


// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
__global__ void lohi_kernel(const double* glo, const double* ghi, double* lohi) {
  if (threadIdx.x == 0) {
    lohi[0] = glo[0];
    lohi[1] = ghi[0];
  }
}

__global__ void diag_hist_kernel(int64_t n, int cplx, const double* __restrict__ band, int64_t ldab,
                                 const double* __restrict__ lohi, unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[kBins];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const double lo = lohi[0], hi = lohi[1];
  const double w = (hi - lo) / kBins;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = cplx ? band[2 * (i * ldab)] : band[i * ldab];
    int k = 0;
    if (w > 0.0) {
      const double t = floor((d - lo) / w);
      k = t < 0.0 ? 0 : (t > (double)(kBins - 1) ? kBins - 1 : (int)t);
    }
    atomicAdd(&h[k], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void feat_head_kernel(int64_t n, const unsigned int* __restrict__ hist, const double* __restrict__ lohi,
                                 float* __restrict__ feat) {
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) feat[i] = (float)((double)hist[i] / (double)n);
  if (threadIdx.x == 0) {
    const double lo = lohi[0], hi = lohi[1];
    double s = fmax(fabs(lo), fabs(hi));
    if (!(s > 0.0)) s = 1.0;
    feat[64] = (float)(0.5 * (lo + hi) / s);
    feat[65] = (float)(0.5 * (hi - lo) / s);
    feat[66] = 1.0f;
  }
}

// probes Z (n x P column-major, real values in the band's scalar type); T0 = Z
template <typename S>
__global__ void probe_kernel(int64_t n, uint64_t seed, S* __restrict__ Z, S* __restrict__ T0) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * kProbes;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r = splitmix64(seed + (uint64_t)e);
    const double v = (r & 1ull) ? -1.0 : 1.0;
    Z[e] = sc<S>::from_re(v);
    T0[e] = sc<S>::from_re(v);
  }
}

// Tn = (Y - c T1)/r (first step) or 2 (Y - c T1)/r - T0 with Y = B T1; block
// partial sums of Re(conj(z) Tn) per probe into part[p * gridDim.x + block].
template <typename S>
__global__ void cheb_step_kernel(int64_t n, const double* __restrict__ lohi, int first, const S* __restrict__ Y,
                                 const S* __restrict__ T1, const S* __restrict__ T0, S* __restrict__ Tn,
                                 const S* __restrict__ Z, double* __restrict__ part) {
  const double c = 0.5 * (lohi[0] + lohi[1]);
  double r = 0.5 * (lohi[1] - lohi[0]);
  if (!(r > 0.0)) r = 1.0;
  const int p = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)p * n + i;
    S v = sc<S>::sub(Y[e], sc<S>::scale(T1[e], c));
    if (first)
      v = sc<S>::scale(v, 1.0 / r);
    else
      v = sc<S>::sub(sc<S>::scale(v, 2.0 / r), T0[e]);
    Tn[e] = v;
    acc += sc<S>::re(sc<S>::mul(sc<S>::conj(Z[e]), v));
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(int64_t)p * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void moment_kernel(int64_t n, int nparts, const double* __restrict__ part, int k, float* feat) {
  __shared__ double red[32];
  double t = 0.0;
  for (int q = threadIdx.x; q < kProbes * nparts; q += blockDim.x) t += part[q];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    feat[66 + k] = (float)(s / ((double)n * kProbes));
  }
}

struct FeatWs {
  double *glo, *ghi, *lohi, *part;
  unsigned int* hist;
  void *Z, *T0, *T1, *T2, *Y;
};

static FeatWs plan_feat(Arena& a, int64_t n, size_t es) {
  FeatWs w;
  w.glo = a.take<double>(gershgorin_ws_doubles() / 2);
  w.ghi = a.take<double>(gershgorin_ws_doubles() / 2);
  w.lohi = a.take<double>(2);
  w.part = a.take<double>(kProbes * kChebBlocks);
  w.hist = a.take<unsigned int>(kBins);
  w.Z = a.take<char>(n * kProbes * es);
  w.T0 = a.take<char>(n * kProbes * es);
  w.T1 = a.take<char>(n * kProbes * es);
  w.T2 = a.take<char>(n * kProbes * es);
  w.Y = a.take<char>(n * kProbes * es);
  return w;
}

template <typename S>
static int features(int64_t n, int b, int cplx, const void* band, int64_t ldab, uint64_t seed, float* d_feat,
                    const FeatWs& w, cudaStream_t st) {
  PD_TRY(gershgorin_device(n, b, cplx, band, ldab, w.glo, w.ghi, st));
  lohi_kernel<<<1, 32, 0, st>>>(w.glo, w.ghi, w.lohi);
  PD_CK_LAUNCH();
  PD_CK(cudaMemsetAsync(w.hist, 0, sizeof(unsigned int) * kBins, st));
  diag_hist_kernel<<<64, 256, 0, st>>>(n, cplx, (const double*)band, ldab, w.lohi, w.hist);
  PD_CK_LAUNCH();
  feat_head_kernel<<<1, 64, 0, st>>>(n, w.hist, w.lohi, d_feat);
  PD_CK_LAUNCH();
  S* Z = (S*)w.Z;
  S* T[3] = {(S*)w.T0, (S*)w.T1, (S*)w.T2};
  S* Y = (S*)w.Y;
  probe_kernel<S><<<152, 256, 0, st>>>(n, seed, Z, T[0]);
  PD_CK_LAUNCH();
  // three-term recurrence T_{k} = 2 Bs T_{k-1} - T_{k-2}, vectors rotating through T[k % 3]
  for (int k = 1; k < kMoments; ++k) {
    S* tprev = T[(k - 1) % 3];
    S* tprev2 = T[(k + 1) % 3];
    S* tk = T[k % 3];
    PD_TRY(launch_band_matmul<S>(n, b, band, ldab, kProbes, tprev, Y, st));
    cheb_step_kernel<S><<<dim3(kChebBlocks, kProbes), 256, 0, st>>>(n, w.lohi, k == 1, Y, tprev, tprev2, tk, Z,
                                                                     w.part);
    PD_CK_LAUNCH();
    moment_kernel<<<1, 256, 0, st>>>(n, kChebBlocks, w.part, k, d_feat);
    PD_CK_LAUNCH();
  }
  return 0;
}

// ---------------------------------------------------------------------------
// network (FP32)
// ---------------------------------------------------------------------------
struct Layer {
  int in, out;
  int64_t w, b;  // offsets of W and bias in the parameter vector
};

static void layer_table(Layer L[4]) {
  const int dims[5] = {kFeat, kHid, kHid, kHid, kOut};
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    L[l].in = dims[l];
    L[l].out = dims[l + 1];
    L[l].w = off;
    off += (int64_t)dims[l] * dims[l + 1];
    L[l].b = off;
    off += dims[l + 1];
  }
}

// Y[bt][o] = act(sum_i X[bt][i] W[o][i] + bias[o]); one CTA per 32 x 32 output tile
__global__ void __launch_bounds__(256) mlp_fwd_kernel(int B, int in, int out, const float* __restrict__ X,
                                                      const float* __restrict__ W, const float* __restrict__ bias,
                                                      float* __restrict__ Y, int relu) {
  __shared__ float Xs[32][33], Ws[32][33];
  const int o0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < in; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      Xs[r][c] = (b0 + r < B && k0 + c < in) ? X[(int64_t)(b0 + r) * in + k0 + c] : 0.f;
      Ws[r][c] = (o0 + r < out && k0 + c < in) ? W[(int64_t)(o0 + r) * in + k0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float wv = Ws[tx][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(Xs[ty + 8 * q][k], wv, acc[q]);
    }
    __syncthreads();
  }
  const int o = o0 + tx;
  if (o >= out) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int bt = b0 + ty + 8 * q;
    if (bt >= B) continue;
    float v = acc[q] + bias[o];
    if (relu) v = fmaxf(v, 0.f);
    Y[(int64_t)bt * out + o] = v;
  }
}

// softmax over the 64 logits of one sample, cumulative sums -> 63 boundaries.
// With a target: per-sample loss share and dL/dlogits.
__global__ void __launch_bounds__(64) mlp_head_kernel(int B, const float* __restrict__ Z, float* __restrict__ bounds,
                                                      const float* __restrict__ target, float* __restrict__ dZ,
                                                      float* __restrict__ loss_part) {
  const int bt = blockIdx.x, j = threadIdx.x;
  __shared__ float p[kOut], cs[kOut], dc[kOut], dp[kOut];
  __shared__ float red[2];
  const float z = Z[(int64_t)bt * kOut + j];
  float m = z;
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((j & 31) == 0) red[j >> 5] = m;
  __syncthreads();
  m = fmaxf(red[0], red[1]);
  __syncthreads();
  const float e = expf(z - m);
  float s = e;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((j & 31) == 0) red[j >> 5] = s;
  __syncthreads();
  s = red[0] + red[1];
  p[j] = e / s;
  __syncthreads();
  if (j == 0) {
    float c = 0.f;
    for (int k = 0; k < kOut; ++k) {
      c += p[k];
      cs[k] = c;
    }
  }
  __syncthreads();
  if (j < kOut - 1) bounds[(int64_t)bt * (kOut - 1) + j] = cs[j];
  if (!target) return;
  const float scale = 1.0f / ((float)B * (float)(kOut - 1));
  float l = 0.f;
  if (j < kOut - 1) {
    const float d = cs[j] - target[(int64_t)bt * (kOut - 1) + j];
    l = d * d * scale;
    dc[j] = 2.f * d * scale;
  } else {
    dc[j] = 0.f;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  __syncthreads();
  if ((j & 31) == 0) red[j >> 5] = l;
  __syncthreads();
  if (j == 0) {
    loss_part[bt] = red[0] + red[1];
    float acc = 0.f;  // dL/dp_k = sum_{i >= k} dL/dc_i
    for (int k = kOut - 1; k >= 0; --k) {
      acc += dc[k];
      dp[k] = acc;
    }
  }
  __syncthreads();
  float sdp = p[j] * dp[j];
  for (int o = 16; o > 0; o >>= 1) sdp += __shfl_xor_sync(0xffffffffu, sdp, o);
  if ((j & 31) == 0) red[j >> 5] = sdp;
  __syncthreads();
  sdp = red[0] + red[1];
  dZ[(int64_t)bt * kOut + j] = p[j] * (dp[j] - sdp);
}

// dX[bt][i] = (sum_o dY[bt][o] W[o][i]) * [Xact[bt][i] > 0]: the gradient with
// respect to the pre-activation of the previous layer
__global__ void __launch_bounds__(256) mlp_bwd_x_kernel(int B, int in, int out, const float* __restrict__ dY,
                                                        const float* __restrict__ W, const float* __restrict__ Xact,
                                                        float* __restrict__ dX) {
  __shared__ float Ds[32][33], Ws[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < out; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      Ds[r][c] = (b0 + r < B && k0 + c < out) ? dY[(int64_t)(b0 + r) * out + k0 + c] : 0.f;
      Ws[r][c] = (k0 + r < out && i0 + c < in) ? W[(int64_t)(k0 + r) * in + i0 + c] : 0.f;  // Ws[o][i]
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float wv = Ws[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(Ds[ty + 8 * q][k], wv, acc[q]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i >= in) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int bt = b0 + ty + 8 * q;
    if (bt >= B) continue;
    const float v = Xact[(int64_t)bt * in + i] > 0.f ? acc[q] : 0.f;
    dX[(int64_t)bt * in + i] = v;
  }
}

// dW[o][i] = sum_bt dY[bt][o] X[bt][i]; the CTAs of the first column tile also
// write db[o] = sum_bt dY[bt][o]
__global__ void __launch_bounds__(256) mlp_bwd_w_kernel(int B, int in, int out, const float* __restrict__ dY,
                                                        const float* __restrict__ X, float* __restrict__ dW,
                                                        float* __restrict__ db) {
  __shared__ float Ds[32][33], Xs[32][33];
  const int i0 = blockIdx.x * 32, o0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (int k0 = 0; k0 < B; k0 += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      Ds[r][c] = (k0 + r < B && o0 + c < out) ? dY[(int64_t)(k0 + r) * out + o0 + c] : 0.f;
      Xs[r][c] = (k0 + r < B && i0 + c < in) ? X[(int64_t)(k0 + r) * in + i0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float xv = Xs[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(Ds[k][ty + 8 * q], xv, acc[q]);
    }
    if (blockIdx.x == 0 && ty == 0)
      for (int k = 0; k < 32; ++k) bacc += Ds[k][tx];
    __syncthreads();
  }
  const int i = i0 + tx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = o0 + ty + 8 * q;
    if (o < out && i < in) dW[(int64_t)o * in + i] = acc[q];
  }
  if (blockIdx.x == 0 && ty == 0 && o0 + tx < out) db[o0 + tx] = bacc;
}

__global__ void adam_kernel(int64_t np, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void loss_sum_kernel(int B, const float* __restrict__ part, float* __restrict__ loss) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = threadIdx.x; i < B; i += blockDim.x) s += part[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *loss = t;
  }
}

struct MlpWs {
  float* act[5];   // act[l] = input of layer l (act[0] unused: the caller's X)
  float* dact[5];  // dact[l] = dL/d(pre-activation feeding act[l])
  float* lpart;
};

static MlpWs plan_mlp(Arena& a, int B) {
  MlpWs w;
  const int dims[5] = {kFeat, kHid, kHid, kHid, kOut};
  for (int l = 0; l < 5; ++l) {
    w.act[l] = l == 0 ? nullptr : a.take<float>((size_t)B * dims[l]);
    w.dact[l] = l == 0 ? nullptr : a.take<float>((size_t)B * dims[l]);
  }
  w.lpart = a.take<float>(B);
  return w;
}

// forward (bounds); with target: loss; with grad: full backward pass into grad
static int mlp_run(int B, const float* params, const float* X, float* bounds, const float* target, float* grad,
                   float* loss, const MlpWs& w, cudaStream_t st) {
  Layer L[4];
  layer_table(L);
  const float* in = X;
  for (int l = 0; l < 4; ++l) {
    dim3 g((unsigned)ceil_div(L[l].out, 32), (unsigned)ceil_div(B, 32));
    mlp_fwd_kernel<<<g, 256, 0, st>>>(B, L[l].in, L[l].out, in, params + L[l].w, params + L[l].b, w.act[l + 1],
                                      l < 3 ? 1 : 0);
    PD_CK_LAUNCH();
    in = w.act[l + 1];
  }
  mlp_head_kernel<<<B, kOut, 0, st>>>(B, w.act[4], bounds, target, w.dact[4], w.lpart);
  PD_CK_LAUNCH();
  if (!target) return 0;
  loss_sum_kernel<<<1, 256, 0, st>>>(B, w.lpart, loss);
  PD_CK_LAUNCH();
  if (!grad) return 0;
  for (int l = 3; l >= 0; --l) {
    const float* xin = l == 0 ? X : w.act[l];
    dim3 gw((unsigned)ceil_div(L[l].in, 32), (unsigned)ceil_div(L[l].out, 32));
    mlp_bwd_w_kernel<<<gw, 256, 0, st>>>(B, L[l].in, L[l].out, w.dact[l + 1], xin, grad + L[l].w, grad + L[l].b);
    PD_CK_LAUNCH();
    if (l > 0) {
      dim3 gx((unsigned)ceil_div(L[l].in, 32), (unsigned)ceil_div(B, 32));
      mlp_bwd_x_kernel<<<gx, 256, 0, st>>>(B, L[l].in, L[l].out, w.dact[l + 1], params + L[l].w, w.act[l],
                                           w.dact[l]);
      PD_CK_LAUNCH();
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// proposal + validation + multisection fix-up
// ---------------------------------------------------------------------------
// Normalised position of count fraction f from the 63 predicted boundaries
// (grid fractions j/64, end points 0 -> 0 and 1 -> 1), piecewise linear.
static double inverse_cdf(const float* c63, double f) {
  if (!c63) return f;  // no network: uniform density over the Gershgorin interval
  f = std::min(1.0, std::max(0.0, f));
  const double x = f * kOut;
  int j = (int)floor(x);
  if (j >= kOut) j = kOut - 1;
  const double t = x - j;
  auto g = [&](int q) -> double {
    if (q <= 0) return 0.0;
    if (q >= kOut) return 1.0;
    return std::min(1.0, std::max(0.0, (double)c63[q - 1]));
  };
  return g(j) + t * (g(j + 1) - g(j));
}

struct Probe {
  double sigma;
  int64_t neg;
};

static int propose(int64_t n, int b, int cplx, const void* band, int64_t ldab, const float* c63, double lo,
                   double hi, double f0, double f1, int K, int count_tol, int fanout, double* bounds,
                   int32_t* counts, int32_t* used_fallback, int64_t* evals_out, int64_t* proposed_counts,
                   void* iw, size_t iws, cudaStream_t st) {
  const double span = hi - lo;
  const double pad = 1e-3 * (span > 0 ? span : 1.0) + 1e-300;
  const double below = lo - pad, above = hi + pad;  // count 0 and n by the Gershgorin theorem
  std::vector<int64_t> tgt(K + 1);
  std::vector<double> sig(K + 1);
  std::vector<int64_t> neg(K + 1, -1);
  for (int k = 0; k <= K; ++k) {
    const double f = f0 + (f1 - f0) * k / K;
    tgt[k] = std::min<int64_t>(n, std::max<int64_t>(0, (int64_t)floor(f * (double)n + 0.5)));
    if (tgt[k] == 0) {
      sig[k] = below;
      neg[k] = 0;
    } else if (tgt[k] == n) {
      sig[k] = above;
      neg[k] = n;
    } else {
      sig[k] = lo + span * inverse_cdf(c63, (double)tgt[k] / (double)n);
    }
  }
  std::vector<Probe> seen = {{below, 0}, {above, n}};
  int64_t evals = 0;
  auto evaluate = [&](const std::vector<double>& s, std::vector<int64_t>& out) -> int {
    out.assign(s.size(), 0);
    if (s.empty()) return 0;
    if (inertia_ws_bytes(b, cplx, (int)s.size()) > iws) return PDESHEP_WORKSPACE_TOO_SMALL;
    bool bad = false;
    PD_TRY(inertia_counts(n, b, cplx, band, ldab, (int)s.size(), s.data(), out.data(), nullptr, iw, iws, st, &bad));
    if (bad) return PDESHEP_NONFINITE_INPUT;
    evals += (int64_t)s.size();
    for (size_t e = 0; e < s.size(); ++e) seen.push_back({s[e], out[e]});
    return 0;
  };
  // 1. validate every proposed interior boundary in one inertia launch
  std::vector<double> s;
  std::vector<int> owner;
  std::vector<int64_t> r;
  for (int k = 0; k <= K; ++k)
    if (neg[k] < 0) {
      s.push_back(sig[k]);
      owner.push_back(k);
    }
  PD_TRY(evaluate(s, r));
  for (size_t e = 0; e < s.size(); ++e) neg[owner[e]] = r[e];
  auto ok = [&](int k) { return llabs(neg[k] - tgt[k]) <= count_tol; };
  std::vector<int> todo;
  for (int k = 0; k <= K; ++k)
    if (!ok(k)) todo.push_back(k);
  if (used_fallback) *used_fallback = (int32_t)todo.size();
  if (proposed_counts)
    for (int k = 0; k <= K; ++k) proposed_counts[k] = neg[k];
  // 2. multisection on the failed boundaries.  Every count evaluated so far
  // (for any boundary) is reused: a point inside a boundary's window is taken
  // at once, the others bracket it as [a, c] with count(a) < target - tol and
  // count(c) > target + tol (counts are monotone in sigma).
  auto closest_in_window = [&](int k) -> const Probe* {
    const Probe* best = nullptr;
    for (const Probe& q : seen)
      if (llabs(q.neg - tgt[k]) <= count_tol && (!best || llabs(q.neg - tgt[k]) < llabs(best->neg - tgt[k])))
        best = &q;
    return best;
  };
  for (int round = 0; round < 200 && !todo.empty(); ++round) {
    s.clear();
    owner.clear();
    std::vector<int> next;
    for (int k : todo) {
      if (const Probe* q = closest_in_window(k)) {
        sig[k] = q->sigma;
        neg[k] = q->neg;
        continue;
      }
      double a = below, c = above;
      int64_t na = 0, nc = n;
      for (const Probe& q : seen) {
        if (q.neg < tgt[k] - count_tol && q.sigma > a) {
          a = q.sigma;
          na = q.neg;
        }
        if (q.neg > tgt[k] + count_tol && q.sigma < c) {
          c = q.sigma;
          nc = q.neg;
        }
      }
      const double w = c - a;
      next.push_back(k);
      if (!(w > 4e-16 * std::max(1.0, std::max(fabs(a), fabs(c))))) continue;  // unsplittable cluster
      auto add = [&](double x) {
        if (x > a && x < c) {
          s.push_back(x);
          owner.push_back(k);
        }
      };
      if (fanout == 1) {
        add(a + 0.5 * w);  // plain bisection
      } else {
        // one point where the straight line through (a, count(a)) and
        // (c, count(c)) reaches the target (regula falsi on the counting
        // function), the others split [a, c] evenly so that the bracket
        // shrinks by fanout whatever the interpolation is worth
        add(a + w * ((double)(tgt[k] - na) / (double)(nc - na)));
        for (int f = 1; f < fanout; ++f) add(a + w * f / fanout);
      }
    }
    todo.swap(next);
    if (s.empty()) break;
    PD_TRY(evaluate(s, r));
  }
  for (size_t e = 0; e < todo.size();) {  // windows met by the last round's points
    const int k = todo[e];
    if (const Probe* q = closest_in_window(k)) {
      sig[k] = q->sigma;
      neg[k] = q->neg;
      todo.erase(todo.begin() + e);
    } else {
      ++e;
    }
  }
  // boundaries whose window could not be reached (a cluster wider than the
  // tolerance): the evaluated point with the closest count
  for (int k : todo) {
    const Probe* bestp = nullptr;
    for (const Probe& q : seen)
      if (!bestp || llabs(q.neg - tgt[k]) < llabs(bestp->neg - tgt[k])) bestp = &q;
    sig[k] = bestp->sigma;
    neg[k] = bestp->neg;
  }
  // order (sigma, count) pairs together; counts are monotone in sigma
  std::vector<Probe> fin(K + 1);
  for (int k = 0; k <= K; ++k) fin[k] = {sig[k], neg[k]};
  std::sort(fin.begin(), fin.end(), [](const Probe& x, const Probe& y) {
    return x.sigma < y.sigma || (x.sigma == y.sigma && x.neg < y.neg);
  });
  for (int k = 0; k <= K; ++k) bounds[k] = fin[k].sigma;
  for (int k = 0; k < K; ++k) counts[k] = (int32_t)(fin[k + 1].neg - fin[k].neg);
  if (evals_out) *evals_out = evals;
  return 0;
}

static size_t propose_inertia_bytes(int b, int cplx, int K, int fanout) {
  return std::max(inertia_ws_bytes(b, cplx, (K + 1) * std::max(1, fanout)), (size_t)4096);
}

}  // namespace pdeshep

using namespace pdeshep;

extern "C" int64_t pdeshep_mlp_param_count(void) { return kNParams; }

extern "C" size_t pdeshep_slice_features_workspace_size(int64_t n, int32_t is_complex) {
  if (n <= 0) return 0;
  Arena a;
  plan_feat(a, n, is_complex ? sizeof(double2) : sizeof(double));
  return a.used();
}

extern "C" int pdeshep_slice_features(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                      uint64_t seed, float* d_features, void* d_work, size_t work_bytes,
                                      void* stream) {
  if (n <= 0) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (!d_features) return -7;
  if (!d_work) return -8;
  Arena a(d_work, work_bytes);
  const FeatWs w = plan_feat(a, n, is_complex ? sizeof(double2) : sizeof(double));
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  if (is_complex) return features<double2>(n, b, 1, d_band, ldab, seed, d_features, w, st);
  return features<double>(n, b, 0, d_band, ldab, seed, d_features, w, st);
}

extern "C" size_t pdeshep_mlp_workspace_size(int32_t batch) {
  if (batch <= 0) return 0;
  Arena a;
  plan_mlp(a, batch);
  a.take<float>(kNParams);
  a.take<float>((size_t)batch * (kOut - 1));
  return a.used();
}

extern "C" int pdeshep_mlp_forward(const float* d_params, int32_t batch, const float* d_x, float* d_bounds,
                                   void* d_work, size_t work_bytes, void* stream) {
  if (!d_params) return -1;
  if (batch <= 0 || batch > 65535) return -2;
  if (!d_x) return -3;
  if (!d_bounds) return -4;
  if (!d_work) return -5;
  Arena a(d_work, work_bytes);
  const MlpWs w = plan_mlp(a, batch);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  return mlp_run(batch, d_params, d_x, d_bounds, nullptr, nullptr, nullptr, w, (cudaStream_t)stream);
}

extern "C" int pdeshep_mlp_grad(const float* d_params, int32_t batch, const float* d_x, const float* d_target,
                                float* d_grad, float* d_loss, void* d_work, size_t work_bytes, void* stream) {
  if (!d_params) return -1;
  if (batch <= 0 || batch > 65535) return -2;
  if (!d_x) return -3;
  if (!d_target) return -4;
  if (!d_grad) return -5;
  if (!d_loss) return -6;
  if (!d_work) return -7;
  Arena a(d_work, work_bytes);
  const MlpWs w = plan_mlp(a, batch);
  float* bounds = a.take<float>((size_t)batch * (kOut - 1));
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  return mlp_run(batch, d_params, d_x, bounds, d_target, d_grad, d_loss, w, (cudaStream_t)stream);
}

extern "C" int pdeshep_mlp_train_step(float* d_params, float* d_adam_m, float* d_adam_v, int32_t step, float lr,
                                      int32_t batch, const float* d_x, const float* d_target, float* d_loss,
                                      void* d_work, size_t work_bytes, void* stream) {
  if (!d_params) return -1;
  if (!d_adam_m) return -2;
  if (!d_adam_v) return -3;
  if (step < 1) return -4;
  if (!(lr > 0.f)) return -5;
  if (batch <= 0 || batch > 65535) return -6;
  if (!d_x) return -7;
  if (!d_target) return -8;
  if (!d_loss) return -9;
  if (!d_work) return -10;
  Arena a(d_work, work_bytes);
  const MlpWs w = plan_mlp(a, batch);
  float* grad = a.take<float>(kNParams);
  float* bounds = a.take<float>((size_t)batch * (kOut - 1));
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  cudaStream_t st = (cudaStream_t)stream;
  PD_TRY(mlp_run(batch, d_params, d_x, bounds, d_target, grad, d_loss, w, st));
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<152, 256, 0, st>>>(kNParams, d_params, grad, d_adam_m, d_adam_v, lr, b1, b2, 1e-8f, c1, c2);
  PD_CK_LAUNCH();
  return 0;
}

extern "C" size_t pdeshep_propose_workspace_size(int64_t n, int32_t b, int32_t is_complex, int32_t nslices,
                                                 int32_t fanout) {
  if (n <= 0 || b < 0 || nslices < 1 || nslices > kMaxSlices || fanout < 1 || fanout > 64) return 0;
  Arena a;
  plan_feat(a, n, is_complex ? sizeof(double2) : sizeof(double));
  plan_mlp(a, 1);
  a.take<float>(kFeat);
  a.take<float>(kOut);
  a.take<char>(propose_inertia_bytes(b, is_complex ? 1 : 0, nslices, fanout));
  return a.used();
}

extern "C" int pdeshep_propose_slices(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                      const float* d_params, uint64_t seed, double frac_lo, double frac_hi,
                                      int32_t nslices, int32_t count_tol, int32_t fanout, double* h_bounds,
                                      int32_t* h_counts, int32_t* h_used_fallback, int64_t* h_inertia_evals,
                                      int64_t* h_proposed_counts, void* d_work, size_t work_bytes,
                                      void* stream) {
  if (n <= 0) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (!(frac_lo >= 0.0 && frac_lo < 1.0)) return -8;
  if (!(frac_hi > frac_lo && frac_hi <= 1.0)) return -9;
  if (nslices < 1 || nslices > kMaxSlices) return -10;
  if (count_tol < 0) return -11;
  if (fanout < 1 || fanout > 64) return -12;
  if (!h_bounds) return -13;
  if (!h_counts) return -14;
  if (!d_work) return -18;
  const int cplx = is_complex ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  Arena a(d_work, work_bytes);
  const FeatWs fw = plan_feat(a, n, cplx ? sizeof(double2) : sizeof(double));
  const MlpWs mw = plan_mlp(a, 1);
  float* feat = a.take<float>(kFeat);
  float* bnd = a.take<float>(kOut);
  const size_t iws = propose_inertia_bytes(b, cplx, nslices, fanout);
  char* iw = a.take<char>(iws);
  if (!a.fits()) return PDESHEP_WORKSPACE_TOO_SMALL;
  double lohi[2];
  float c63[kOut - 1];
  if (d_params) {
    if (cplx)
      PD_TRY(features<double2>(n, b, 1, d_band, ldab, seed, feat, fw, st));
    else
      PD_TRY(features<double>(n, b, 0, d_band, ldab, seed, feat, fw, st));
    PD_TRY(mlp_run(1, d_params, feat, bnd, nullptr, nullptr, nullptr, mw, st));
    PD_CK(cudaMemcpyAsync(c63, bnd, sizeof(float) * (kOut - 1), cudaMemcpyDeviceToHost, st));
  } else {
    PD_TRY(gershgorin_device(n, b, cplx, d_band, ldab, fw.glo, fw.ghi, st));
    lohi_kernel<<<1, 32, 0, st>>>(fw.glo, fw.ghi, fw.lohi);
    PD_CK_LAUNCH();
  }
  PD_CK(cudaMemcpyAsync(lohi, fw.lohi, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  PD_CK(cudaStreamSynchronize(st));
  if (!std::isfinite(lohi[0]) || !std::isfinite(lohi[1])) return PDESHEP_NONFINITE_INPUT;
  int32_t used = 0;
  int64_t evals = 0;
  PD_TRY(propose(n, b, cplx, d_band, ldab, d_params ? c63 : nullptr, lohi[0], lohi[1], frac_lo, frac_hi, nslices,
                 count_tol, fanout, h_bounds, h_counts, &used, &evals, h_proposed_counts, iw, iws, st));
  if (h_used_fallback) *h_used_fallback = used;
  if (h_inertia_evals) *h_inertia_evals = evals;
  return 0;
}

// ---------------------------------------------------------------------------
// Training labels of the proposer: the equal-count boundaries, each the
// midpoint between eigenvalues t_k - 1 and t_k (t_k = round(k n / nslices),
// k = 1..nslices-1, clipped to [1, n-1]) enclosed by bisection on inertia,
// normalised to the Gershgorin interval [lo, hi] and clipped to [0, 1].
// ---------------------------------------------------------------------------
extern "C" size_t pdeshep_equal_count_targets_workspace_size(int64_t n, int32_t b, int32_t is_complex,
                                                             int32_t nslices, int32_t fanout) {
  if (nslices < 2 || fanout < 1) return 0;
  const size_t bis = pdeshep_bisect_workspace_size(n, b, is_complex, 2 * (nslices - 1), fanout);
  return std::max(bis, sizeof(double) * gershgorin_ws_doubles());
}

extern "C" int pdeshep_equal_count_targets(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                           int32_t nslices, double rtol, int32_t fanout, float* h_targets,
                                           void* d_work, size_t work_bytes, void* stream) {
  if (n < 2) return -1;
  if (b < 0) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (nslices < 2 || nslices > 65536) return -6;
  if (!(rtol > 0.0)) return -7;
  if (fanout < 1 || fanout > 64) return -8;
  if (!h_targets) return -9;
  if (!d_work || work_bytes < pdeshep_equal_count_targets_workspace_size(n, b, is_complex, nslices, fanout))
    return -10;
  double lo = 0.0, hi = 0.0;
  PD_TRY(pdeshep_gershgorin(n, b, is_complex, d_band, ldab, &lo, &hi, d_work, work_bytes, stream));
  const int nb = nslices - 1;
  std::vector<int64_t> t(nb), idx;
  for (int k = 1; k <= nb; ++k) {
    int64_t v = (2 * (int64_t)k * n + nslices) / (2 * (int64_t)nslices);
    t[k - 1] = std::min<int64_t>(std::max<int64_t>(v, 1), n - 1);
    idx.push_back(t[k - 1] - 1);
    idx.push_back(t[k - 1]);
  }
  std::sort(idx.begin(), idx.end());
  idx.erase(std::unique(idx.begin(), idx.end()), idx.end());
  std::vector<double> elo(idx.size()), ehi(idx.size());
  PD_TRY(pdeshep_bisect(n, b, is_complex, d_band, ldab, (int32_t)idx.size(), idx.data(), rtol, fanout, elo.data(),
                        ehi.data(), d_work, work_bytes, stream));
  auto mid = [&](int64_t k) {
    const size_t p = std::lower_bound(idx.begin(), idx.end(), k) - idx.begin();
    return 0.5 * (elo[p] + ehi[p]);
  };
  const double span = hi > lo ? hi - lo : 1.0;
  for (int k = 0; k < nb; ++k) {
    const double sig = 0.5 * (mid(t[k] - 1) + mid(t[k]));
    const double u = (sig - lo) / span;
    h_targets[k] = (float)(u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u));
  }
  return 0;
}
