// partition.cu -- re-slicing the spectrum from the eigenvalues of the previous
// matrix of a sequence (Section 3.1 of arXiv 2012.00506), and the outer bounds
// of the wanted part of the spectrum (Section 3.2, Algorithm 4).
//
// The partitions are host work: one pass (or a few sweeps) over the sorted
// eigenvalues of the previous step, microseconds for the tens of thousands of
// values a call handles, while the counts that validate them come from the
// inertia kernel.  Groups are defined by value, G_i = {d : b_{i-1} <= d < b_i},
// so a group and the slice [b_{i-1}, b_i) of pdeshep_band_slice count the same
// eigenvalues and ties never straddle a boundary.
//
//  * equal counts ("Approach-1"): K groups of floor(n/K) or floor(n/K)+1 points
//    (the first n mod K groups hold the extra point), boundaries at the midpoints
//    of the gaps between consecutive groups;
//  * equal widths ("Approach-2"): [b0, bK] cut into K equal pieces;
//  * simplified one-dimensional k-means (Algorithm 3): from the equal-count
//    start, every inner boundary in turn moves to the midpoint of the gap that
//    follows the midpoint of its two groups' centroids (a group's centroid is the
//    mean of its extreme points); the sweeps repeat until no boundary moves, and
//    groups that become empty are merged away, so K may shrink.
//
// After a re-slicing the start vectors of the next call come from the previous
// call's vectors whose Ritz values fall in each new slice (the paper interlaces
// random vectors when a slice grows and removes some when it shrinks):
// pdeshep_restart_plan lists, per new slice, the previous columns to copy and the
// number of random ones.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace pdeshep {
namespace {

// first index with d[k] >= x / d[k] > x
int64_t lower_idx(const double* d, int64_t n, double x) { return std::lower_bound(d, d + n, x) - d; }
int64_t upper_idx(const double* d, int64_t n, double x) { return std::upper_bound(d, d + n, x) - d; }

void dedup(std::vector<double>& b) {
  std::vector<double> out;
  out.reserve(b.size());
  for (double v : b)
    if (out.empty() || v != out.back()) out.push_back(v);
  b.swap(out);
}

std::vector<double> equal_counts(const double* d, int64_t n, int K, double b0, double bK) {
  const int64_t q = n / K, r = n % K;
  std::vector<double> b(1, b0);
  int64_t end = 0;
  for (int i = 1; i < K; ++i) {
    end += q + (i <= r ? 1 : 0);
    if (end <= 0)
      b.push_back(b0);
    else if (end >= n)
      b.push_back(bK);
    else
      b.push_back(0.5 * (d[end - 1] + d[end]));
  }
  b.push_back(bK);
  dedup(b);
  return b;
}

std::vector<double> equal_widths(int K, double b0, double bK) {
  std::vector<double> b;
  for (int i = 0; i < K; ++i) b.push_back(b0 + (bK - b0) * (double)i / (double)K);
  b.push_back(bK);
  dedup(b);
  return b;
}

int kmeans(const double* d, int64_t n, int K, double b0, double bK, int max_sweeps, std::vector<double>& b) {
  b = equal_counts(d, n, K, b0, bK);
  int sweeps = 0;
  while (sweeps < max_sweeps) {
    ++sweeps;
    const std::vector<double> old = b;
    for (size_t i = 1; i + 1 < b.size(); ++i) {
      const int64_t l0 = lower_idx(d, n, b[i - 1]), l1 = lower_idx(d, n, b[i]), l2 = lower_idx(d, n, b[i + 1]);
      if (l1 <= l0 || l2 <= l1) continue;  // an empty neighbour: merged away below
      const double c_left = 0.5 * (d[l0] + d[l1 - 1]);
      const double c_right = 0.5 * (d[l1] + d[l2 - 1]);
      const double t = 0.5 * (c_left + c_right);
      const int64_t ell = upper_idx(d, n, t);  // d[ell-1] <= t < d[ell]; c_left < t < c_right keeps 1 <= ell < n
      b[i] = 0.5 * (d[ell] + d[ell - 1]);
    }
    dedup(b);
    if (b == old) break;
  }
  return sweeps;
}

}  // namespace
}  // namespace pdeshep

using namespace pdeshep;

extern "C" int pdeshep_partition(int32_t method, int64_t n, const double* h_d, int32_t K, double b0, double bK,
                                 int32_t max_sweeps, double* h_bounds, int32_t* h_counts, int32_t* h_k_out,
                                 int32_t* h_sweeps) {
  if (method < PDESHEP_PART_KMEANS || method > PDESHEP_PART_EQUAL_WIDTH) return -1;
  if (n < 1) return -2;
  if (!h_d) return -3;
  for (int64_t k = 1; k < n; ++k)
    if (!(h_d[k - 1] <= h_d[k])) return -3;  // ascending, no NaN
  if (K < 1) return -4;
  if (!(b0 <= h_d[0])) return -5;
  if (!(h_d[n - 1] < bK)) return -6;
  if (method == PDESHEP_PART_KMEANS && max_sweeps < 1) return -7;
  if (!h_bounds) return -8;
  if (!h_counts) return -9;
  if (!h_k_out) return -10;
  std::vector<double> b;
  int sweeps = 0;
  if (method == PDESHEP_PART_KMEANS)
    sweeps = kmeans(h_d, n, K, b0, bK, max_sweeps, b);
  else if (method == PDESHEP_PART_EQUAL_COUNT)
    b = equal_counts(h_d, n, K, b0, bK);
  else
    b = equal_widths(K, b0, bK);
  const int kout = (int)b.size() - 1;
  for (int i = 0; i <= kout; ++i) h_bounds[i] = b[i];
  for (int i = 0; i < kout; ++i)
    h_counts[i] = (int32_t)(lower_idx(h_d, n, b[i + 1]) - lower_idx(h_d, n, b[i]));
  *h_k_out = kout;
  if (h_sweeps) *h_sweeps = sweeps;
  return 0;
}

extern "C" int pdeshep_restart_plan(int64_t nprev, const double* h_prev_vals, int32_t K, const double* h_bounds,
                                    const int32_t* h_m0, int32_t mode, int64_t* h_src) {
  if (nprev < 0) return -1;
  if (nprev > 0 && !h_prev_vals) return -2;
  for (int64_t k = 0; k < nprev; ++k)
    if (!std::isfinite(h_prev_vals[k])) return -2;
  if (K < 1) return -3;
  if (!h_bounds) return -4;
  for (int i = 0; i < K; ++i)
    if (!(h_bounds[i] < h_bounds[i + 1])) return -4;
  if (!h_m0) return -5;
  for (int i = 0; i < K; ++i)
    if (h_m0[i] < 0) return -5;
  if (mode != 0 && mode != 1) return -6;
  if (!h_src) return -7;
  const double* v = h_prev_vals;
  int64_t off = 0;
  for (int i = 0; i < K; ++i) {
    const double lo = h_bounds[i], hi = h_bounds[i + 1], c = 0.5 * (lo + hi);
    const int64_t m = h_m0[i];
    std::vector<int64_t> inside, outside;
    for (int64_t k = 0; k < nprev; ++k) (lo <= v[k] && v[k] < hi ? inside : outside).push_back(k);
    if ((int64_t)inside.size() > m) {  // keep the m nearest to the centre
      std::stable_sort(inside.begin(), inside.end(), [&](int64_t a, int64_t b) {
        const double da = fabs(v[a] - c), db = fabs(v[b] - c);
        return da < db || (da == db && a < b);
      });
      inside.resize(m);
    }
    std::stable_sort(inside.begin(), inside.end(),
                     [&](int64_t a, int64_t b) { return v[a] < v[b] || (v[a] == v[b] && a < b); });
    int64_t q = 0;
    for (int64_t k : inside) h_src[off + q++] = k;
    if (mode == 1 && q < m) {  // then the nearest columns outside the slice
      auto dist = [&](int64_t k) { return v[k] < lo ? lo - v[k] : v[k] - hi; };
      std::stable_sort(outside.begin(), outside.end(), [&](int64_t a, int64_t b) {
        const double da = dist(a), db = dist(b);
        if (da != db) return da < db;
        if (v[a] != v[b]) return v[a] < v[b];
        return a < b;
      });
      for (size_t t = 0; t < outside.size() && q < m; ++t) h_src[off + q++] = outside[t];
    }
    for (; q < m; ++q) h_src[off + q] = -1;  // a random start vector
    off += m;
  }
  return 0;
}

extern "C" size_t pdeshep_outer_bounds_workspace_size(int64_t n, int32_t b, int32_t is_complex) {
  return pdeshep_inertia_workspace_size(n, b, is_complex, 1);
}

extern "C" int pdeshep_outer_bounds(int64_t n, int32_t b, int32_t is_complex, const void* d_band, int64_t ldab,
                                    int64_t nprev, const double* h_prev, int64_t i0, int64_t nev, double alpha,
                                    double m_hat, int32_t max_it, double* h_b0, double* h_bK, int32_t* h_iters,
                                    void* d_work, size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (b < 0 || b >= n) return -2;
  if (!d_band) return -4;
  if (ldab < b + 1) return -5;
  if (!h_prev) return -7;
  if (nprev < 1) return -6;
  for (int64_t k = 1; k < nprev; ++k)
    if (!(h_prev[k - 1] <= h_prev[k])) return -7;
  if (i0 < 0 || i0 >= nprev) return -8;
  if (nev < 1 || i0 + nev > nprev || i0 + nev > n) return -9;
  if (!(m_hat >= 0.0) || !std::isfinite(alpha)) return -11;
  if (max_it < 1) return -12;
  if (!h_b0 || !h_bK) return -13;
  if (!d_work) return -16;
  auto count_below = [&](double sigma, int64_t* neg) -> int {
    return pdeshep_inertia(n, b, is_complex, d_band, ldab, 1, &sigma, neg, nullptr, d_work, work_bytes, stream);
  };
  // upper bound (Algorithm 4): stop once every wanted eigenvalue lies below it
  const double du = h_prev[i0 + nev - 1];
  const double delta = nev >= 2 ? du - h_prev[i0 + nev - 2] : 0.0;
  double step = std::max(fabs(alpha * du), m_hat * delta);
  if (!(step > 0.0)) step = ldexp(1.0, -40) * std::max(1.0, fabs(du));
  double bK = du + step;
  int it_hi = 1;
  bool hi_ok = false;
  for (;;) {
    int64_t neg = 0;
    PD_TRY(count_below(bK, &neg));
    hi_ok = neg >= i0 + nev;
    if (hi_ok || it_hi >= max_it) break;
    bK = bK + step;
    ++it_hi;
  }
  // lower bound: stop once no wanted eigenvalue lies below it
  const double dl = h_prev[i0];
  const double delta2 = i0 + 1 < nprev ? h_prev[i0 + 1] - dl : 0.0;
  double step2 = std::max(fabs(alpha * dl), m_hat * delta2);
  if (!(step2 > 0.0)) step2 = ldexp(1.0, -40) * std::max(1.0, fabs(dl));
  double b0 = dl - step2;
  int it_lo = 1;
  bool lo_ok = false;
  for (;;) {
    int64_t neg = 0;
    PD_TRY(count_below(b0, &neg));
    lo_ok = neg <= i0;
    if (lo_ok || it_lo >= max_it) break;
    b0 = b0 - step2;
    ++it_lo;
  }
  *h_b0 = b0;
  *h_bK = bK;
  if (h_iters) {
    h_iters[0] = it_lo;
    h_iters[1] = it_hi;
  }
  // a search that used its max_it counts without reaching its target leaves bounds
  // that do not enclose the wanted eigenvalues
  return hi_ok && lo_ok ? 0 : PDESHEP_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------
// The start block of a re-sliced call from a restart plan, on the device:
// column j of d_dst is column h_src[j] of d_prev, or (h_src[j] < 0) column
// col0 + j of the library's start-vector stream (the random vectors that
// interlace the previous ones, Section 3.1).
// ---------------------------------------------------------------------------
namespace pdeshep {
namespace {
template <typename S>
__global__ void gather_columns_kernel(int64_t n, int ncols, const int64_t* __restrict__ src, const S* __restrict__ prev,
                                      int64_t col0, uint64_t seed, S* __restrict__ dst) {
  const int64_t total = n * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, i = e % n;
    const int64_t sc = src[c];
    if (sc >= 0) {
      dst[e] = prev[i + sc * n];
    } else {
      const uint64_t k = (uint64_t)((col0 + c) * n + i);
      if constexpr (std::is_same<S, double>::value)
        dst[e] = uniform_pm1(splitmix64(seed + k));
      else
        dst[e] = make_double2(uniform_pm1(splitmix64(seed + 2 * k)), uniform_pm1(splitmix64(seed + 2 * k + 1)));
    }
  }
}
}  // namespace
}  // namespace pdeshep

extern "C" size_t pdeshep_gather_columns_workspace_size(int32_t ncols) {
  return ncols > 0 ? (((size_t)ncols * sizeof(int64_t) + 255) & ~size_t(255)) : 0;
}

extern "C" int pdeshep_gather_columns(int64_t n, int32_t is_complex, const void* d_prev, int64_t nprev, int32_t ncols,
                                      const int64_t* h_src, uint64_t seed, int64_t col0, void* d_dst, void* d_work,
                                      size_t work_bytes, void* stream) {
  if (n <= 0) return -1;
  if (nprev < 0 || (nprev > 0 && !d_prev)) return -4;
  if (ncols < 0) return -5;
  if (ncols > 0 && !h_src) return -6;
  for (int j = 0; j < ncols; ++j)
    if (h_src[j] >= nprev) return -6;
  if (col0 < 0) return -8;
  if (ncols > 0 && !d_dst) return -9;
  if (ncols == 0) return 0;
  if (!d_work || work_bytes < pdeshep_gather_columns_workspace_size(ncols)) return -10;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t* d_src = (int64_t*)d_work;
  PD_CK(cudaMemcpyAsync(d_src, h_src, sizeof(int64_t) * ncols, cudaMemcpyHostToDevice, st));
  const int64_t total = n * ncols;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  if (is_complex)
    gather_columns_kernel<double2><<<blocks, 256, 0, st>>>(n, ncols, d_src, (const double2*)d_prev, col0, seed,
                                                           (double2*)d_dst);
  else
    gather_columns_kernel<double><<<blocks, 256, 0, st>>>(n, ncols, d_src, (const double*)d_prev, col0, seed,
                                                          (double*)d_dst);
  PD_CK_LAUNCH();
  return 0;
}
