// band_lu.cu -- shifted band LU with partial pivoting inside the band and the
// multi-right-hand-side solves of eq. (10) of arXiv 2012.00506:
//     (z_j I - B) Q^(j) = X~,   j = 1..n_e.
//
// The band of semi-bandwidth b is handled as a block band of T x T tiles
// (T = 32, block semi-bandwidth bt = ceil(b/T)).  Partial pivoting over the
// rows k..k+b of column k is the same as pivoting over the (bt+1)T rows of
// the block panel, because the rows past k+b are structurally zero there, so
// the pivots equal those of LAPACK's gbtrf (first maximum of |Re|+|Im|).
// The U factor fills to 2b superdiagonals (2bt tiles).
//
// factor_kernel: one thread block per shifted system (the L2 level of the
//   paper's parallelism is the batch dimension).  Per block column K: the
//   panel ((bt+1)T x T) is factored in shared memory (warp-shuffle pivot
//   search, row swaps, rank-1 updates); the panel permutation is gathered
//   into each trailing block column on load; the top tile is multiplied by
//   the inverted unit-lower diagonal block and the tiles below get the
//   T-deep Schur update.  The inverses of the diagonal blocks are stored so
//   that every solve step is a tile product.
// solve kernels: one thread block per (system, 32-column block of right-hand
//   sides); forward L sweep then backward U sweep (trans = 0), or U^H then
//   L^H and the inverse permutation (trans = 1, the conjugate node conj(z)
//   of a Hermitian band).  Factor tiles stream from L2/HBM through shared
//   memory; each is reused by the 32 right-hand sides of the block.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "band_lu.cuh"

namespace pdeshep {

constexpr int kThreads = 256;
constexpr int kLdt = kTile + 1;

// ---------------------------------------------------------------------------
// init: tiles of z I - B (identity padding past n, zero fill slots)
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(kThreads) init_factor_kernel(FactorGeom g, int cplx,
                                                              const double* __restrict__ band,
                                                              int64_t ldab, const SysDesc* sys,
                                                              char* arena) {
  using R = typename real_of<C>::type;
  const int s = blockIdx.y;
  const SysDesc d = sys[s];
  FactorPtr<C> f = factor_ptr<C>(g, arena + d.factor_off);
  const int T = kTile;
  for (int64_t t = blockIdx.x; t < g.tiles; t += gridDim.x) {
    const int I = (int)(t / g.nslot);
    const int J = I + (int)(t % g.nslot) - g.bt;
    C* tile = f.tiles + t * g.tile_elems;
    for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
      const int r = e % T, c = e / T;
      const int64_t i = (int64_t)I * T + r, j = (int64_t)J * T + c;
      R vr = 0, vi = 0;
      if (J >= 0 && J < g.Nb) {
        if (i >= g.n || j >= g.n) {
          vr = (i == j) ? R(1) : R(0);
        } else {
          const int64_t dd = i - j;
          if (dd >= -g.b && dd <= g.b) {
            double br, bi;
            if (dd >= 0) {
              if (cplx) {
                br = band[2 * (dd + j * ldab)];
                bi = band[2 * (dd + j * ldab) + 1];
              } else {
                br = band[dd + j * ldab];
                bi = 0.0;
              }
            } else {
              if (cplx) {
                br = band[2 * (-dd + i * ldab)];
                bi = -band[2 * (-dd + i * ldab) + 1];
              } else {
                br = band[-dd + i * ldab];
                bi = 0.0;
              }
            }
            if (i == j) {
              vr = (R)(d.zre - br);
              vi = (R)d.zim;
            } else {
              vr = (R)(-br);
              vi = (R)(-bi);
            }
          }
        }
      }
      tile[e] = cmk<C>(vr, vi);
    }
  }
}

// (value, index) of the warp's largest value, the lowest index on ties, in every lane
template <typename R>
__device__ __forceinline__ void warp_argmax(R& best, int& idx) {
  for (int o = 16; o > 0; o >>= 1) {
    const R ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ob > best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
    }
  }
}

// ---------------------------------------------------------------------------
// factorization: one thread block per system
// ---------------------------------------------------------------------------
template <typename C>
__global__ void __launch_bounds__(kThreads) factor_kernel(FactorGeom g, const SysDesc* sys,
                                                         char* arena, int* status, int32_t* ipiv) {
  using R = typename real_of<C>::type;
  extern __shared__ __align__(16) char smem[];
  const int T = kTile;
  const int bt = g.bt;
  const int Pmax = (bt + 1) * T;
  const int ldp = Pmax + 1;
  C* Pan = (C*)smem;
  C* Cb = Pan + (size_t)ldp * T;
  C* Li = Cb + (size_t)ldp * T;
  C* Ui = Li + T * T;
  int* perm = (int*)(Ui + T * T);
  int* pos = perm + Pmax;  // [2][Pmax]
  __shared__ R wbest[64];
  __shared__ int widx[64];
  __shared__ int sh_status;

  const int sidx = blockIdx.x;
  const SysDesc d = sys[sidx];
  FactorPtr<C> f = factor_ptr<C>(g, arena + d.factor_off);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) sh_status = 0;

  for (int K = 0; K < g.Nb; ++K) {
    const int nbb = min(bt, g.Nb - 1 - K);
    const int nbr = min(2 * bt, g.Nb - 1 - K);
    const int P = (nbb + 1) * T;
    // load panel tiles (K+q, K)
    for (int e = tid; e < P * T; e += blockDim.x) {
      const int q = (e / (T * T)), w = e % (T * T);
      const int r = w % T, c = w / T;
      const C* tile = f.tiles + g.tile_index(K + q, K) * g.tile_elems;
      Pan[q * T + r + c * ldp] = tile[w];
    }
    for (int r = tid; r < P; r += blockDim.x) {
      perm[r] = r;
      pos[r] = r;
    }
    __syncthreads();
    // panel LU with partial pivoting, one CTA barrier per column.  Rows are addressed through
    // pos[] (logical -> physical row), so an interchange moves no data; a thread owns logical rows
    // tid, tid + blockDim.x, ...: it eliminates them and, in the same phase, takes their part of the
    // next column's pivot search (warp maxima in wbest/widx; every thread then reduces the warp
    // maxima itself).  The pivot is the largest |re| + |im| with the lowest row on ties, and every
    // element sees the same operations in the same order as with physical interchanges.
    {
      const int nw = blockDim.x >> 5;
      // the pivot search of column 0
      {
        R best = R(-1);
        int idx = 0x7fffffff;
        for (int r = tid; r < P; r += blockDim.x) {
          const R v = cabs1(Pan[r]);
          if (v > best) {
            best = v;
            idx = r;
          }
        }
        warp_argmax(best, idx);
        if (lane == 0) {
          wbest[warp] = best;
          widx[warp] = idx;
        }
      }
      __syncthreads();
      for (int c = 0; c < T; ++c) {
        const int cur = c & 1;
        const int* posc = pos + cur * Pmax;
        int* posn = pos + (cur ^ 1) * Pmax;
        R best = R(-1);
        int p = 0x7fffffff;
        for (int w = 0; w < nw; ++w) {
          const R ob = wbest[cur * 32 + w];
          const int oi = widx[cur * 32 + w];
          if (ob > best || (ob == best && oi < p)) {
            best = ob;
            p = oi;
          }
        }
        const int pp = posc[p], pc = posc[c];  // physical rows of the pivot and of logical row c
        if (tid == 0) {
          if (p != c) {
            int tp = perm[c];
            perm[c] = perm[p];
            perm[p] = tp;
          }
          const int64_t k = (int64_t)K * T + c;
          if (ipiv && k < g.n) ipiv[(int64_t)sidx * g.n + k] = (int32_t)((int64_t)K * T + p);
          if (!(best > R(0)) && sh_status == 0) sh_status = (int)(k + 1);
        }
        const bool ok = best > R(0);
        const C inv = ok ? crecip(Pan[pp + c * ldp]) : cmk<C>(0, 0);
        R nb = R(-1);
        int ni = 0x7fffffff;
        for (int r = tid; r < P; r += blockDim.x) {
          const int phys = r == c ? pp : (r == p ? pc : posc[r]);
          posn[r] = phys;
          if (r <= c) continue;
          if (ok) {
            const C l = cmul(Pan[phys + c * ldp], inv);
            Pan[phys + c * ldp] = l;
            for (int j = c + 1; j < T; ++j) cfms(Pan[phys + j * ldp], l, Pan[pp + j * ldp]);
          }
          if (c + 1 < T) {
            const R v = cabs1(Pan[phys + (c + 1) * ldp]);
            if (v > nb) {
              nb = v;
              ni = r;
            }
          }
        }
        warp_argmax(nb, ni);
        if (lane == 0) {
          wbest[(cur ^ 1) * 32 + warp] = nb;
          widx[(cur ^ 1) * 32 + warp] = ni;
        }
        __syncthreads();
      }
      // rows back in logical order (pos of column T, an even count: buffer 0)
      for (int e = tid; e < P * T; e += blockDim.x) {
        const int r = e % P, cc = e / P;
        Cb[r + cc * ldp] = Pan[pos[r] + cc * ldp];
      }
      __syncthreads();
      C* tmp = Pan;
      Pan = Cb;
      Cb = tmp;
    }
    // write back the panel (L multipliers and the packed diagonal block)
    for (int e = tid; e < P * T; e += blockDim.x) {
      const int q = (e / (T * T)), w = e % (T * T);
      const int r = w % T, c = w / T;
      C* tile = f.tiles + g.tile_index(K + q, K) * g.tile_elems;
      tile[w] = Pan[q * T + r + c * ldp];
    }
    {
      int16_t* pg = f.perm + (int64_t)K * Pmax;
      for (int r = tid; r < Pmax; r += blockDim.x) pg[r] = (int16_t)(r < P ? perm[r] : r);
    }
    // inverses of the unit-lower and upper diagonal blocks
    if (tid < T) {
      const int j = tid;
      for (int i = 0; i < T; ++i) Li[i + j * T] = cmk<C>(i == j ? R(1) : R(0), R(0));
      for (int i = j + 1; i < T; ++i) {
        C s = cmk<C>(0, 0);
        for (int k = j; k < i; ++k) cfma(s, Pan[i + k * ldp], Li[k + j * T]);
        Li[i + j * T] = cmk<C>(-s.x, -s.y);
      }
    } else if (tid >= 32 && tid < 32 + T) {
      const int j = tid - 32;
      for (int i = 0; i < T; ++i) Ui[i + j * T] = cmk<C>(0, 0);
      Ui[j + j * T] = crecip(Pan[j + j * ldp]);
      for (int i = j - 1; i >= 0; --i) {
        C s = cmk<C>(0, 0);
        for (int k = i + 1; k <= j; ++k) cfma(s, Pan[i + k * ldp], Ui[k + j * T]);
        const C ri = crecip(Pan[i + i * ldp]);
        Ui[i + j * T] = cmk<C>(-(s.x * ri.x - s.y * ri.y), -(s.x * ri.y + s.y * ri.x));
      }
    }
    __syncthreads();
    {
      C* li = f.inv + (int64_t)(2 * K) * g.tile_elems;
      C* ui = f.inv + (int64_t)(2 * K + 1) * g.tile_elems;
      for (int e = tid; e < T * T; e += blockDim.x) {
        li[e] = Li[e];
        ui[e] = Ui[e];
      }
    }
    // trailing block columns K+1 .. K+nbr: warp w owns columns w, w+8, w+16, w+24 of every block
    // column through the gather (rows in panel order), U(K, Jc) = Linv Cb[0:T], the rows below
    // (Cb[T:P] -= L U) and the scatter, so the warps need no barrier between them
    for (int jb = 1; jb <= nbr; ++jb) {
      const int Jc = K + jb;
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = warp + 8 * jj;
        for (int r = lane; r < P; r += 32) {
          const int sr = perm[r];
          const int q = sr / T, rr = sr % T;
          const C* tile = f.tiles + g.tile_index(K + q, Jc) * g.tile_elems;
          Cb[r + c * ldp] = tile[rr + c * T];
        }
      }
      __syncwarp();
      // top block: U(K, Jc) = Linv * Cb[0:T]
      C acc[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) acc[jj] = cmk<C>(0, 0);
      for (int k = 0; k < T; ++k) {
        const C a = Li[lane + k * T];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) cfma(acc[jj], a, Cb[k + (warp + 8 * jj) * ldp]);
      }
      __syncwarp();
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) Cb[lane + (warp + 8 * jj) * ldp] = acc[jj];
      __syncwarp();
      // rows below: Cb[T:P] -= L(panel rows T:P) * U(K, Jc)
      for (int q = 1; q <= nbb; ++q) {
        const int r = q * T + lane;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[jj] = Cb[r + (warp + 8 * jj) * ldp];
        for (int k = 0; k < T; ++k) {
          const C a = Pan[r + k * ldp];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) cfms(acc[jj], a, Cb[k + (warp + 8 * jj) * ldp]);
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) Cb[r + (warp + 8 * jj) * ldp] = acc[jj];
      }
      __syncwarp();
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = warp + 8 * jj;
        for (int r = lane; r < P; r += 32) {
          const int q = r / T, rr = r % T;
          C* tile = f.tiles + g.tile_index(K + q, Jc) * g.tile_elems;
          tile[rr + c * T] = Cb[r + c * ldp];
        }
      }
      __syncwarp();
    }
    __syncthreads();  // block column K+1 (the next panel) and the tiles below are written
  }
  if (tid == 0) status[sidx] = sh_status;
}

// ---------------------------------------------------------------------------
// solve helpers.  A solve block covers CW right-hand sides with 8 warps: lane
// = row of a tile, warp w owns columns w + 8 jj, jj < NJ = CW / 8.
// ---------------------------------------------------------------------------
// Load one T x T tile into Tb (ld kLdt); conjugate-transposed if CT.
template <typename C, bool CT>
__device__ __forceinline__ void load_tile(C* Tb, const C* __restrict__ src) {
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int r = e % kTile, c = e / kTile;
    const C v = src[e];
    if (CT)
      Tb[c + r * kLdt] = cconj(v);
    else
      Tb[r + c * kLdt] = v;
  }
}

// acc[jj] += / -= Tb(lane, :) * Bm(:, col_jj), Bm with leading dimension ldb.
template <typename C, int NJ, bool SUB>
__device__ __forceinline__ void tile_mul(C acc[NJ], const C* Tb, const C* Bm, int ldb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 8
  for (int k = 0; k < kTile; ++k) {
    const C a = Tb[lane + k * kLdt];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const C bv = Bm[k + (warp + 8 * jj) * ldb];
      if (SUB)
        cfms(acc[jj], a, bv);
      else
        cfma(acc[jj], a, bv);
    }
  }
}

template <typename C, int NJ>
__device__ __forceinline__ void load_rhs_block(C* dst, int ldd, const C* __restrict__ Y, int64_t n,
                                               int64_t row0, int col0, int ncols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const int c = warp + 8 * jj;
    const int64_t i = row0 + lane;
    C v = cmk<C>(0, 0);
    if (i < n && col0 + c < ncols) v = Y[i + (int64_t)(col0 + c) * n];
    dst[lane + c * ldd] = v;
  }
}

template <typename C, int NJ>
__device__ __forceinline__ void store_rows(C* __restrict__ X, int64_t n, int64_t row0, int col0,
                                           int ncols, const C acc[NJ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const int c = warp + 8 * jj;
    const int64_t i = row0 + lane;
    if (i < n && col0 + c < ncols) X[i + (int64_t)(col0 + c) * n] = acc[jj];
  }
}

template <typename C, int NJ>
__device__ __forceinline__ void load_acc(C acc[NJ], const C* __restrict__ X, int64_t n, int64_t row0,
                                         int col0, int ncols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const int c = warp + 8 * jj;
    const int64_t i = row0 + lane;
    acc[jj] = (i < n && col0 + c < ncols) ? X[i + (int64_t)(col0 + c) * n] : cmk<C>(0, 0);
  }
}

template <typename C, int NJ>
__device__ __forceinline__ void put_acc(C* dst, int ldd, const C acc[NJ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) dst[lane + (warp + 8 * jj) * ldd] = acc[jj];
}

template <typename C, int NJ>
__device__ __forceinline__ void get_acc(C acc[NJ], const C* src, int lds) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) acc[jj] = src[lane + (warp + 8 * jj) * lds];
}

template <typename C, int NJ>
__device__ __forceinline__ void zero_acc(C acc[NJ]) {
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) acc[jj] = cmk<C>(0, 0);
}

// ---------------------------------------------------------------------------
// Factor tiles reach shared memory through a two-slot cp.async pipeline: the
// tile of the next step is requested before the current one is used, so its
// L2/HBM latency overlaps the current tile product.  Tiles keep their stored
// layout (element (r, c) at r + c kLdt); conjugate-transposed use reads them
// transposed (tile_mul_ct).
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void cp_async_tile(C* dst, const C* __restrict__ src) {
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int r = e % kTile, c = e / kTile;
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + r + c * kLdt);
    if constexpr (sizeof(C) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + e));
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + e));
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

// acc[jj] += / -= Tc(:, lane)^H-row times Bm: a = conj(Traw(k, lane))
template <typename C, int NJ, bool SUB>
__device__ __forceinline__ void tile_mul_ct(C acc[NJ], const C* Traw, const C* Bm, int ldb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 8
  for (int k = 0; k < kTile; ++k) {
    const C a = cconj(Traw[k + lane * kLdt]);
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const C bv = Bm[k + (warp + 8 * jj) * ldb];
      if (SUB)
        cfms(acc[jj], a, bv);
      else
        cfma(acc[jj], a, bv);
    }
  }
}

// Ordered tile requests of one sweep.  next() returns the source of the
// following request (nullptr after the last); acquire() starts the request
// after the current one, waits for the current one and returns its slot.
template <typename C>
struct TilePipe {
  C* slot[2];
  int cur = 0;
  const C* pending = nullptr;  // source of the request issued into slot[cur ^ 1]
  __device__ void start(const C* first, const C* second) {
    cur = 0;
    cp_async_tile(slot[0], first);
    pending = second;
    if (second) cp_async_tile(slot[1], second);
  }
  // current tile is ready on return; `after_next` is the request after the pending one
  __device__ C* acquire() {
    if (pending)
      asm volatile("cp.async.wait_group 1;\n" ::);
    else
      asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    return slot[cur];
  }
  // the current slot is free again (every thread is past its use): refill it
  __device__ void release(const C* after_next) {
    __syncthreads();
    cur ^= 1;
    const C* next = after_next;
    if (pending && next) cp_async_tile(slot[cur ^ 1], next);
    pending = pending ? next : nullptr;
  }
};

// Iterators over the tile requests of each sweep (same order as the sweeps).
struct SweepIt {
  int K, q;
};

// ---------------------------------------------------------------------------
// trans = 0: forward (P, L) then backward (U), for columns col0 .. col0+CW-1
// ---------------------------------------------------------------------------
template <typename C, int CW>
__device__ void solve_n_body(const FactorGeom& g, const SysDesc& d, int col0, const char* arena, const C* rhs,
                             C* out, char* smem) {
  constexpr int NJ = CW / 8;
  const int T = kTile, bt = g.bt;
  const int Pmax = (bt + 1) * T;
  const int ldw = Pmax;
  const FactorPtr<C> f = factor_ptr<C>(g, (char*)arena + d.factor_off);
  const C* Y = rhs + d.rhs_off;
  C* X = out + d.out_off;
  const int64_t n = g.n;
  const int ncols = d.ncols;
  const int tid = threadIdx.x;
  const int Nb = g.Nb;

  TilePipe<C> pipe;
  pipe.slot[0] = (C*)smem;                     // T x kLdt
  pipe.slot[1] = pipe.slot[0] + T * kLdt;      // T x kLdt
  C* tS = pipe.slot[1] + T * kLdt;             // T x CW
  C* U0 = tS + T * CW;                         // union area
  C* Wn = U0;                                  // Pmax x CW
  C* G = U0 + (size_t)Pmax * CW;               // Pmax x CW
  C* xwin = U0;                                // 2bt slots of T x CW

  // forward requests: per K, Linv(K) then L(K+q, K), q = 1..min(bt, Nb-1-K)
  auto fsrc = [&](SweepIt it) -> const C* {
    if (it.K >= Nb) return nullptr;
    return it.q == 0 ? f.inv + (int64_t)(2 * it.K) * g.tile_elems
                     : f.tiles + g.tile_index(it.K + it.q, it.K) * g.tile_elems;
  };
  auto fnext = [&](SweepIt it) -> SweepIt {
    if (it.q < min(bt, Nb - 1 - it.K)) return SweepIt{it.K, it.q + 1};
    return SweepIt{it.K + 1, 0};
  };
  // ---------------- forward ----------------
  {
    SweepIt it0{0, 0};
    SweepIt it1 = fnext(it0);
    SweepIt it2 = fnext(it1);
    pipe.start(fsrc(it0), fsrc(it1));
    const int nbb0 = min(bt, Nb - 1);
    for (int q = 0; q <= nbb0; ++q) load_rhs_block<C, NJ>(Wn + q * T, ldw, Y, n, (int64_t)q * T, col0, ncols);
    __syncthreads();
    for (int K = 0; K < Nb; ++K) {
      const int nbb = min(bt, Nb - 1 - K);
      const int P = (nbb + 1) * T;
      const int16_t* pm = f.perm + (int64_t)K * Pmax;
      for (int e = tid; e < P * CW; e += blockDim.x) {
        const int r = e % P, c = e / P;
        G[r + c * ldw] = Wn[pm[r] + c * ldw];
      }
      C* Tb = pipe.acquire();
      C acc[NJ];
      zero_acc<C, NJ>(acc);
      tile_mul<C, NJ, false>(acc, Tb, G, ldw);
      pipe.release(fsrc(it2));
      it2 = fnext(it2);
      put_acc<C, NJ>(G, ldw, acc);
      store_rows<C, NJ>(X, n, (int64_t)K * T, col0, ncols, acc);
      __syncthreads();
      for (int q = 1; q <= nbb; ++q) {
        Tb = pipe.acquire();
        get_acc<C, NJ>(acc, G + q * T, ldw);
        tile_mul<C, NJ, true>(acc, Tb, G, ldw);
        put_acc<C, NJ>(G + q * T, ldw, acc);
        pipe.release(fsrc(it2));
        it2 = fnext(it2);
      }
      if (K + 1 < Nb) {
        for (int e = tid; e < nbb * T * CW; e += blockDim.x) {
          const int r = e % (nbb * T), c = e / (nbb * T);
          Wn[r + c * ldw] = G[T + r + c * ldw];
        }
        const int nbn = min(bt, Nb - 2 - K);
        if (nbn == nbb)
          load_rhs_block<C, NJ>(Wn + nbb * T, ldw, Y, n, (int64_t)(K + bt + 1) * T, col0, ncols);
        __syncthreads();
      }
    }
  }
  // backward requests: per K (descending), U(K, K+q), q = 1..min(2bt, Nb-1-K), then Uinv(K)
  auto bsrc = [&](SweepIt it) -> const C* {
    if (it.K < 0) return nullptr;
    return it.q > 0 ? f.tiles + g.tile_index(it.K, it.K + it.q) * g.tile_elems
                    : f.inv + (int64_t)(2 * it.K + 1) * g.tile_elems;
  };
  auto bfirst = [&](int K) -> SweepIt { return SweepIt{K, min(2 * bt, Nb - 1 - K) > 0 ? 1 : 0}; };
  auto bnext = [&](SweepIt it) -> SweepIt {
    if (it.q > 0 && it.q < min(2 * bt, Nb - 1 - it.K)) return SweepIt{it.K, it.q + 1};
    if (it.q > 0) return SweepIt{it.K, 0};
    return it.K - 1 >= 0 ? bfirst(it.K - 1) : SweepIt{-1, 0};
  };
  // ---------------- backward ----------------
  {
    const int ns = 2 * bt;
    SweepIt it0 = bfirst(Nb - 1);
    SweepIt it1 = bnext(it0);
    SweepIt it2 = bnext(it1);
    pipe.start(bsrc(it0), bsrc(it1));
    for (int K = Nb - 1; K >= 0; --K) {
      const int nbr = min(2 * bt, Nb - 1 - K);
      C acc[NJ];
      load_acc<C, NJ>(acc, X, n, (int64_t)K * T, col0, ncols);
      for (int q = 1; q <= nbr; ++q) {
        C* Tb = pipe.acquire();
        tile_mul<C, NJ, true>(acc, Tb, xwin + ((K + q) % ns) * T * CW, T);
        pipe.release(bsrc(it2));
        it2 = bnext(it2);
      }
      put_acc<C, NJ>(tS, T, acc);
      C* Tb = pipe.acquire();
      zero_acc<C, NJ>(acc);
      tile_mul<C, NJ, false>(acc, Tb, tS, T);
      put_acc<C, NJ>(xwin + (K % ns) * T * CW, T, acc);
      store_rows<C, NJ>(X, n, (int64_t)K * T, col0, ncols, acc);
      pipe.release(bsrc(it2));
      it2 = bnext(it2);
    }
  }
}

// ---------------------------------------------------------------------------
// trans = 1: forward U^H, backward L^H then P^T
// ---------------------------------------------------------------------------
template <typename C, int CW>
__device__ void solve_c_body(const FactorGeom& g, const SysDesc& d, int col0, const char* arena, const C* rhs,
                             C* out, char* smem) {
  constexpr int NJ = CW / 8;
  const int T = kTile, bt = g.bt;
  const int Pmax = (bt + 1) * T;
  const int ldw = Pmax;
  const FactorPtr<C> f = factor_ptr<C>(g, (char*)arena + d.factor_off);
  const C* Y = rhs + d.rhs_off;
  C* X = out + d.out2_off;
  const int64_t n = g.n;
  const int ncols = d.ncols;
  const int tid = threadIdx.x;
  const int Nb = g.Nb;

  TilePipe<C> pipe;
  pipe.slot[0] = (C*)smem;
  pipe.slot[1] = pipe.slot[0] + T * kLdt;
  C* tS = pipe.slot[1] + T * kLdt;
  C* U0 = tS + T * CW;
  C* wwin = U0;                        // 2bt slots of T x CW
  C* V = U0;                           // Pmax x CW
  C* Vn = U0 + (size_t)Pmax * CW;      // Pmax x CW

  // forward requests: per K, U(K-q, K), q = 1..min(2bt, K), then Uinv(K)
  auto fsrc = [&](SweepIt it) -> const C* {
    if (it.K >= Nb) return nullptr;
    return it.q > 0 ? f.tiles + g.tile_index(it.K - it.q, it.K) * g.tile_elems
                    : f.inv + (int64_t)(2 * it.K + 1) * g.tile_elems;
  };
  auto ffirst = [&](int K) -> SweepIt { return SweepIt{K, min(2 * bt, K) > 0 ? 1 : 0}; };
  auto fnext = [&](SweepIt it) -> SweepIt {
    if (it.q > 0 && it.q < min(2 * bt, it.K)) return SweepIt{it.K, it.q + 1};
    if (it.q > 0) return SweepIt{it.K, 0};
    return ffirst(it.K + 1);
  };
  // ---------------- forward: U^H w = y ----------------
  {
    const int ns = 2 * bt;
    SweepIt it0 = ffirst(0);
    SweepIt it1 = fnext(it0);
    SweepIt it2 = fnext(it1);
    pipe.start(fsrc(it0), fsrc(it1));
    for (int K = 0; K < Nb; ++K) {
      C acc[NJ];
      load_acc<C, NJ>(acc, Y, n, (int64_t)K * T, col0, ncols);
      const int nq = min(2 * bt, K);
      for (int q = 1; q <= nq; ++q) {
        C* Tb = pipe.acquire();
        tile_mul_ct<C, NJ, true>(acc, Tb, wwin + ((K - q) % ns) * T * CW, T);
        pipe.release(fsrc(it2));
        it2 = fnext(it2);
      }
      put_acc<C, NJ>(tS, T, acc);
      C* Tb = pipe.acquire();
      zero_acc<C, NJ>(acc);
      tile_mul_ct<C, NJ, false>(acc, Tb, tS, T);
      put_acc<C, NJ>(wwin + (K % ns) * T * CW, T, acc);
      store_rows<C, NJ>(X, n, (int64_t)K * T, col0, ncols, acc);
      pipe.release(fsrc(it2));
      it2 = fnext(it2);
    }
  }
  // backward requests: per K (descending), L(K+q, K), q = 1..min(bt, Nb-1-K), then Linv(K)
  auto bsrc = [&](SweepIt it) -> const C* {
    if (it.K < 0) return nullptr;
    return it.q > 0 ? f.tiles + g.tile_index(it.K + it.q, it.K) * g.tile_elems
                    : f.inv + (int64_t)(2 * it.K) * g.tile_elems;
  };
  auto bfirst = [&](int K) -> SweepIt { return SweepIt{K, min(bt, Nb - 1 - K) > 0 ? 1 : 0}; };
  auto bnext = [&](SweepIt it) -> SweepIt {
    if (it.q > 0 && it.q < min(bt, Nb - 1 - it.K)) return SweepIt{it.K, it.q + 1};
    if (it.q > 0) return SweepIt{it.K, 0};
    return it.K - 1 >= 0 ? bfirst(it.K - 1) : SweepIt{-1, 0};
  };
  // ---------------- backward: x = P_0^T E_0^H ... P_{Nb-1}^T E_{Nb-1}^H w ----------------
  {
    SweepIt it0 = bfirst(Nb - 1);
    SweepIt it1 = bnext(it0);
    SweepIt it2 = bnext(it1);
    pipe.start(bsrc(it0), bsrc(it1));
    for (int K = Nb - 1; K >= 0; --K) {
      const int nbb = min(bt, Nb - 1 - K);
      const int P = (nbb + 1) * T;
      C acc[NJ];
      load_acc<C, NJ>(acc, X, n, (int64_t)K * T, col0, ncols);
      for (int q = 1; q <= nbb; ++q) {
        C* Tb = pipe.acquire();
        tile_mul_ct<C, NJ, true>(acc, Tb, V + q * T, ldw);
        pipe.release(bsrc(it2));
        it2 = bnext(it2);
      }
      put_acc<C, NJ>(tS, T, acc);
      C* Tb = pipe.acquire();
      zero_acc<C, NJ>(acc);
      tile_mul_ct<C, NJ, false>(acc, Tb, tS, T);
      pipe.release(bsrc(it2));
      it2 = bnext(it2);
      put_acc<C, NJ>(V, ldw, acc);
      __syncthreads();
      const int16_t* pm = f.perm + (int64_t)K * Pmax;
      for (int e = tid; e < P * CW; e += blockDim.x) {
        const int r = e % P, c = e / P;
        Vn[pm[r] + c * ldw] = V[r + c * ldw];
      }
      __syncthreads();
      if (nbb == bt) {
        // block K+bt is final
#pragma unroll
        for (int jj = 0; jj < NJ; ++jj) acc[jj] = Vn[bt * T + (tid & 31) + ((tid >> 5) + 8 * jj) * ldw];
        store_rows<C, NJ>(X, n, (int64_t)(K + bt) * T, col0, ncols, acc);
      }
      const int nbn = min(bt, Nb - K);  // window blocks kept for step K-1 (beyond its top block)
      for (int e = tid; e < nbn * T * CW; e += blockDim.x) {
        const int r = e % (nbn * T), c = e / (nbn * T);
        V[T + r + c * ldw] = Vn[r + c * ldw];
      }
      __syncthreads();
    }
    // remaining window blocks 0 .. min(bt, Nb)-1 sit in V[T : ...]
    const int nrem = min(bt, Nb);
    for (int q = 0; q < nrem; ++q) {
      C acc[NJ];
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) acc[jj] = V[T + q * T + (tid & 31) + ((tid >> 5) + 8 * jj) * ldw];
      store_rows<C, NJ>(X, n, (int64_t)q * T, col0, ncols, acc);
    }
  }
}

// Persistent solve: the grid holds as many blocks as fit on the GPU at once;
// each block takes (system, column block) items from a shared counter until
// the list is exhausted, so systems of uneven m0 keep every SM busy.
template <typename C, int CW, int TRANS>
__global__ void __launch_bounds__(kThreads) solve_kernel(FactorGeom g, const SysDesc* sys, const char* arena,
                                                        const C* rhs, C* out, const int2* items, int nitems,
                                                        int* counter) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int sh_item;
  for (;;) {
    if (threadIdx.x == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    __syncthreads();  // every thread has its item before thread 0 fetches the next one
    if (item >= nitems) return;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    if (TRANS == 0)
      solve_n_body<C, CW>(g, d, w.y, arena, rhs, out, smem);
    else
      solve_c_body<C, CW>(g, d, w.y, arena, rhs, out, smem);
    __syncthreads();
  }
}

size_t solve_smem_bytes(const FactorGeom& g, int chunk, size_t es, int trans) {
  (void)trans;
  const int T = kTile;
  const size_t Pmax = (size_t)(g.bt + 1) * T;
  size_t uni = 2 * Pmax * (size_t)chunk;
  size_t win = (size_t)2 * g.bt * T * chunk;
  if (win > uni) uni = win;
  return es * ((size_t)2 * T * kLdt + (size_t)T * chunk + uni);  // two tile slots
}

static size_t factor_smem_bytes(const FactorGeom& g, size_t es) {
  const int T = kTile;
  const size_t Pmax = (size_t)(g.bt + 1) * T;
  return es * (2 * (Pmax + 1) * T + 2 * (size_t)T * T) + sizeof(int) * 3 * Pmax;
}

template <typename C>
int launch_factor(const FactorGeom& g, int cplx, const void* band, int64_t ldab, int nsys,
                  const SysDesc* d_sys, char* factor_arena, int* d_status, int32_t* d_ipiv,
                  cudaStream_t st) {
  if (nsys <= 0) return 0;
  dim3 gi((unsigned)(g.tiles < 4096 ? g.tiles : 4096), (unsigned)nsys);
  init_factor_kernel<C><<<gi, kThreads, 0, st>>>(g, cplx, (const double*)band, ldab, d_sys, factor_arena);
  PD_CK_LAUNCH();
  const size_t smem = factor_smem_bytes(g, sizeof(C));
  if (smem > 227 * 1024) {
    set_last_error_msg("band too wide for the factor kernel's shared memory");
    return PDESHEP_CUDA_ERROR;
  }
  PD_CK(cudaFuncSetAttribute(factor_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  factor_kernel<C><<<nsys, kThreads, smem, st>>>(g, d_sys, factor_arena, d_status, d_ipiv);
  PD_CK_LAUNCH();
  return 0;
}

// Scratch of the solve work queue for nsys systems of at most max_cols
// right-hand sides (enough for the narrowest column block, 16).
size_t solve_queue_bytes(int nsys, int max_cols) {
  Arena a;
  a.take<int>(1);
  a.take<int2>((size_t)nsys * ceil_div(max_cols, 16));
  return a.used();
}

// Work list of (system, first column) items of `chunk` right-hand sides into
// the queue scratch (counter first, then the items).  Returns the item count.
int upload_solve_items(int nsys, const SysDesc* h_sys, int chunk, void* queue, cudaStream_t st, int* nitems) {
  if (chunk == kTcChunk) chunk = kTmChunk;  // the tensor-core solve also takes 128 right-hand sides per item
  std::vector<int2> it;
  for (int s = 0; s < nsys; ++s)
    for (int c = 0; c < h_sys[s].ncols; c += chunk) it.push_back(make_int2(s, c));
  *nitems = (int)it.size();
  if (it.empty()) return 0;
  Arena qa(queue, ~size_t(0));
  qa.take<int>(1);
  int2* d_items = qa.take<int2>(it.size());
  PD_CK(cudaMemcpyAsync(d_items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice, st));
  return 0;
}

template <typename C, int CW, int TRANS>
static int launch_solve_cw(const FactorGeom& g, int nitems, const SysDesc* d_sys, const char* factor_arena,
                           const C* rhs_arena, C* out_arena, void* queue, cudaStream_t st) {
  const size_t smem = solve_smem_bytes(g, CW, sizeof(C), TRANS);
  if (smem > 227 * 1024) {
    set_last_error_msg("band too wide for the solve kernel's shared memory at this column block");
    return PDESHEP_CUDA_ERROR;
  }
  if (!nitems) return 0;
  Arena qa(queue, ~size_t(0));
  int* counter = qa.take<int>(1);
  const int2* d_items = qa.take<int2>((size_t)nitems);
  auto kern = solve_kernel<C, CW, TRANS>;
  PD_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, dev = 0, sms = 0;
  PD_CK(cudaGetDevice(&dev));
  PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  const int grid = std::max(1, std::min(nitems, sms * std::max(1, per_sm)));
  PD_CK(cudaMemsetAsync(counter, 0, sizeof(int), st));
  kern<<<grid, kThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems, counter);
  PD_CK_LAUNCH();
  return 0;
}

template <typename C>
int launch_solve_queued(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                        const C* rhs_arena, C* out_arena, int chunk, void* queue, cudaStream_t st) {
  if (chunk == kTmChunk || chunk == kTcChunk) {
    if constexpr (std::is_same<C, float2>::value) {
      if (chunk == kTcChunk)
        return launch_solve_tc(g, trans, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
      return launch_solve_tm(g, trans, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    }
    set_last_error_msg("the tensor-memory and tensor-core solves are complex64 only");
    return PDESHEP_CUDA_ERROR;
  }
  switch (chunk * 2 + (trans ? 1 : 0)) {
    case 32: return launch_solve_cw<C, 16, 0>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    case 33: return launch_solve_cw<C, 16, 1>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    case 64: return launch_solve_cw<C, 32, 0>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    case 65: return launch_solve_cw<C, 32, 1>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    case 128: return launch_solve_cw<C, 64, 0>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    case 129: return launch_solve_cw<C, 64, 1>(g, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st);
    default:
      set_last_error_msg("right-hand-side block width must be 16, 32 or 64");
      return PDESHEP_CUDA_ERROR;
  }
}

template <typename C>
int launch_solve(const FactorGeom& g, int trans, int nsys, const SysDesc* h_sys, const SysDesc* d_sys,
                 const char* factor_arena, const C* rhs_arena, C* out_arena, int chunk, void* queue,
                 cudaStream_t st) {
  if (nsys <= 0) return 0;
  if (chunk <= 0) chunk = 32;
  if (chunk != 16 && chunk != 32 && chunk != 64 && chunk != kTmChunk && chunk != kTcChunk) {
    set_last_error_msg("right-hand-side block width must be 16, 32, 64, 128 or 256");
    return PDESHEP_CUDA_ERROR;
  }
  int nitems = 0;
  PD_TRY(upload_solve_items(nsys, h_sys, chunk, queue, st, &nitems));
  return launch_solve_queued<C>(g, trans, nitems, d_sys, factor_arena, rhs_arena, out_arena, chunk, queue, st);
}

template int launch_factor<float2>(const FactorGeom&, int, const void*, int64_t, int, const SysDesc*,
                                   char*, int*, int32_t*, cudaStream_t);
template int launch_factor<double2>(const FactorGeom&, int, const void*, int64_t, int, const SysDesc*,
                                    char*, int*, int32_t*, cudaStream_t);
template int launch_solve_queued<float2>(const FactorGeom&, int, int, const SysDesc*, const char*, const float2*,
                                         float2*, int, void*, cudaStream_t);
template int launch_solve_queued<double2>(const FactorGeom&, int, int, const SysDesc*, const char*, const double2*,
                                          double2*, int, void*, cudaStream_t);
template int launch_solve<float2>(const FactorGeom&, int, int, const SysDesc*, const SysDesc*, const char*,
                                  const float2*, float2*, int, void*, cudaStream_t);
template int launch_solve<double2>(const FactorGeom&, int, int, const SysDesc*, const SysDesc*, const char*,
                                   const double2*, double2*, int, void*, cudaStream_t);

}  // namespace pdeshep
