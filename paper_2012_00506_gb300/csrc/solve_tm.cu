// solve_tm.cu -- complex64 multi-right-hand-side band solves of eq. (10) with
// the sweep window held in tensor memory.
//
// Same factor layout and the same arithmetic as the solves of band_lu.cu
// (every entry is the same sequence of FP32 FMAs: tile products accumulate
// over the tile's columns in ascending order), organised for GB300:
//   * a CTA of 256 threads takes 128 right-hand sides of one system.  TMEM lane
//     l is right-hand side l; the warps w and w+4 share lane quadrant w, and
//     of every block of 32 complex rows warp w (< 4) owns rows 0..15, warp
//     w+4 rows 16..31.  The window of partly eliminated rows (forward
//     sweeps) or of solved blocks (backward sweeps) -- up to 8 blocks, 512
//     TMEM columns at b = 128 -- never touches shared memory;
//   * a tile product is 16 x 32 complex multiply-adds per thread with the
//     factor tile read by broadcast from shared memory; the 32-row vector it
//     multiplies is either a block read whole from TMEM (backward sweeps) or
//     assembled by the two threads of a right-hand side in one shared row
//     (forward sweeps), with a barrier of those two warps;
//   * the only CTA-wide barrier of a step is the arrival of its tiles, which
//     are copied in one step ahead (cp.async, two buffers);
//   * the row interchanges of a panel (forward sweep) and their inverse
//     (adjoint backward sweep) move at most 64 rows: the old top block passes
//     through a shared row per right-hand side, the other rows are read and
//     written in place in TMEM.
// Block J of a window sits in TMEM columns [64 s, 64 s + 64), s = J mod
// (ring size): the 32 real parts, then the 32 imaginary parts.
#include <algorithm>

#include "band_lu.cuh"

namespace pdeshep {
namespace {

constexpr int kTmThreads = 256;
constexpr int kTmCols = 128;  // right-hand sides per CTA (TMEM lanes)
constexpr int kSRow = 65;     // floats per shared row (conflict-free)

// ---------------------------------------------------------------------------
// tcgen05 tensor-memory access (a warp reaches the 32 lanes of its quadrant)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tm_ld16(uint32_t a, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
}
__device__ __forceinline__ void tm_st16(uint32_t a, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16};" ::"r"(a),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ uint32_t tm_ld1(uint32_t a) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(a));
  return r;
}
__device__ __forceinline__ void tm_st1(uint32_t a, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// after a wait::ld: the registers pass through an empty asm so that no use moves above the wait
__device__ __forceinline__ void reg_fence16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}
// a barrier that also orders TMEM accesses of the threads it joins
__device__ __forceinline__ void tm_bar(int id, int nthreads) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// half a block (16 complex rows) and a whole block of this thread's right-hand side
struct Half {
  float re[16], im[16];
};
struct Blk {
  float re[32], im[32];
};

__device__ __forceinline__ void half_zero(Half& b) {
#pragma unroll
  for (int r = 0; r < 16; ++r) b.re[r] = b.im[r] = 0.f;
}

// TMEM: this thread's half (rows 16h..16h+15) of the block at column `blk`
__device__ __forceinline__ void half_from_tm(Half& b, uint32_t tb, uint32_t blk, int h) {
  uint32_t vr[16], vi[16];
  tm_ld16(tb + blk + 16 * h, vr);
  tm_ld16(tb + blk + 32 + 16 * h, vi);
  tm_wait_ld();
  reg_fence16(vr);
  reg_fence16(vi);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    b.re[i] = __uint_as_float(vr[i]);
    b.im[i] = __uint_as_float(vi[i]);
  }
}
__device__ __forceinline__ void half_to_tm(const Half& b, uint32_t tb, uint32_t blk, int h) {
  uint32_t vr[16], vi[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    vr[i] = __float_as_uint(b.re[i]);
    vi[i] = __float_as_uint(b.im[i]);
  }
  tm_st16(tb + blk + 16 * h, vr);
  tm_st16(tb + blk + 32 + 16 * h, vi);
  tm_wait_st();
}
// the whole block (both halves)
__device__ __forceinline__ void blk_from_tm(Blk& b, uint32_t tb, uint32_t blk) {
  uint32_t v0[16], v1[16], v2[16], v3[16];
  tm_ld16(tb + blk, v0);
  tm_ld16(tb + blk + 16, v1);
  tm_ld16(tb + blk + 32, v2);
  tm_ld16(tb + blk + 48, v3);
  tm_wait_ld();
  reg_fence16(v0);
  reg_fence16(v1);
  reg_fence16(v2);
  reg_fence16(v3);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    b.re[i] = __uint_as_float(v0[i]);
    b.re[16 + i] = __uint_as_float(v1[i]);
    b.im[i] = __uint_as_float(v2[i]);
    b.im[16 + i] = __uint_as_float(v3[i]);
  }
}

// global rows row0+16h .. row0+16h+15 of this thread's right-hand side (zero past n)
__device__ __forceinline__ void half_from_global(Half& b, const float2* __restrict__ Y, int64_t n, int64_t row0,
                                                 bool valid) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    float2 v = make_float2(0.f, 0.f);
    if (valid && row0 + i < n) v = Y[row0 + i];
    b.re[i] = v.x;
    b.im[i] = v.y;
  }
}
__device__ __forceinline__ void half_to_global(const Half& b, float2* __restrict__ X, int64_t n, int64_t row0,
                                               bool valid) {
  if (!valid) return;
#pragma unroll
  for (int i = 0; i < 16; ++i)
    if (row0 + i < n) X[row0 + i] = make_float2(b.re[i], b.im[i]);
}
// this thread's half into the right-hand side's shared row (re at [0,32), im at [32,64))
__device__ __forceinline__ void half_to_row(const Half& b, float* row, int h) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    row[16 * h + i] = b.re[i];
    row[32 + 16 * h + i] = b.im[i];
  }
}

// acc (+/-)= M(rows 16h..16h+15, :) v, M a 32 x 32 complex tile in shared memory, accumulated over
// the tile's columns in ascending order.  CT = false: M(r, c) = T[r + 32 c] (the stored tile);
// CT = true: M(r, c) = conj(T[c + 32 r]).  v from a shared row (vs) or from registers (vb).
template <bool SUB, bool CT>
__device__ __forceinline__ void mac_col(Half& acc, const float2* __restrict__ T, int h, int c, float2 x) {
  if (!CT) {
    const float4* col = (const float4*)(T + 32 * c + 16 * h);
#pragma unroll
    for (int i2 = 0; i2 < 8; ++i2) {
      const float4 m = col[i2];
      float2 a0 = make_float2(acc.re[2 * i2], acc.im[2 * i2]);
      float2 a1 = make_float2(acc.re[2 * i2 + 1], acc.im[2 * i2 + 1]);
      if (SUB) {
        cfms(a0, make_float2(m.x, m.y), x);
        cfms(a1, make_float2(m.z, m.w), x);
      } else {
        cfma(a0, make_float2(m.x, m.y), x);
        cfma(a1, make_float2(m.z, m.w), x);
      }
      acc.re[2 * i2] = a0.x;
      acc.im[2 * i2] = a0.y;
      acc.re[2 * i2 + 1] = a1.x;
      acc.im[2 * i2 + 1] = a1.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float2 m = cconj(T[c + 32 * (16 * h + i)]);
      float2 a = make_float2(acc.re[i], acc.im[i]);
      if (SUB)
        cfms(a, m, x);
      else
        cfma(a, m, x);
      acc.re[i] = a.x;
      acc.im[i] = a.y;
    }
  }
}
template <bool SUB, bool CT>
__device__ __forceinline__ void tile_apply_s(Half& acc, const float2* __restrict__ T, int h,
                                             const float* __restrict__ vs) {
#pragma unroll 2
  for (int c = 0; c < 32; ++c) mac_col<SUB, CT>(acc, T, h, c, make_float2(vs[c], vs[32 + c]));
}
template <bool SUB, bool CT>
__device__ __forceinline__ void tile_apply_r(Half& acc, const float2* __restrict__ T, int h, const Blk& vb) {
#pragma unroll
  for (int c = 0; c < 32; ++c) mac_col<SUB, CT>(acc, T, h, c, make_float2(vb.re[c], vb.im[c]));
}

// ---------------------------------------------------------------------------
// steps: sweep 0 then sweep 1 of one work item; tiles of each step in use order
// ---------------------------------------------------------------------------
struct StepInfo {
  int sweep, K, ntiles;
};

template <int TRANS>
__device__ __forceinline__ StepInfo step_info(const FactorGeom& g, int s) {
  const int Nb = g.Nb, bt = g.bt;
  StepInfo st;
  st.sweep = s < Nb ? 0 : 1;
  st.K = st.sweep == 0 ? s : Nb - 1 - (s - Nb);
  const int K = st.K;
  if (TRANS == 0)
    st.ntiles = st.sweep == 0 ? 1 + min(bt, Nb - 1 - K) : 1 + min(2 * bt, Nb - 1 - K);
  else
    st.ntiles = st.sweep == 0 ? 1 + min(2 * bt, K) : 1 + min(bt, Nb - 1 - K);
  return st;
}

// source of tile i of step st (the order in which the step uses them)
template <int TRANS>
__device__ __forceinline__ const float2* tile_src(const FactorGeom& g, const FactorPtr<float2>& f, const StepInfo& st,
                                                  int i) {
  const int K = st.K;
  const int last = st.ntiles - 1;
  if (TRANS == 0) {
    if (st.sweep == 0)  // Linv(K), then L(K+q, K)
      return i == 0 ? f.inv + (int64_t)(2 * K) * g.tile_elems : f.tiles + g.tile_index(K + i, K) * g.tile_elems;
    // U(K, K+q) q = 1..nbr, then Uinv(K)
    return i < last ? f.tiles + g.tile_index(K, K + 1 + i) * g.tile_elems
                    : f.inv + (int64_t)(2 * K + 1) * g.tile_elems;
  }
  if (st.sweep == 0)  // U(K-q, K) q = 1..nq, then Uinv(K)
    return i < last ? f.tiles + g.tile_index(K - 1 - i, K) * g.tile_elems
                    : f.inv + (int64_t)(2 * K + 1) * g.tile_elems;
  // L(K+q, K) q = 1..nbb, then Linv(K)
  return i < last ? f.tiles + g.tile_index(K + 1 + i, K) * g.tile_elems : f.inv + (int64_t)(2 * K) * g.tile_elems;
}

// copy the tiles (and, for the interchange sweeps, the panel permutation) of step s into a buffer
template <int TRANS>
__device__ __forceinline__ void prefetch_step(const FactorGeom& g, const FactorPtr<float2>& f, int s, float2* tbuf,
                                              int16_t* pbuf) {
  const StepInfo st = step_info<TRANS>(g, s);
  for (int i = 0; i < st.ntiles; ++i) {
    const float2* src = tile_src<TRANS>(g, f, st, i);
    float2* dst = tbuf + i * 1024;
    for (int e = threadIdx.x; e < 512; e += blockDim.x) {  // 512 16-byte chunks per tile
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst + 2 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 2 * e));
    }
  }
  if ((TRANS == 0 && st.sweep == 0) || (TRANS == 1 && st.sweep == 1)) {
    const int Pmax = (g.bt + 1) * kTile;  // int16 entries, a multiple of 8
    const int16_t* src = f.perm + (int64_t)st.K * Pmax;
    for (int e = threadIdx.x; e < Pmax / 8; e += blockDim.x) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(pbuf + 8 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 8 * e));
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

struct WinCtx {
  uint32_t tb;
  int K, ring;
  // TMEM address of the real part of window row rho (block K + rho/32)
  __device__ __forceinline__ uint32_t addr(int rho) const {
    return tb + (uint32_t)(64 * ((K + rho / 32) % ring) + rho % 32);
  }
};

// Permute the window rows [0, P) of this thread's right-hand side: new row r = old row src(r),
// where src(r) is r, or a row of the old top block, or (r < 32) any row.  The old top block is in
// the shared row `old` (complete); the new top half is returned in `top`; the rows below that
// receive old top rows are written in TMEM by the thread owning them.  `src` is the gather map
// (forward: the panel permutation; adjoint backward: its inverse).
template <typename SrcF>
__device__ __forceinline__ void permute_window(Half& top, const float* old, SrcF src, int P, int h, const WinCtx& wc,
                                               int bar_id, int bar_n) {
  // the new top half: gathered before any row is overwritten
  uint32_t ur[16], ui[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int s = src(16 * h + i);
    ur[i] = ui[i] = 0u;
    if (s >= 32) {
      const uint32_t a = wc.addr(s);
      ur[i] = tm_ld1(a);
      ui[i] = tm_ld1(a + 32);
    }
  }
  tm_wait_ld();
  reg_fence16(ur);
  reg_fence16(ui);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int s = src(16 * h + i);
    if (s < 32) {
      top.re[i] = old[s];
      top.im[i] = old[32 + s];
    } else {
      top.re[i] = __uint_as_float(ur[i]);
      top.im[i] = __uint_as_float(ui[i]);
    }
  }
  tm_bar(bar_id, bar_n);  // every gather of both halves is done
  for (int r = 32 + 16 * h; r < P; r += 32) {
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int s = src(r + i);
      if (s < 32) {
        const uint32_t a = wc.addr(r + i);
        tm_st1(a, __float_as_uint(old[s]));
        tm_st1(a + 32, __float_as_uint(old[32 + s]));
      }
    }
  }
  tm_wait_st();
}

// ---------------------------------------------------------------------------
// the persistent kernel: CTAs take (system, 128-column block) items from a counter
// ---------------------------------------------------------------------------
template <int TRANS>
__global__ void __launch_bounds__(kTmThreads, 1)
    solve_tm_kernel(FactorGeom g, const SysDesc* sys, const char* arena, const float2* rhs, float2* out,
                    const int2* items, int nitems, int* counter, uint32_t tmem_cols, int max_tiles, int sweep0,
                    int sweep1) {
  extern __shared__ __align__(16) char smem[];
  const int Pmax = (g.bt + 1) * kTile;
  float2* tbuf0 = (float2*)smem;                               // 2 buffers of max_tiles tiles
  float2* tbuf1 = tbuf0 + (size_t)max_tiles * 1024;
  float* vrow = (float*)(tbuf1 + (size_t)max_tiles * 1024);    // kTmCols x kSRow
  float* orow = vrow + kTmCols * kSRow;                        // kTmCols x kSRow
  int16_t* pbuf0 = (int16_t*)(orow + kTmCols * kSRow);         // 2 x Pmax
  int16_t* pbuf1 = pbuf0 + Pmax;
  int* pinv = (int*)(pbuf1 + Pmax);                            // Pmax
  __shared__ uint32_t tslot;
  __shared__ int sh_item;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int q4 = warp & 3, h = warp >> 2;  // lane quadrant, row half
  const int ci = 32 * q4 + lane;           // right-hand side within the item
  const int pair_bar = 1 + q4;             // barrier of warps q4 and q4 + 4
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(&tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tm_bar(0, kTmThreads);
  const uint32_t tb = tslot + ((uint32_t)(32 * q4) << 16);
  float* myv = vrow + ci * kSRow;
  float* myo = orow + ci * kSRow;
  const int bt = g.bt, Nb = g.Nb;
  const int64_t n = g.n;
  const int nslot_w = bt + 1;  // window ring of the interchange sweeps
  const int nslot_s = 2 * bt;  // ring of solved blocks of the other sweeps
  auto blk_col = [&](int J, int ring) -> uint32_t { return (uint32_t)(64 * (J % ring)); };

  for (;;) {
    if (t == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    if (item >= nitems) break;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    const FactorPtr<float2> f = factor_ptr<float2>(g, (char*)arena + d.factor_off);
    const int col = w.y + ci;
    const bool valid = col < d.ncols;
    const float2* Y = rhs + d.rhs_off + (int64_t)(valid ? col : 0) * n;
    float2* X = out + (TRANS == 0 ? d.out_off : d.out2_off) + (int64_t)(valid ? col : 0) * n;
    const int s_begin = sweep0 * Nb, nsteps = sweep1 * Nb;  // the sweeps [sweep0, sweep1) of the item

    prefetch_step<TRANS>(g, f, s_begin, (s_begin & 1) ? tbuf1 : tbuf0, (s_begin & 1) ? pbuf1 : pbuf0);
    if (TRANS == 0 && sweep0 == 0) {  // the first window of the forward sweep: blocks 0 .. min(bt, Nb-1) of Y
      Half y;
      for (int q = 0; q <= min(bt, Nb - 1); ++q) {
        half_from_global(y, Y, n, (int64_t)q * kTile + 16 * h, valid);
        half_to_tm(y, tb, blk_col(q, nslot_w), h);
      }
    }
    for (int s = s_begin; s < nsteps; ++s) {
      float2* tbs = (s & 1) ? tbuf1 : tbuf0;
      int16_t* pb = (s & 1) ? pbuf1 : pbuf0;
      asm volatile("cp.async.wait_group 0;\n" ::);
      tm_bar(0, kTmThreads);  // step s's tiles are here; every thread is past step s-1
      if (s + 1 < nsteps) prefetch_step<TRANS>(g, f, s + 1, (s & 1) ? tbuf0 : tbuf1, (s & 1) ? pbuf0 : pbuf1);
      const StepInfo st = step_info<TRANS>(g, s);
      const int K = st.K;
      const int64_t hrow = (int64_t)K * kTile + 16 * h;  // first global row of this thread's half
      Half acc, x;
      if (TRANS == 0 && st.sweep == 0) {
        // ---- forward: P_K, then x_K = Linv_K (top block), then the L updates below ----
        const int nbb = st.ntiles - 1;
        const int P = (nbb + 1) * kTile;
        const uint32_t top = blk_col(K, nslot_w);
        half_from_tm(acc, tb, top, h);
        half_to_row(acc, myo, h);  // the old top block, by right-hand side
        tm_bar(pair_bar, 64);
        const WinCtx wc{tb, K, nslot_w};
        permute_window(x, myo, [&](int r) { return (int)pb[r]; }, P, h, wc, pair_bar, 64);
        half_to_row(x, myv, h);
        tm_bar(pair_bar, 64);  // the new top block is complete
        half_zero(acc);
        tile_apply_s<false, false>(acc, tbs, h, myv);  // x_K = Linv_K g
        tm_bar(pair_bar, 64);                          // both halves have read g
        half_to_row(acc, myv, h);
        half_to_global(acc, X, n, hrow, valid);
        tm_bar(pair_bar, 64);  // x_K is complete
        for (int q = 1; q <= nbb; ++q) {
          const uint32_t a = blk_col(K + q, nslot_w);
          half_from_tm(x, tb, a, h);
          tile_apply_s<true, false>(x, tbs + q * 1024, h, myv);  // rows of block K+q -= L(K+q, K) x_K
          half_to_tm(x, tb, a, h);
        }
        if (K + bt + 1 < Nb) {  // block K+bt+1 of Y enters the slot block K leaves
          half_from_global(x, Y, n, (int64_t)(K + bt + 1) * kTile + 16 * h, valid);
          half_to_tm(x, tb, top, h);
        }
      } else if (TRANS == 0) {
        // ---- backward: x_K = Uinv_K (w_K - sum_q U(K, K+q) x_{K+q}) ----
        const int nbr = st.ntiles - 1;
        half_from_global(acc, X, n, hrow, valid);  // w_K, written by this thread in the forward sweep
        Blk v;
        for (int q = 1; q <= nbr; ++q) {
          blk_from_tm(v, tb, blk_col(K + q, nslot_s));
          tile_apply_r<true, false>(acc, tbs + (q - 1) * 1024, h, v);
        }
        half_to_row(acc, myv, h);
        tm_bar(pair_bar, 64);
        half_zero(x);
        tile_apply_s<false, false>(x, tbs + nbr * 1024, h, myv);
        half_to_tm(x, tb, blk_col(K, nslot_s), h);
        half_to_global(x, X, n, hrow, valid);
      } else if (st.sweep == 0) {
        // ---- adjoint forward: w_K = Uinv_K^H (y_K - sum_q U(K-q, K)^H w_{K-q}) ----
        const int nq = st.ntiles - 1;
        half_from_global(acc, Y, n, hrow, valid);
        Blk v;
        for (int q = 1; q <= nq; ++q) {
          blk_from_tm(v, tb, blk_col(K - q, nslot_s));
          tile_apply_r<true, true>(acc, tbs + (q - 1) * 1024, h, v);
        }
        half_to_row(acc, myv, h);
        tm_bar(pair_bar, 64);
        half_zero(x);
        tile_apply_s<false, true>(x, tbs + nq * 1024, h, myv);
        half_to_tm(x, tb, blk_col(K, nslot_s), h);
        half_to_global(x, X, n, hrow, valid);
      } else {
        // ---- adjoint backward: v_K = Linv_K^H (w_K - sum_q L(K+q, K)^H v_{K+q}), then P_K^T ----
        const int nbb = st.ntiles - 1;
        const int P = (nbb + 1) * kTile;
        for (int r = t; r < P; r += blockDim.x) pinv[pb[r]] = r;  // P_K^T moves window row r to pm[r]
        half_from_global(acc, X, n, hrow, valid);                  // w_K from the adjoint forward sweep
        Blk v;
        for (int q = 1; q <= nbb; ++q) {
          blk_from_tm(v, tb, blk_col(K + q, nslot_w));
          tile_apply_r<true, true>(acc, tbs + (q - 1) * 1024, h, v);
        }
        half_to_row(acc, myv, h);
        tm_bar(pair_bar, 64);
        half_zero(x);
        tile_apply_s<false, true>(x, tbs + nbb * 1024, h, myv);
        half_to_row(x, myo, h);  // v_K: the old top block of the interchange
        tm_bar(0, kTmThreads);   // pinv and both halves of v_K are complete
        const WinCtx wc{tb, K, nslot_w};
        permute_window(acc, myo, [&](int r) { return pinv[r]; }, P, h, wc, pair_bar, 64);
        half_to_tm(acc, tb, blk_col(K, nslot_w), h);
        if (nbb == bt) {  // block K+bt is final
          half_from_tm(x, tb, blk_col(K + bt, nslot_w), h);
          half_to_global(x, X, n, (int64_t)(K + bt) * kTile + 16 * h, valid);
        }
        if (K == 0) {  // the blocks left in the window are final
          for (int J = 0; J < min(bt, Nb); ++J) {
            half_from_tm(x, tb, blk_col(J, nslot_w), h);
            half_to_global(x, X, n, (int64_t)J * kTile + 16 * h, valid);
          }
        }
      }
    }
    __syncthreads();
  }
  tm_bar(0, kTmThreads);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(tmem_cols));
}

}  // namespace

// Largest band the TMEM window holds: 2 bt blocks of 64 columns within 512.
bool solve_tm_supported(const FactorGeom& g) { return g.bt >= 1 && 2 * g.bt * 64 <= 512; }

size_t solve_tm_smem_bytes(const FactorGeom& g) {
  const int max_tiles = 2 * g.bt + 1;
  const int Pmax = (g.bt + 1) * kTile;
  size_t bytes = (size_t)2 * max_tiles * 1024 * sizeof(float2) + (size_t)2 * kTmCols * kSRow * sizeof(float) +
                 (size_t)2 * Pmax * sizeof(int16_t) + (size_t)Pmax * sizeof(int);
  // at least 116 KiB, so that one CTA (and its TMEM allocation) owns each SM
  return std::max(bytes, (size_t)116 * 1024);
}

int launch_solve_tm(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                    const float2* rhs_arena, float2* out_arena, void* queue, cudaStream_t st, int sweep0, int sweep1) {
  if (!nitems) return 0;
  if (!solve_tm_supported(g)) {
    set_last_error_msg("band too wide for the tensor-memory solve window");
    return PDESHEP_CUDA_ERROR;
  }
  const size_t smem = solve_tm_smem_bytes(g);
  const int max_tiles = 2 * g.bt + 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(64 * std::max(2 * g.bt, g.bt + 1))) cols *= 2;
  Arena qa(queue, ~size_t(0));
  int* counter = qa.take<int>(1);
  const int2* d_items = qa.take<int2>((size_t)nitems);
  int dev = 0, sms = 0;
  PD_CK(cudaGetDevice(&dev));
  PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(nitems, sms));
  PD_CK(cudaMemsetAsync(counter, 0, sizeof(int), st));
  if (trans) {
    PD_CK(cudaFuncSetAttribute(solve_tm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_tm_kernel<1><<<grid, kTmThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                       counter, cols, max_tiles, sweep0, sweep1);
  } else {
    PD_CK(cudaFuncSetAttribute(solve_tm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_tm_kernel<0><<<grid, kTmThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                       counter, cols, max_tiles, sweep0, sweep1);
  }
  PD_CK_LAUNCH();
  return 0;
}

}  // namespace pdeshep
