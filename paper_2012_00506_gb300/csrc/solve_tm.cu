// solve_tm.cu -- complex64 multi-right-hand-side band solves of eq. (10) with
// one thread per right-hand side and the sweep window held in tensor memory.
//
// Same factor layout and the same arithmetic as the solves of band_lu.cu
// (every entry is the same sequence of FP32 FMAs: tile products accumulate
// over the tile's columns in ascending order), organised for GB300:
//   * a CTA of 128 threads takes 128 right-hand sides of one system; thread t
//     owns column t and TMEM lane t, so the window of partly eliminated rows
//     (forward sweeps) or of solved blocks (backward sweeps) -- up to 8 blocks
//     of 32 complex rows, 512 TMEM columns at b = 128 -- is private to its
//     thread and never touches shared memory;
//   * a tile product is 32 x 32 complex multiply-adds per thread with the
//     factor tile read by broadcast from shared memory (two tile entries per
//     16-byte load in the normal sweeps), so the only CTA-wide barrier of a
//     step is the arrival of the next step's tiles, which are copied in ahead
//     (cp.async, two buffers);
//   * the row interchanges of a panel (forward sweep) and their inverse
//     (adjoint backward sweep) move at most 64 rows: the top block passes
//     through a per-thread row of shared memory, the other rows are read and
//     written in place in TMEM.
// Row block J of the window sits in TMEM columns [64 s, 64 s + 64) with
// s = J mod (ring size): the 32 real parts, then the 32 imaginary parts.
#include <algorithm>

#include "band_lu.cuh"

namespace pdeshep {
namespace {

constexpr int kTmThreads = 128;
constexpr int kSRow = 65;  // floats per thread row of the vector scratch (conflict-free)

// ---------------------------------------------------------------------------
// tcgen05 tensor-memory access (32 lanes x 32-bit per warp; lane = thread)
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
__device__ __forceinline__ void reg_fence1(uint32_t& r) { asm volatile("" : "+r"(r)); }

// A block of 32 complex rows of this thread's column in registers.
struct Blk {
  float re[32], im[32];
};

__device__ __forceinline__ void blk_zero(Blk& b) {
#pragma unroll
  for (int r = 0; r < 32; ++r) b.re[r] = b.im[r] = 0.f;
}

// TMEM block <-> registers
__device__ __forceinline__ void blk_from_tm(Blk& b, uint32_t taddr) {
  uint32_t v[16];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    tm_ld16(taddr + 16 * h, v);
    tm_wait_ld();
    reg_fence16(v);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = 16 * h + i;
      if (c < 32)
        b.re[c] = __uint_as_float(v[i]);
      else
        b.im[c - 32] = __uint_as_float(v[i]);
    }
  }
}
__device__ __forceinline__ void blk_to_tm(const Blk& b, uint32_t taddr) {
  uint32_t v[16];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int c = 16 * h + i;
      v[i] = __float_as_uint(c < 32 ? b.re[c] : b.im[c - 32]);
    }
    tm_st16(taddr + 16 * h, v);
  }
  tm_wait_st();
}

// global column block rows row0..row0+31 (zero past n) <-> registers
__device__ __forceinline__ void blk_from_global(Blk& b, const float2* __restrict__ Y, int64_t n, int64_t row0,
                                                bool valid) {
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float2 v = make_float2(0.f, 0.f);
    if (valid && row0 + r < n) v = Y[row0 + r];
    b.re[r] = v.x;
    b.im[r] = v.y;
  }
}
__device__ __forceinline__ void blk_to_global(const Blk& b, float2* __restrict__ X, int64_t n, int64_t row0,
                                              bool valid) {
  if (!valid) return;
#pragma unroll
  for (int r = 0; r < 32; ++r)
    if (row0 + r < n) X[row0 + r] = make_float2(b.re[r], b.im[r]);
}

// this thread's vector row of the scratch <-> registers
__device__ __forceinline__ void blk_to_row(const Blk& b, float* row) {
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    row[r] = b.re[r];
    row[32 + r] = b.im[r];
  }
}

// acc (+/-)= M v, M a 32 x 32 complex tile in shared memory, v the thread's vector row
// (re at [0,32), im at [32,64)), accumulated over the tile's columns in ascending order.
// CT = false: M(r, c) = T[r + 32 c] (the stored tile); CT = true: M(r, c) = conj(T[c + 32 r]).
template <bool SUB, bool CT>
__device__ __forceinline__ void tile_apply(Blk& acc, const float2* __restrict__ T, const float* __restrict__ v) {
#pragma unroll 2
  for (int c = 0; c < 32; ++c) {
    const float2 x = make_float2(v[c], v[32 + c]);
    if (!CT) {
      const float4* col = (const float4*)(T + 32 * c);
#pragma unroll
      for (int r2 = 0; r2 < 16; ++r2) {
        const float4 m = col[r2];
        float2 a0 = make_float2(acc.re[2 * r2], acc.im[2 * r2]);
        float2 a1 = make_float2(acc.re[2 * r2 + 1], acc.im[2 * r2 + 1]);
        if (SUB) {
          cfms(a0, make_float2(m.x, m.y), x);
          cfms(a1, make_float2(m.z, m.w), x);
        } else {
          cfma(a0, make_float2(m.x, m.y), x);
          cfma(a1, make_float2(m.z, m.w), x);
        }
        acc.re[2 * r2] = a0.x;
        acc.im[2 * r2] = a0.y;
        acc.re[2 * r2 + 1] = a1.x;
        acc.im[2 * r2 + 1] = a1.y;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const float2 m = cconj(T[c + 32 * r]);
        float2 a = make_float2(acc.re[r], acc.im[r]);
        if (SUB)
          cfms(a, m, x);
        else
          cfma(a, m, x);
        acc.re[r] = a.x;
        acc.im[r] = a.y;
      }
    }
  }
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

// copy the tiles (and, for the interchange steps, the panel permutation) of step s into buffer `buf`
template <int TRANS>
__device__ __forceinline__ void prefetch_step(const FactorGeom& g, const FactorPtr<float2>& f, int s, float2* tbuf,
                                              int16_t* pbuf) {
  const StepInfo st = step_info<TRANS>(g, s);
  const int chunks = 512;  // 16-byte chunks of a 32 x 32 complex64 tile
  for (int i = 0; i < st.ntiles; ++i) {
    const float2* src = tile_src<TRANS>(g, f, st, i);
    float2* dst = tbuf + i * 1024;
    for (int e = threadIdx.x; e < chunks; e += blockDim.x) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst + 2 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 2 * e));
    }
  }
  const bool perm = (TRANS == 0 && st.sweep == 0) || (TRANS == 1 && st.sweep == 1);
  if (perm) {
    const int Pmax = (g.bt + 1) * kTile;  // int16 entries, a multiple of 8 (16-byte chunks)
    const int16_t* src = f.perm + (int64_t)st.K * Pmax;
    for (int e = threadIdx.x; e < Pmax / 8; e += blockDim.x) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(pbuf + 8 * e);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + 8 * e));
    }
  }
  asm volatile("cp.async.commit_group;\n" ::);
}

// ---------------------------------------------------------------------------
// the persistent kernel: CTAs take (system, 128-column block) items from a counter
// ---------------------------------------------------------------------------
template <int TRANS>
__global__ void __launch_bounds__(kTmThreads, 1)
    solve_tm_kernel(FactorGeom g, const SysDesc* sys, const char* arena, const float2* rhs, float2* out,
                    const int2* items, int nitems, int* counter, uint32_t tmem_cols, int max_tiles) {
  extern __shared__ __align__(16) char smem[];
  const int Pmax = (g.bt + 1) * kTile;
  float2* tbuf0 = (float2*)smem;                               // 2 buffers of max_tiles tiles
  float2* tbuf1 = tbuf0 + (size_t)max_tiles * 1024;
  float* vrow = (float*)(tbuf1 + (size_t)max_tiles * 1024);    // kTmThreads x kSRow
  float* orow = vrow + kTmThreads * kSRow;                     // kTmThreads x kSRow
  int16_t* pbuf0 = (int16_t*)(orow + kTmThreads * kSRow);      // 2 x Pmax
  int16_t* pbuf1 = pbuf0 + Pmax;
  int* pinv = (int*)(pbuf1 + Pmax);                            // Pmax
  __shared__ uint32_t tslot;
  __shared__ int sh_item;

  const int t = threadIdx.x, warp = t >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(&tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tslot + ((uint32_t)(32 * (warp & 3)) << 16);
  float* myv = vrow + t * kSRow;  // the vector operand of tile_apply
  float* myo = orow + t * kSRow;  // the old top block during an interchange
  const int bt = g.bt, Nb = g.Nb;
  const int64_t n = g.n;

  for (;;) {
    if (t == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    if (item >= nitems) break;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    const FactorPtr<float2> f = factor_ptr<float2>(g, (char*)arena + d.factor_off);
    const int col = w.y + t;
    const bool valid = col < d.ncols;
    const float2* Y = rhs + d.rhs_off + (int64_t)(valid ? col : 0) * n;
    float2* X = out + (TRANS == 0 ? d.out_off : d.out2_off) + (int64_t)(valid ? col : 0) * n;
    const int nsteps = 2 * Nb;
    const int nslot_w = bt + 1;  // window ring of the interchange sweeps
    const int nslot_s = 2 * bt;  // ring of solved blocks of the other sweeps
    auto slot_addr = [&](int J, int ring) -> uint32_t { return tbase + (uint32_t)(64 * (J % ring)); };

    prefetch_step<TRANS>(g, f, 0, tbuf0, pbuf0);
    if (TRANS == 0) {  // the first window of the forward sweep: blocks 0 .. min(bt, Nb-1) of Y
      Blk y;
      for (int q = 0; q <= min(bt, Nb - 1); ++q) {
        blk_from_global(y, Y, n, (int64_t)q * kTile, valid);
        blk_to_tm(y, slot_addr(q, nslot_w));
      }
    }
    for (int s = 0; s < nsteps; ++s) {
      float2* tb = (s & 1) ? tbuf1 : tbuf0;
      int16_t* pb = (s & 1) ? pbuf1 : pbuf0;
      asm volatile("cp.async.wait_group 0;\n" ::);
      __syncthreads();  // step s's tiles are here; every thread is past step s-1's tiles
      if (s + 1 < nsteps) prefetch_step<TRANS>(g, f, s + 1, (s & 1) ? tbuf0 : tbuf1, (s & 1) ? pbuf0 : pbuf1);
      const StepInfo st = step_info<TRANS>(g, s);
      const int K = st.K;
      const int64_t row0 = (int64_t)K * kTile;
      Blk acc, x;
      if (TRANS == 0 && st.sweep == 0) {
        // ---- forward: P_K, then x_K = Linv_K (top block), then the L updates below ----
        const int nbb = st.ntiles - 1;
        const int P = (nbb + 1) * kTile;
        const uint32_t top = slot_addr(K, nslot_w);
        blk_from_tm(acc, top);
        blk_to_row(acc, myo);  // the old top block, by row
        // new row r of the window is old row perm[r]: the top rows gather (the old top from the row
        // scratch, lower rows from TMEM), then the old top rows that move down are written in place
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int src = pb[r];
          if (src < 32) {
            x.re[r] = myo[src];
            x.im[r] = myo[32 + src];
          } else {
            const uint32_t a = slot_addr(K + src / 32, nslot_w) + (uint32_t)(src % 32);
            uint32_t vr = tm_ld1(a), vi = tm_ld1(a + 32);
            tm_wait_ld();
            reg_fence1(vr);
            reg_fence1(vi);
            x.re[r] = __uint_as_float(vr);
            x.im[r] = __uint_as_float(vi);
          }
        }
        for (int r = 32; r < P; ++r) {
          const int src = pb[r];
          if (src < 32) {
            const uint32_t a = slot_addr(K + r / 32, nslot_w) + (uint32_t)(r % 32);
            tm_st1(a, __float_as_uint(myo[src]));
            tm_st1(a + 32, __float_as_uint(myo[32 + src]));
          }
        }
        tm_wait_st();
        blk_to_row(x, myv);
        blk_zero(acc);
        tile_apply<false, false>(acc, tb, myv);  // x_K = Linv_K g
        blk_to_global(acc, X, n, row0, valid);
        blk_to_row(acc, myv);
        for (int q = 1; q <= nbb; ++q) {
          const uint32_t a = slot_addr(K + q, nslot_w);
          blk_from_tm(x, a);
          tile_apply<true, false>(x, tb + q * 1024, myv);  // rows of block K+q -= L(K+q, K) x_K
          blk_to_tm(x, a);
        }
        if (K + bt + 1 < Nb) {  // block K+bt+1 of Y enters the slot block K leaves
          blk_from_global(x, Y, n, (int64_t)(K + bt + 1) * kTile, valid);
          blk_to_tm(x, top);
        }
      } else if (TRANS == 0) {
        // ---- backward: x_K = Uinv_K (w_K - sum_q U(K, K+q) x_{K+q}) ----
        const int nbr = st.ntiles - 1;
        blk_from_global(acc, X, n, row0, valid);  // w_K, written by this thread's forward sweep
        for (int q = 1; q <= nbr; ++q) {
          blk_from_tm(x, slot_addr(K + q, nslot_s));
          blk_to_row(x, myv);
          tile_apply<true, false>(acc, tb + (q - 1) * 1024, myv);
        }
        blk_to_row(acc, myv);
        blk_zero(x);
        tile_apply<false, false>(x, tb + nbr * 1024, myv);
        blk_to_tm(x, slot_addr(K, nslot_s));
        blk_to_global(x, X, n, row0, valid);
      } else if (st.sweep == 0) {
        // ---- adjoint forward: w_K = Uinv_K^H (y_K - sum_q U(K-q, K)^H w_{K-q}) ----
        const int nq = st.ntiles - 1;
        blk_from_global(acc, Y, n, row0, valid);
        for (int q = 1; q <= nq; ++q) {
          blk_from_tm(x, slot_addr(K - q, nslot_s));
          blk_to_row(x, myv);
          tile_apply<true, true>(acc, tb + (q - 1) * 1024, myv);
        }
        blk_to_row(acc, myv);
        blk_zero(x);
        tile_apply<false, true>(x, tb + nq * 1024, myv);
        blk_to_tm(x, slot_addr(K, nslot_s));
        blk_to_global(x, X, n, row0, valid);
      } else {
        // ---- adjoint backward: v_K = Linv_K^H (w_K - sum_q L(K+q, K)^H v_{K+q}), then P_K^T ----
        const int nbb = st.ntiles - 1;
        const int P = (nbb + 1) * kTile;
        for (int r = t; r < P; r += blockDim.x) pinv[pb[r]] = r;  // P_K^T puts window row r at pm[r]
        blk_from_global(acc, X, n, row0, valid);                   // w_K from the adjoint forward sweep
        for (int q = 1; q <= nbb; ++q) {
          blk_from_tm(x, slot_addr(K + q, nslot_w));
          blk_to_row(x, myv);
          tile_apply<true, true>(acc, tb + (q - 1) * 1024, myv);
        }
        blk_to_row(acc, myv);
        blk_zero(x);
        tile_apply<false, true>(x, tb + nbb * 1024, myv);
        blk_to_row(x, myo);  // the old top block (v_K), by row
        __syncthreads();     // pinv complete
        // new row r of the window is old row pinv[r]
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int src = pinv[r];
          if (src < 32) {
            acc.re[r] = myo[src];
            acc.im[r] = myo[32 + src];
          } else {
            const uint32_t a = slot_addr(K + src / 32, nslot_w) + (uint32_t)(src % 32);
            uint32_t vr = tm_ld1(a), vi = tm_ld1(a + 32);
            tm_wait_ld();
            reg_fence1(vr);
            reg_fence1(vi);
            acc.re[r] = __uint_as_float(vr);
            acc.im[r] = __uint_as_float(vi);
          }
        }
        for (int r = 32; r < P; ++r) {
          const int src = pinv[r];
          if (src < 32) {
            const uint32_t a = slot_addr(K + r / 32, nslot_w) + (uint32_t)(r % 32);
            tm_st1(a, __float_as_uint(myo[src]));
            tm_st1(a + 32, __float_as_uint(myo[32 + src]));
          }
        }
        tm_wait_st();
        blk_to_tm(acc, slot_addr(K, nslot_w));
        if (nbb == bt) {  // block K+bt is final
          blk_from_tm(x, slot_addr(K + bt, nslot_w));
          blk_to_global(x, X, n, (int64_t)(K + bt) * kTile, valid);
        }
        if (K == 0) {  // the blocks left in the window are final
          for (int J = 0; J < min(bt, Nb); ++J) {
            blk_from_tm(x, slot_addr(J, nslot_w));
            blk_to_global(x, X, n, (int64_t)J * kTile, valid);
          }
        }
      }
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(tmem_cols));
}

}  // namespace

// Largest band the TMEM window holds: 2 bt blocks of 64 columns within 512.
bool solve_tm_supported(const FactorGeom& g) { return g.bt >= 1 && 2 * g.bt * 64 <= 512 && (g.bt + 1) * 64 <= 512; }

size_t solve_tm_smem_bytes(const FactorGeom& g) {
  const int max_tiles = 2 * g.bt + 1;
  const int Pmax = (g.bt + 1) * kTile;
  size_t bytes = (size_t)2 * max_tiles * 1024 * sizeof(float2) + (size_t)2 * kTmThreads * kSRow * sizeof(float) +
                 (size_t)2 * Pmax * sizeof(int16_t) + (size_t)Pmax * sizeof(int);
  // at least 116 KiB, so that one CTA (and its TMEM allocation) owns each SM
  return std::max(bytes, (size_t)116 * 1024);
}

int launch_solve_tm(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                    const float2* rhs_arena, float2* out_arena, void* queue, cudaStream_t st) {
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
                                                       counter, cols, max_tiles);
  } else {
    PD_CK(cudaFuncSetAttribute(solve_tm_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_tm_kernel<0><<<grid, kTmThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                       counter, cols, max_tiles);
  }
  PD_CK_LAUNCH();
  return 0;
}

}  // namespace pdeshep
