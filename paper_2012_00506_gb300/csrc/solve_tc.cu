// solve_tc.cu -- complex64 band solves of eq. (10) with the tile products on
// the tcgen05 tensor cores (3xTF32: FP32-class accuracy).
//
// A CTA of 128 threads takes 128 right-hand sides of one system; thread m owns
// right-hand side m and TMEM lane m.  Every tile product of a sweep step is
// one MMA group D(128 x 64) (+)= A(128 x 64) B(64 x 64)^T in real arithmetic:
//   A = [Re x | Im x] of the 128 right-hand sides (the vector of the step),
//   B = the factor tile T (or its conjugate transpose) embedded as
//       [[s Tr, -s Ti], [s Ti, s Tr]] (rows: real parts then imaginary parts
//       of the 32 output rows; columns: Re x then Im x), s = +1 or -1,
//   D = a block of 32 complex rows in TMEM as [Re | Im] (FP32 accumulator),
// and A, B split into TF32 high and low parts, D += A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the low-by-low term is below FP32 rounding).  Operands are written
// by the threads into shared memory in the K-major 64-byte-swizzle layout and
// issued by one thread; completion is tracked by mbarriers whose waits are
// bounded (a give-up sets the error word and the CTA stops).
//
// Sweeps (all right-looking, so that every update is a product into TMEM):
//   trans 0, forward:  P_K on the window (blocks K..K+bt), x_K = Linv_K g_K,
//                      block K+q += (-L(K+q, K)) x_K           q = 1..bt
//   trans 0, backward: x_K = Uinv_K acc_K,  block K-q += (-U(K-q, K)) x_K
//                      q = 1..2bt (pending blocks start as the forward result)
//   trans 1, forward (U^H w = y): w_K = Uinv_K^H acc_K,
//                      block K+q += (-U(K, K+q)^H) w_K          q = 1..2bt
// The adjoint backward sweep (L^H with the inverse interchanges, whose window
// rows move between steps) runs on the TMEM kernel of solve_tm.cu.
#include <algorithm>

#include "band_lu.cuh"

namespace pdeshep {
namespace {

constexpr int kTcThreads = 128;
constexpr int kARows = 128, kBRows = 64, kK = 64;
constexpr int kABytes = kARows * kK * 4;   // one TF32 part of A: 32 KiB
constexpr int kBBytes = kBRows * kK * 4;   // one TF32 part of B: 16 KiB
constexpr int kSRow = 65;
// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBRows >> 3) << 17) |
                            ((uint32_t)(kARows >> 4) << 24);
constexpr int kPollLimit = 1 << 22;

// set when a bounded wait of the kernel gave up (read and cleared by the host)
__device__ int g_tc_solve_err;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------------------------
// TMEM, mbarrier and MMA wrappers
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
__device__ __forceinline__ void reg_fence16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// bounded wait for the phase of the given parity; false if it never completed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < kPollLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 32) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
      : "memory");
}

// byte offset of element (row, k) of an operand of R rows x 64 TF32 in the K-major
// 64-byte-swizzle layout: 4 regions of 16 K-elements, each R rows x 64 bytes in groups of
// 8 rows (512 bytes); 16-byte granule g of row r sits at granule g ^ ((r >> 1) & 3)
__device__ __forceinline__ uint32_t sw_off(int row, int k, int R) {
  const int kin = k & 15, g = kin >> 2, r8 = row & 7;
  return (uint32_t)((k >> 4) * (R * 64) + (row >> 3) * 512 + r8 * 64 + ((g ^ ((r8 >> 1) & 3)) << 4) + ((kin & 3) << 2));
}

__device__ __forceinline__ uint32_t tf32_hi(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

// A row m: values a[0..63] (re 0..31, im 32..63) -> TF32 high and low parts
__device__ __forceinline__ void write_a_row(unsigned char* Ahi, unsigned char* Alo, int m, const float (&a)[64]) {
#pragma unroll
  for (int g = 0; g < 16; ++g) {
    uint4 h, l;
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float v = a[4 * g + e];
      hv[e] = tf32_hi(v);
      lv[e] = tf32_hi(v - __uint_as_float(hv[e]));
    }
    h = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    l = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    const uint32_t off = sw_off(m, 4 * g, kARows);
    *(uint4*)(Ahi + off) = h;
    *(uint4*)(Alo + off) = l;
  }
}

// Register prefetch of one factor tile as M = T (CT = false) or M = T^H (CT = true): thread t holds
// M(r, c0..c0+7) with r = t % 32, c0 = 8 (t / 32) (for M = T the 32 lanes read 32 consecutive rows
// of a column: coalesced).
struct TileRegs {
  float2 v[8];
};
template <bool CT>
__device__ __forceinline__ void tile_fetch(TileRegs& r, const float2* __restrict__ T) {
  const int i = threadIdx.x & 31, c0 = 8 * (threadIdx.x >> 5);
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    if (CT) {
      const float2 v = T[(c0 + jj) + 32 * i];
      r.v[jj] = make_float2(v.x, -v.y);
    } else {
      r.v[jj] = T[i + 32 * (c0 + jj)];
    }
  }
}
// four values -> TF32 high and low granules at byte offset off
__device__ __forceinline__ void put_granule(unsigned char* Bhi, unsigned char* Blo, uint32_t off, float a, float b,
                                            float c, float d) {
  const float v[4] = {a, b, c, d};
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    h[e] = tf32_hi(v[e]);
    l[e] = tf32_hi(v[e] - __uint_as_float(h[e]));
  }
  *(uint4*)(Bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *(uint4*)(Blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}
// B (TF32 high and low parts) of the embedded tile: B[n][k] = s [[Mr, -Mi], [Mi, Mr]],
// n = output row (re 0..31, im 32..63), k = input (re 0..31, im 32..63); 16-byte granules
struct BOffsets {  // this thread's 8 granule offsets in a B part (constant per thread)
  uint32_t o[8];
  __device__ void init() {
    const int r = threadIdx.x & 31, c0 = 8 * (threadIdx.x >> 5);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int k = c0 + 4 * g;
      o[4 * g + 0] = sw_off(r, k, kBRows);
      o[4 * g + 1] = sw_off(r, 32 + k, kBRows);
      o[4 * g + 2] = sw_off(32 + r, k, kBRows);
      o[4 * g + 3] = sw_off(32 + r, 32 + k, kBRows);
    }
  }
};
__device__ __forceinline__ void write_b(unsigned char* Bhi, unsigned char* Blo, const TileRegs& t, float s,
                                        const BOffsets& bo) {
  float mr[8], mi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    mr[j] = s * t.v[j].x;
    mi[j] = s * t.v[j].y;
  }
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const float* R = mr + 4 * g;
    const float* I = mi + 4 * g;
    put_granule(Bhi, Blo, bo.o[4 * g + 0], R[0], R[1], R[2], R[3]);
    put_granule(Bhi, Blo, bo.o[4 * g + 1], -I[0], -I[1], -I[2], -I[3]);
    put_granule(Bhi, Blo, bo.o[4 * g + 2], I[0], I[1], I[2], I[3]);
    put_granule(Bhi, Blo, bo.o[4 * g + 3], R[0], R[1], R[2], R[3]);
  }
}

// L2 prefetch of `lines` 128-byte lines from p, spread over the CTA's threads (offset by `slot`)
__device__ __forceinline__ void l2_prefetch(const void* p, int lines, int slot) {
  for (int l = (threadIdx.x + slot * 37) % kTcThreads; l < lines; l += kTcThreads)
    asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)p + 128 * l));
}
// this thread's right-hand side, rows row0..row0+31 (two lines)
__device__ __forceinline__ void l2_prefetch_rows(const float2* X, int64_t n, int64_t row0, bool valid) {
  if (!valid || row0 >= n) return;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(X + row0));
  if (row0 + 16 < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(X + row0 + 16));
}

// the 3xTF32 product of one tile: 8 K-steps of 8, three MMAs each.  The descriptor of K-step s is
// the base descriptor plus the step's byte offset / 16 (the start-address field; no carry out of
// it below 256 KiB of shared memory).
__device__ __forceinline__ void mma_group(uint32_t d, uint64_t dahi, uint64_t dalo, uint64_t dbhi, uint64_t dblo,
                                          bool accumulate) {
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const uint64_t ka = (uint64_t)(((s >> 1) * (kARows * 64) + (s & 1) * 32) >> 4);
    const uint64_t kb = (uint64_t)(((s >> 1) * (kBRows * 64) + (s & 1) * 32) >> 4);
    mma_tf32(d, dahi + ka, dbhi + kb, (accumulate || s > 0) ? 1u : 0u);
    mma_tf32(d, dahi + ka, dblo + kb, 1u);
    mma_tf32(d, dalo + ka, dbhi + kb, 1u);
  }
}

// TMEM block (64 columns of this thread's lane) <-> 64 registers
__device__ __forceinline__ void blk_from_tm(float (&b)[64], uint32_t a) {
  uint32_t v0[16], v1[16], v2[16], v3[16];
  tm_ld16(a, v0);
  tm_ld16(a + 16, v1);
  tm_ld16(a + 32, v2);
  tm_ld16(a + 48, v3);
  tm_wait_ld();
  reg_fence16(v0);
  reg_fence16(v1);
  reg_fence16(v2);
  reg_fence16(v3);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    b[i] = __uint_as_float(v0[i]);
    b[16 + i] = __uint_as_float(v1[i]);
    b[32 + i] = __uint_as_float(v2[i]);
    b[48 + i] = __uint_as_float(v3[i]);
  }
}
__device__ __forceinline__ void blk_to_tm(const float (&b)[64], uint32_t a) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    uint32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __float_as_uint(b[16 * h + i]);
    tm_st16(a + 16 * h, v);
  }
  tm_wait_st();
}
// global rows row0..row0+31 of this thread's right-hand side <-> [re | im] registers
__device__ __forceinline__ void blk_from_global(float (&b)[64], const float2* __restrict__ Y, int64_t n, int64_t row0,
                                                bool valid) {
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float2 v = make_float2(0.f, 0.f);
    if (valid && row0 + r < n) v = Y[row0 + r];
    b[r] = v.x;
    b[32 + r] = v.y;
  }
}
__device__ __forceinline__ void blk_to_global(const float (&b)[64], float2* __restrict__ X, int64_t n, int64_t row0,
                                              bool valid) {
  if (!valid) return;
#pragma unroll
  for (int r = 0; r < 32; ++r)
    if (row0 + r < n) X[row0 + r] = make_float2(b[r], b[32 + r]);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
struct Sync {
  uint32_t bar_b[2], bar_x, bar_step;
  int uses_b[2], nx, nstep;
  int* sh_bad;
  // a bounded wait without a barrier: a give-up is recorded for the next barrier to see
  __device__ void wait_nb(uint32_t bar, int k) {
    if (!mbar_wait(bar, (uint32_t)((k - 1) & 1))) {
      atomicExch(&g_tc_solve_err, 1);
      *sh_bad = 1;
    }
  }
  // a CTA-uniform bounded wait for the k-th completion (k >= 1) of bar
  __device__ bool wait(uint32_t bar, int k) {
    bool ok = mbar_wait(bar, (uint32_t)((k - 1) & 1));
    if (!ok) {
      atomicExch(&g_tc_solve_err, 1);
      *sh_bad = 1;
    }
    return __syncthreads_or(!ok) == 0;
  }
};

template <int TRANS>
__global__ void __launch_bounds__(kTcThreads, 1)
    solve_tc_kernel(FactorGeom g, const SysDesc* sys, const char* arena, const float2* rhs, float2* out,
                    const int2* items, int nitems, int* counter) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* Ahi = sm;
  unsigned char* Alo = Ahi + kABytes;
  unsigned char* Bhi[2] = {Alo + kABytes, Alo + kABytes + 2 * kBBytes};
  unsigned char* Blo[2] = {Bhi[0] + kBBytes, Bhi[1] + kBBytes};
  float* orow = (float*)(Bhi[1] + 2 * kBBytes);             // kTcThreads x kSRow
  const int Pmax = (g.bt + 1) * kTile;
  int16_t* perm = (int16_t*)(orow + kTcThreads * kSRow);     // Pmax
  uint64_t* bars = (uint64_t*)(((uintptr_t)(perm + Pmax) + 7) & ~(uintptr_t)7);
  __shared__ uint32_t tslot;
  __shared__ int sh_item, sh_bad;

  const int t = threadIdx.x, warp = t >> 5;
  Sync sy;
  sy.bar_b[0] = smem_u32(bars);
  sy.bar_b[1] = smem_u32(bars + 1);
  sy.bar_x = smem_u32(bars + 2);
  sy.bar_step = smem_u32(bars + 3);
  sy.uses_b[0] = sy.uses_b[1] = sy.nx = sy.nstep = 0;
  sy.sh_bad = &sh_bad;
  if (t == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(bars + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh_bad = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tslot;                          // lane 0, column 0 (MMA destinations)
  const uint32_t tb = tslot + ((uint32_t)(32 * warp) << 16);  // this thread's lane quadrant
  const uint64_t da_hi = sw64_desc(smem_u32(Ahi)), da_lo = sw64_desc(smem_u32(Alo));
  const uint64_t db_hi[2] = {sw64_desc(smem_u32(Bhi[0])), sw64_desc(smem_u32(Bhi[1]))};
  const uint64_t db_lo[2] = {sw64_desc(smem_u32(Blo[0])), sw64_desc(smem_u32(Blo[1]))};
  float* myo = orow + t * kSRow;
  const int bt = g.bt, Nb = g.Nb;
  const int64_t n = g.n;
  const int ringw = bt + 1, rings = 2 * bt;
  const uint32_t scratch = (uint32_t)(64 * ringw);       // forward: x_K's TMEM block after the window
  int cur = 0;                                           // B buffer for the next tile
  BOffsets boff;
  boff.init();
  bool alive = true;

  // B buffer `cur` <- tile (after the MMA that last read it), then the tile's MMA group into TMEM
  // column d; returns false if a wait gave up
  auto issue_tile = [&](const TileRegs& tr, float s, uint32_t d, bool accumulate, bool commit_x,
                        bool commit_step) -> bool {
    const int b = cur;
    // the MMA that last read this buffer (two groups ago) is normally long done; a wait that
    // gives up is seen by every thread after the barrier below
    if (sy.uses_b[b] > 0) sy.wait_nb(sy.bar_b[b], sy.uses_b[b]);
    write_b(Bhi[b], Blo[b], tr, s, boff);
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    if (sh_bad) return false;
    if (t == 0) {
      tc_fence_after();
      mma_group(tbase + d, da_hi, da_lo, db_hi[b], db_lo[b], accumulate);
      tc_commit(sy.bar_b[b]);
      if (commit_x) tc_commit(sy.bar_x);
      if (commit_step) tc_commit(sy.bar_step);
    }
    sy.uses_b[b] += 1;
    if (commit_x) sy.nx += 1;
    if (commit_step) sy.nstep += 1;
    cur ^= 1;
    return true;
  };
  // A <- this thread's 64 values (after the MMAs that read the previous A)
  auto write_a = [&](const float (&a)[64]) {
    write_a_row(Ahi, Alo, t, a);
    proxy_fence();
  };

  for (;;) {
    if (t == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    if (item >= nitems || !alive) break;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    const FactorPtr<float2> f = factor_ptr<float2>(g, (char*)arena + d.factor_off);
    const int col = w.y + t;
    const bool valid = col < d.ncols;
    const float2* Y = rhs + d.rhs_off + (int64_t)(valid ? col : 0) * n;
    float2* X = out + (TRANS == 0 ? d.out_off : d.out2_off) + (int64_t)(valid ? col : 0) * n;
    auto tile_of = [&](int I, int J) { return f.tiles + g.tile_index(I, J) * g.tile_elems; };
    float v[64], x[64];
    TileRegs tr;

    if (TRANS == 0) {
      // ======================= forward: P, L =======================
      for (int q = 0; q <= min(bt, Nb - 1); ++q) {
        blk_from_global(v, Y, n, (int64_t)q * kTile, valid);
        blk_to_tm(v, tb + (uint32_t)(64 * (q % ringw)));
      }
      for (int K = 0; K < Nb && alive; ++K) {
        const int nbb = min(bt, Nb - 1 - K);
        const int P = (nbb + 1) * kTile;
        // the window's updates of the previous step are complete
        if (sy.nstep > 0 && !sy.wait(sy.bar_step, sy.nstep)) { alive = false; break; }
        tc_fence_after();
        for (int r = t; r < P; r += kTcThreads) perm[r] = f.perm[(int64_t)K * Pmax + r];
        if (K + 1 < Nb) {  // the next step's tiles, permutation and entering block toward L2
          const int nb1 = min(bt, Nb - 2 - K);
          l2_prefetch(f.inv + (int64_t)(2 * (K + 1)) * g.tile_elems, 64, 0);
          for (int q = 1; q <= nb1; ++q) l2_prefetch(tile_of(K + 1 + q, K + 1), 64, q);
          l2_prefetch(f.perm + (int64_t)(K + 1) * Pmax, (Pmax * 2 + 127) / 128, 7);
          l2_prefetch_rows(Y, n, (int64_t)(K + bt + 2) * kTile, valid);
        }
        tile_fetch<false>(tr, f.inv + (int64_t)(2 * K) * g.tile_elems);
        const uint32_t top = (uint32_t)(64 * (K % ringw));
        blk_from_tm(v, tb + top);
#pragma unroll
        for (int r = 0; r < 64; ++r) myo[r] = v[r];
        __syncthreads();  // perm is complete
        // new row r = old row perm[r]: the top rows gather, the old top rows that move down
        uint32_t ur[32], ui[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int s = perm[r];
          ur[r] = ui[r] = 0u;
          if (s >= 32) {
            const uint32_t a = tb + (uint32_t)(64 * ((K + s / 32) % ringw) + s % 32);
            ur[r] = tm_ld1(a);
            ui[r] = tm_ld1(a + 32);
          }
        }
        tm_wait_ld();
        reg_fence16(*(uint32_t(*)[16])&ur[0]);
        reg_fence16(*(uint32_t(*)[16])&ur[16]);
        reg_fence16(*(uint32_t(*)[16])&ui[0]);
        reg_fence16(*(uint32_t(*)[16])&ui[16]);
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int s = perm[r];
          v[r] = s < 32 ? myo[s] : __uint_as_float(ur[r]);
          v[32 + r] = s < 32 ? myo[32 + s] : __uint_as_float(ui[r]);
        }
        for (int rho = 32; rho < P; ++rho) {
          const int s = perm[rho];
          if (s < 32) {
            const uint32_t a = tb + (uint32_t)(64 * ((K + rho / 32) % ringw) + rho % 32);
            tm_st1(a, __float_as_uint(myo[s]));
            tm_st1(a + 32, __float_as_uint(myo[32 + s]));
          }
        }
        tm_wait_st();
        // x_K = Linv_K g (A's previous readers, the last step's updates, finished with bar_step)
        write_a(v);
        if (!issue_tile(tr, 1.f, scratch, false, true, nbb == 0)) { alive = false; break; }
        if (nbb >= 1) tile_fetch<false>(tr, tile_of(K + 1, K));
        if (!sy.wait(sy.bar_x, sy.nx)) { alive = false; break; }
        tc_fence_after();
        blk_from_tm(x, tb + scratch);
        write_a(x);
        for (int q = 1; q <= nbb; ++q) {
          const TileRegs cur_t = tr;
          if (q < nbb) tile_fetch<false>(tr, tile_of(K + q + 1, K));
          if (!issue_tile(cur_t, -1.f, (uint32_t)(64 * ((K + q) % ringw)), true, false, q == nbb)) {
            alive = false;
            break;
          }
          if (q == 1) blk_to_global(x, X, n, (int64_t)K * kTile, valid);  // while the first update runs
        }
        if (!alive) break;
        if (nbb == 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid);
        if (K + bt + 1 < Nb) {  // block K+bt+1 of Y enters the slot block K leaves (no update writes it)
          blk_from_global(v, Y, n, (int64_t)(K + bt + 1) * kTile, valid);
          blk_to_tm(v, tb + top);
        }
      }
      if (!alive) break;
      // ======================= backward: U =======================
      if (sy.nstep > 0 && !sy.wait(sy.bar_step, sy.nstep)) { alive = false; break; }
      tc_fence_after();
      for (int J = Nb - 1; J >= max(0, Nb - rings); --J) {  // pending blocks start as the forward result
        blk_from_global(v, X, n, (int64_t)J * kTile, valid);
        blk_to_tm(v, tb + (uint32_t)(64 * (J % rings)));
      }
      for (int K = Nb - 1; K >= 0 && alive; --K) {
        const int nq = min(rings, K);
        const uint32_t sk = (uint32_t)(64 * (K % rings));
        if (sy.nstep > 0 && !sy.wait(sy.bar_step, sy.nstep)) { alive = false; break; }
        tc_fence_after();
        tile_fetch<false>(tr, f.inv + (int64_t)(2 * K + 1) * g.tile_elems);
        if (K >= 1) {  // the next step's tiles and entering block toward L2
          const int nq1 = min(rings, K - 1);
          l2_prefetch(f.inv + (int64_t)(2 * (K - 1) + 1) * g.tile_elems, 64, 0);
          for (int q = 1; q <= nq1; ++q) l2_prefetch(tile_of(K - 1 - q, K - 1), 64, q);
          if (K - 1 - rings >= 0) l2_prefetch_rows(X, n, (int64_t)(K - 1 - rings) * kTile, valid);
        }
        blk_from_tm(v, tb + sk);  // acc_K is complete
        write_a(v);
        if (!issue_tile(tr, 1.f, sk, false, true, nq == 0)) { alive = false; break; }
        if (nq >= 1) tile_fetch<false>(tr, tile_of(K - 1, K));
        if (!sy.wait(sy.bar_x, sy.nx)) { alive = false; break; }
        tc_fence_after();
        blk_from_tm(x, tb + sk);
        write_a(x);
        for (int q = 1; q <= nq; ++q) {
          const TileRegs cur_t = tr;
          if (q < nq) tile_fetch<false>(tr, tile_of(K - q - 1, K));
          if (!issue_tile(cur_t, -1.f, (uint32_t)(64 * ((K - q) % rings)), true, false, q == nq)) {
            alive = false;
            break;
          }
          if (q == 1) {  // while the first update runs: x_K out, and block K-2bt enters the slot K leaves
            blk_to_global(x, X, n, (int64_t)K * kTile, valid);
            if (K - rings >= 0) {
              blk_from_global(v, X, n, (int64_t)(K - rings) * kTile, valid);
              blk_to_tm(v, tb + sk);
            }
          }
        }
        if (nq == 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid);
      }
    } else {
      // ======================= adjoint forward: U^H =======================
      for (int J = 0; J < min(rings, Nb); ++J) {  // pending blocks start as y
        blk_from_global(v, Y, n, (int64_t)J * kTile, valid);
        blk_to_tm(v, tb + (uint32_t)(64 * (J % rings)));
      }
      for (int K = 0; K < Nb && alive; ++K) {
        const int nq = min(rings, Nb - 1 - K);
        const uint32_t sk = (uint32_t)(64 * (K % rings));
        if (sy.nstep > 0 && !sy.wait(sy.bar_step, sy.nstep)) { alive = false; break; }
        tc_fence_after();
        tile_fetch<true>(tr, f.inv + (int64_t)(2 * K + 1) * g.tile_elems);
        if (K + 1 < Nb) {  // the next step's tiles and entering block toward L2
          const int nq1 = min(rings, Nb - 2 - K);
          l2_prefetch(f.inv + (int64_t)(2 * (K + 1) + 1) * g.tile_elems, 64, 0);
          for (int q = 1; q <= nq1; ++q) l2_prefetch(tile_of(K + 1, K + 1 + q), 64, q);
          if (K + 1 + rings < Nb) l2_prefetch_rows(Y, n, (int64_t)(K + 1 + rings) * kTile, valid);
        }
        blk_from_tm(v, tb + sk);
        write_a(v);
        if (!issue_tile(tr, 1.f, sk, false, true, nq == 0)) { alive = false; break; }
        if (nq >= 1) tile_fetch<true>(tr, tile_of(K, K + 1));
        if (!sy.wait(sy.bar_x, sy.nx)) { alive = false; break; }
        tc_fence_after();
        blk_from_tm(x, tb + sk);
        write_a(x);
        for (int q = 1; q <= nq; ++q) {
          const TileRegs cur_t = tr;
          if (q < nq) tile_fetch<true>(tr, tile_of(K, K + q + 1));
          if (!issue_tile(cur_t, -1.f, (uint32_t)(64 * ((K + q) % rings)), true, false, q == nq)) {
            alive = false;
            break;
          }
          if (q == 1) {  // while the first update runs: w_K out, and block K+2bt enters the slot K leaves
            blk_to_global(x, X, n, (int64_t)K * kTile, valid);
            if (K + rings < Nb) {
              blk_from_global(v, Y, n, (int64_t)(K + rings) * kTile, valid);
              blk_to_tm(v, tb + sk);
            }
          }
        }
        if (nq == 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid);
      }
    }
    if (!alive) break;
    // the item's last products are complete before the next item reuses TMEM
    if (sy.nstep > 0 && !sy.wait(sy.bar_step, sy.nstep)) { alive = false; break; }
    tc_fence_after();
    __syncthreads();
  }
  // drain: wait (bounded) for every committed group before TMEM is released
  for (int b = 0; b < 2; ++b)
    if (sy.uses_b[b] > 0) mbar_wait(sy.bar_b[b], (uint32_t)((sy.uses_b[b] - 1) & 1));
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(512u));
}

}  // namespace

bool solve_tc_supported(const FactorGeom& g) { return g.bt >= 1 && 64 * 2 * g.bt <= 512 && 64 * (g.bt + 2) <= 512; }

size_t solve_tc_smem_bytes(const FactorGeom& g) {
  const int Pmax = (g.bt + 1) * kTile;
  return 1024 + 2 * (size_t)kABytes + 4 * (size_t)kBBytes + (size_t)kTcThreads * kSRow * sizeof(float) +
         (size_t)Pmax * sizeof(int16_t) + 64;
}

int solve_tc_error(int* h_err, int clear, cudaStream_t st) {
  int* p = nullptr;
  PD_CK(cudaGetSymbolAddress((void**)&p, g_tc_solve_err));
  if (h_err) {
    PD_CK(cudaMemcpyAsync(h_err, p, sizeof(int), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
  }
  if (clear) PD_CK(cudaMemsetAsync(p, 0, sizeof(int), st));
  return 0;
}

int launch_solve_tc(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                    const float2* rhs_arena, float2* out_arena, void* queue, cudaStream_t st) {
  if (!nitems) return 0;
  if (!solve_tc_supported(g)) {
    set_last_error_msg("band too wide for the tensor-core solve window");
    return PDESHEP_CUDA_ERROR;
  }
  const size_t smem = solve_tc_smem_bytes(g);
  Arena qa(queue, ~size_t(0));
  int* counter = qa.take<int>(1);
  const int2* d_items = qa.take<int2>((size_t)nitems);
  int dev = 0, sms = 0;
  PD_CK(cudaGetDevice(&dev));
  PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, std::min(nitems, sms));
  PD_CK(cudaMemsetAsync(counter, 0, sizeof(int), st));
  if (trans) {
    PD_CK(cudaFuncSetAttribute(solve_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    solve_tc_kernel<1><<<grid, kTcThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                       counter);
    PD_CK_LAUNCH();
    // the adjoint backward sweep (L^H, inverse interchanges) on the TMEM kernel
    return launch_solve_tm(g, 1, nitems, d_sys, factor_arena, rhs_arena, out_arena, queue, st, 1, 2);
  }
  PD_CK(cudaFuncSetAttribute(solve_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  solve_tc_kernel<0><<<grid, kTcThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                     counter);
  PD_CK_LAUNCH();
  return 0;
}

}  // namespace pdeshep
