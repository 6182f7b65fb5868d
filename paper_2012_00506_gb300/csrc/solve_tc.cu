// solve_tc.cu -- complex64 band solves of eq. (10) with the tile products on
// the tcgen05 tensor cores (bf16x6 products: FP32-level accuracy).
//
// A CTA takes 128 right-hand sides of one system: four compute warps, thread m
// owning right-hand side m and TMEM lane m, and a fifth warp that only issues
// the MMAs (warp-specialised: operands are handed over through full/empty
// mbarriers, so preparing the next tile overlaps the running products and no
// CTA-wide barrier is taken inside a sweep).  Every tile product of a step is
// one MMA group D(128 x 64) (+)= A(128 x 64) B(64 x 64)^T in real arithmetic:
//   A = [Re x | Im x] of the 128 right-hand sides (the vector of the step),
//   B = the factor tile T (or its conjugate transpose) embedded as
//       [[s Tr, -s Ti], [s Ti, s Tr]] (rows: real parts then imaginary parts
//       of the 32 output rows; columns: Re x then Im x), s = +1 or -1,
//   D = a block of 32 complex rows in TMEM as [Re | Im] (FP32 accumulator),
// and A, B each split into three bf16 parts (a = a0 + a1 + a2, each part the
// round-to-nearest bf16 of the remainder: 24 significant bits, an FP32 value
// up to rounding at its last bit), D += a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 +
// a2 b0 (the dropped terms are below 2^-24 of the product).  Operands are written
// by the compute threads into shared memory in the K-major 64-byte-swizzle
// layout; the factor tiles reach shared memory by cp.async one step ahead, each
// warp copying exactly the part it reads.  Every mbarrier wait is bounded (a
// give-up sets the error word and the CTA stops at its next item).
//
// Sweeps (all right-looking, so that every update is a product into TMEM):
//   trans 0, forward:  P_K on the window (blocks K..K+bt), x_K = Linv_K g_K,
//                      block K+q += (-L(K+q, K)) x_K           q = 1..bt
//   trans 0, backward: x_K = Uinv_K acc_K,  block K-q += (-U(K-q, K)) x_K
//                      q = 1..2bt (pending blocks start as the forward result)
//   trans 1, forward (U^H w = y): w_K = Uinv_K^H acc_K,
//                      block K+q += (-U(K, K+q)^H) w_K          q = 1..2bt
//   trans 1, backward (L^H with the inverse interchanges, whose window rows move
//                      between steps, so it is left-looking): solve_tca_kernel below.
#include <algorithm>

#include "band_lu.cuh"

namespace pdeshep {
namespace {

constexpr int kTcCompute = 128;             // compute warps 0..3
constexpr int kTcThreads = kTcCompute + 32;  // + the MMA warp
constexpr int kARows = 128, kBRows = 64, kK = 64;
constexpr int kABytes = kARows * kK * 2;   // one bf16 part of A: 16 KiB
constexpr int kBBytes = kBRows * kK * 2;   // one bf16 part of B: 8 KiB
// instruction descriptor (kind::f16): D FP32, A and B BF16, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBRows >> 3) << 17) |
                            ((uint32_t)(kARows >> 4) << 24);
constexpr int kPollLimit = 1 << 22;

// set when a bounded wait of the kernel gave up (read and cleared by the host)
__device__ int g_tc_solve_err;
// polls after which the main waits give up (a testing hook lowers it; the drains before TMEM is
// released always use kPollLimit)
__device__ int g_tc_solve_polls = kPollLimit;

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
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc)
      : "memory");
}

// byte offset of bf16 element (row, k) of an operand of R rows x 64 in the K-major 64-byte-swizzle
// layout: 2 regions of 32 K-elements, each R rows x 64 bytes in groups of 8 rows (512 bytes);
// 16-byte granule g (8 elements) of row r sits at granule g ^ ((r >> 1) & 3)
__device__ __forceinline__ uint32_t sw_off(int row, int k, int R) {
  const int kin = k & 31, g = kin >> 3, r8 = row & 7;
  return (uint32_t)((k >> 5) * (R * 64) + (row >> 3) * 512 + r8 * 64 + ((g ^ ((r8 >> 1) & 3)) << 4) + ((kin & 7) << 1));
}

// (lo, hi) -> packed bf16x2, round to nearest (lo in the low half: the lower address)
__device__ __forceinline__ uint32_t bf2_rn(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// two values -> three packed bf16x2 words with e = p0 + p1 + p2 (each remainder is exact in FP32)
__device__ __forceinline__ void split3(float e0, float e1, uint32_t& w0, uint32_t& w1, uint32_t& w2) {
  w0 = bf2_rn(e0, e1);
  const float r0 = e0 - __uint_as_float(w0 << 16), r1 = e1 - __uint_as_float(w0 & 0xffff0000u);
  w1 = bf2_rn(r0, r1);
  w2 = bf2_rn(r0 - __uint_as_float(w1 << 16), r1 - __uint_as_float(w1 & 0xffff0000u));
}
// eight values -> the three parts' 16-byte granules
struct Granule3 {
  uint4 p[3];
};
__device__ __forceinline__ Granule3 split3x8(const float* v) {
  uint32_t w[3][4];
#pragma unroll
  for (int e = 0; e < 4; ++e) split3(v[2 * e], v[2 * e + 1], w[0][e], w[1][e], w[2][e]);
  Granule3 g;
#pragma unroll
  for (int q = 0; q < 3; ++q) g.p[q] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  return g;
}

// A row m: values a[0..63] (re 0..31, im 32..63) -> the three bf16 parts (kABytes apart)
__device__ __forceinline__ void write_a_row(unsigned char* A, int m, const float (&a)[64]) {
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const Granule3 q = split3x8(a + 8 * g);
    const uint32_t off = sw_off(m, 8 * g, kARows);
#pragma unroll
    for (int p = 0; p < 3; ++p) *(uint4*)(A + p * kABytes + off) = q.p[p];
  }
}

// One factor tile's 8 elements per thread: M = T (CT = false) or M = T^H (CT = true), thread t holds
// M(r, c0..c0+7) with r = t % 32, c0 = 8 (t / 32).
struct TileRegs {
  float2 v[8];
};

// Factor tiles are staged into shared memory by cp.async one sweep step ahead.  Staged layout of a
// column-major 32 x 32 complex64 tile: column c (256 bytes) at 256 c, its 16-byte chunk k (rows 2k,
// 2k+1) at chunk position k ^ (c & 15), so that reading along a row or along a column both spread
// over the banks.
constexpr int kSlotBytes = kTile * kTile * 8;
__device__ __forceinline__ uint32_t slot_off(int r, int c) {
  return (uint32_t)(c * 256 + (((r >> 1) ^ (c & 15)) << 4) + ((r & 1) << 3));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// the part of one tile (16-byte aligned in global memory) that compute warp w later reads, into the
// slot at shared address dst: columns 8w..8w+7 (CT = false) or rows 8w..8w+7 (CT = true); 4 chunks
// per lane
template <bool CT>
__device__ __forceinline__ void stage_tile_warp(uint32_t dst, const float2* __restrict__ T, int w, int lane) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = lane + 32 * j;
    const int c = CT ? (i >> 2) : 8 * w + (i >> 4);
    const int k = CT ? 4 * w + (i & 3) : (i & 15);
    cp_async16(dst + (uint32_t)(c * 256 + ((k ^ (c & 15)) << 4)), T + c * 32 + 2 * k);
  }
}
// `bytes` (a multiple of 16, at most 512) from p to the shared address dst, by one warp
__device__ __forceinline__ void stage_bytes_warp(uint32_t dst, const void* p, int bytes, int lane) {
  if (16 * lane < bytes) cp_async16(dst + (uint32_t)(16 * lane), (const char*)p + 16 * lane);
}
// wait until at most n of this thread's most recent cp.async groups are still in flight
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    case 7: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    case 8: asm volatile("cp.async.wait_group 8;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
  }
}
template <bool CT>
__device__ __forceinline__ void tile_from_slot(TileRegs& r, const unsigned char* slot) {
  const int i = threadIdx.x & 31, c0 = 8 * (threadIdx.x >> 5);
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    if (CT) {  // M(i, c) = conj T(c, i)
      const float2 v = *(const float2*)(slot + slot_off(c0 + jj, i));
      r.v[jj] = make_float2(v.x, -v.y);
    } else {
      r.v[jj] = *(const float2*)(slot + slot_off(i, c0 + jj));
    }
  }
}
// B (three bf16 parts, kBBytes apart) of the embedded tile: B[n][k] = s [[Mr, -Mi], [Mi, Mr]],
// n = output row (re 0..31, im 32..63), k = input (re 0..31, im 32..63).  Thread (r, c0) writes the
// four granules of rows r and 32 + r at k = c0..c0+7 and 32+c0..32+c0+7.
struct BOffsets {  // this thread's 4 granule offsets in a B part (constant per thread)
  uint32_t o[4];
  __device__ void init() {
    const int r = threadIdx.x & 31, c0 = 8 * (threadIdx.x >> 5);
    o[0] = sw_off(r, c0, kBRows);
    o[1] = sw_off(r, 32 + c0, kBRows);
    o[2] = sw_off(32 + r, c0, kBRows);
    o[3] = sw_off(32 + r, 32 + c0, kBRows);
  }
};
__device__ __forceinline__ void write_b(unsigned char* B, const TileRegs& t, float s, const BOffsets& bo) {
  float mr[8], mi[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    mr[j] = s * t.v[j].x;
    mi[j] = s * t.v[j].y;
  }
  const Granule3 R = split3x8(mr), I = split3x8(mi);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    unsigned char* Bp = B + p * kBBytes;
    const uint4 ni = make_uint4(I.p[p].x ^ 0x80008000u, I.p[p].y ^ 0x80008000u, I.p[p].z ^ 0x80008000u,
                                I.p[p].w ^ 0x80008000u);  // -Mi: the parts of -v are the negated parts of v
    *(uint4*)(Bp + bo.o[0]) = R.p[p];
    *(uint4*)(Bp + bo.o[1]) = ni;
    *(uint4*)(Bp + bo.o[2]) = I.p[p];
    *(uint4*)(Bp + bo.o[3]) = R.p[p];
  }
}

// L2 prefetch of compute warp w's quarter of one 8 KiB tile
__device__ __forceinline__ void l2_prefetch_tile(const void* p, int w, int lane) {
  if (lane < 16) asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)p + 128 * (16 * w + lane)));
}
// this thread's right-hand side, rows row0..row0+31 (two lines)
__device__ __forceinline__ void l2_prefetch_rows(const float2* X, int64_t n, int64_t row0, bool valid) {
  if (!valid || row0 >= n) return;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(X + row0));
  if (row0 + 16 < n) asm volatile("prefetch.global.L2 [%0];" ::"l"(X + row0 + 16));
}

// the bf16x6 product of one tile: 4 K-steps of 16, six MMAs each.  The descriptor of K-step s is
// the base descriptor plus the step's byte offset / 16 (the start-address field; no carry out of
// it below 256 KiB of shared memory).  da, db: descriptors of the three parts.
__device__ __forceinline__ void mma_group(uint32_t d, const uint64_t (&da)[3], const uint64_t (&db)[3],
                                          bool accumulate) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const uint64_t ka = (uint64_t)(((s >> 1) * (kARows * 64) + (s & 1) * 32) >> 4);
    const uint64_t kb = (uint64_t)(((s >> 1) * (kBRows * 64) + (s & 1) * 32) >> 4);
    mma_bf16(d, da[0] + ka, db[0] + kb, (accumulate || s > 0) ? 1u : 0u);
    mma_bf16(d, da[0] + ka, db[1] + kb, 1u);
    mma_bf16(d, da[1] + ka, db[0] + kb, 1u);
    mma_bf16(d, da[0] + ka, db[2] + kb, 1u);
    mma_bf16(d, da[1] + ka, db[1] + kb, 1u);
    mma_bf16(d, da[2] + ka, db[0] + kb, 1u);
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
// global rows row0..row0+31 of this thread's right-hand side <-> [re | im] registers; 16-byte
// accesses where the column is 16-byte aligned and the block is whole
__device__ __forceinline__ void blk_from_global(float (&b)[64], const float2* __restrict__ Y, int64_t n, int64_t row0,
                                                bool valid) {
  const float2* p = Y + row0;
  if (valid && row0 + 32 <= n && ((uintptr_t)p & 15) == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float4 q = *(const float4*)(p + 2 * k);
      b[2 * k] = q.x;
      b[32 + 2 * k] = q.y;
      b[2 * k + 1] = q.z;
      b[33 + 2 * k] = q.w;
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float2 v = make_float2(0.f, 0.f);
    if (valid && row0 + r < n) v = p[r];
    b[r] = v.x;
    b[32 + r] = v.y;
  }
}
// the row pairs (2k, 2k+1), k0 <= k < k1, of the block
__device__ __forceinline__ void blk_to_global(const float (&b)[64], float2* __restrict__ X, int64_t n, int64_t row0,
                                              bool valid, int k0, int k1) {
  if (!valid) return;
  float2* p = X + row0;
  const bool vec = row0 + 32 <= n && ((uintptr_t)p & 15) == 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k < k0 || k >= k1) continue;
    if (vec) {
      *(float4*)(p + 2 * k) = make_float4(b[2 * k], b[32 + 2 * k], b[2 * k + 1], b[33 + 2 * k]);
    } else {
      if (row0 + 2 * k < n) p[2 * k] = make_float2(b[2 * k], b[32 + 2 * k]);
      if (row0 + 2 * k + 1 < n) p[2 * k + 1] = make_float2(b[2 * k + 1], b[33 + 2 * k]);
    }
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// bounded wait for the k-th completion (k >= 1) of bar; gives up early once another warp has
// recorded a failure (unless `early` is false).  A give-up sets the error word and the CTA's
// failure flag.
__device__ __forceinline__ bool wait_k(uint32_t bar, int k, volatile int* bad, bool early = true,
                                       int polls = kPollLimit) {
  const uint32_t parity = (uint32_t)((k - 1) & 1);
  for (int it = 0; it < polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 32) {
      if (early && (it & 255) == 0 && *bad) break;
      __nanosleep(64);
    }
  }
  atomicExch(&g_tc_solve_err, 1);
  *bad = 1;
  return false;
}

// mbarriers of the CTA
enum { kBarFull0 = 0, kBarFull1, kBarEmpty0, kBarEmpty1, kBarAFull, kBarX, kBarStep, kBarDrain, kNumBars };

template <int TRANS>
__global__ void __launch_bounds__(kTcThreads, 1)
    solve_tc_kernel(FactorGeom g, const SysDesc* sys, const char* arena, const float2* rhs, float2* out,
                    const int2* items, int nitems, int* counter) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* Abuf = sm;                                   // A: three bf16 parts
  unsigned char* Bbuf = Abuf + 3 * kABytes;                   // B buffer b: three bf16 parts
  auto Bof = [&](int b) { return Bbuf + (size_t)b * 3 * kBBytes; };
  unsigned char* slots = Bbuf + 6 * kBBytes;                  // 2 bt + 1 staged factor tiles
  const int Pmax = (g.bt + 1) * kTile;
  int16_t* perm_base = (int16_t*)(slots + (size_t)(2 * g.bt + 1) * kSlotBytes);  // [warp][2][Pmax]
  uint64_t* bars = (uint64_t*)(((uintptr_t)(perm_base + 8 * Pmax) + 7) & ~(uintptr_t)7);
  __shared__ uint32_t tslot;
  __shared__ int sh_item;
  __shared__ volatile int sh_bad;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto bar = [&](int i) { return smem_u32(bars + i); };
  // a warp-uniform bounded wait (a give-up by any lane fails the whole warp; the warp reconverges)
  const int polls = g_tc_solve_polls;
  auto wwait = [&](uint32_t b, int k) -> bool { return __all_sync(~0u, wait_k(b, k, &sh_bad, true, polls)) != 0; };
  if (t == 0) {
    for (int i = 0; i < kNumBars; ++i)
      mbar_init(bar(i), (i == kBarFull0 || i == kBarFull1 || i == kBarAFull) ? 4u : 1u);
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
  const uint32_t tbase = tslot;                               // lane 0, column 0 (MMA destinations)
  const uint32_t tb = tslot + ((uint32_t)(32 * (warp & 3)) << 16);  // a compute warp's lane quadrant
  const int bt = g.bt, Nb = g.Nb;
  const int64_t n = g.n, te = g.tile_elems;
  const int ringw = bt + 1, rings = 2 * bt;
  const uint32_t scratch = (uint32_t)(64 * ringw);            // forward: x_K's TMEM block after the window
  // completion counts, kept identically by every thread that waits on the barrier
  int uses[2] = {0, 0};  // groups issued on B buffer b (= completions of its empty barrier)
  int cur = 0;           // B buffer of the next tile
  int nx = 0, nstep = 0, na = 0;

  for (;;) {
    if (t == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    if (item >= nitems || sh_bad) break;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    const FactorPtr<float2> f = factor_ptr<float2>(g, (char*)arena + d.factor_off);

    if (warp == 4) {
      // ================= the MMA warp: the step sequence of the sweeps, products only =================
      uint64_t da[3];
      for (int p = 0; p < 3; ++p) da[p] = sw64_desc(smem_u32(Abuf + p * kABytes));
      // the next tile's group into TMEM column dcol once its operands are in place
      auto group = [&](uint32_t dcol, bool accumulate, bool wait_a, bool commit_x, bool commit_step) -> bool {
        if (wait_a && !wwait(bar(kBarAFull), ++na)) return false;
        const int b = cur;
        if (!wwait(bar(kBarFull0 + b), uses[b] + 1)) return false;
        tc_fence_after();
        if (lane == 0) {
          uint64_t db[3];
          for (int p = 0; p < 3; ++p) db[p] = sw64_desc(smem_u32(Bof(b) + p * kBBytes));
          mma_group(tbase + dcol, da, db, accumulate);
          tc_commit(bar(kBarEmpty0 + b));
          if (commit_x) tc_commit(bar(kBarX));
          if (commit_step) tc_commit(bar(kBarStep));
        }
        __syncwarp();
        uses[b] += 1;
        cur ^= 1;
        return true;
      };
      bool ok = true;
      if (TRANS == 0) {
        for (int K = 0; K < Nb && ok; ++K) {  // forward: x_K into the scratch block, then block K+q
          const int nbb = min(bt, Nb - 1 - K), kmod = K % ringw;
          ok = group(scratch, false, true, true, nbb == 0);
          for (int q = 1; q <= nbb && ok; ++q) {
            const int sl = kmod + q;
            ok = group((uint32_t)(64 * (sl >= ringw ? sl - ringw : sl)), true, q == 1, false, q == nbb);
          }
        }
        for (int K = Nb - 1; K >= 0 && ok; --K) {  // backward: x_K in place, then block K-q
          const int nq = min(rings, K);
          ok = group((uint32_t)(64 * (K % rings)), false, true, true, nq == 0);
          for (int q = 1; q <= nq && ok; ++q)
            ok = group((uint32_t)(64 * ((K - q) % rings)), true, q == 1, false, q == nq);
        }
      } else {
        for (int K = 0; K < Nb && ok; ++K) {  // adjoint forward: w_K in place, then block K+q
          const int nq = min(rings, Nb - 1 - K);
          ok = group((uint32_t)(64 * (K % rings)), false, true, true, nq == 0);
          for (int q = 1; q <= nq && ok; ++q)
            ok = group((uint32_t)(64 * ((K + q) % rings)), true, q == 1, false, q == nq);
        }
      }
    } else {
      // ================= compute warps =================
      const int col = w.y + t;
      const bool valid = col < d.ncols;
      const float2* Y = rhs + d.rhs_off + (int64_t)(valid ? col : 0) * n;
      float2* X = out + (TRANS == 0 ? d.out_off : d.out2_off) + (int64_t)(valid ? col : 0) * n;
      auto tile_of = [&](int I, int J) { return f.tiles + g.tile_index(I, J) * te; };
      auto slot = [&](int q) { return slots + (size_t)q * kSlotBytes; };
      auto permbuf = [&](int K) { return perm_base + (size_t)(2 * warp + (K & 1)) * Pmax; };
      BOffsets boff;
      boff.init();
      float v[64], x[64];
      bool ok = true;
      // this warp's part of tile T into slot q, as one cp.async group (with P_K if given)
      auto stage = [&](int q, const float2* T, int Kperm) {
        stage_tile_warp<TRANS == 1>(smem_u32(slot(q)), T, warp, lane);
        if (Kperm >= 0) stage_bytes_warp(smem_u32(permbuf(Kperm)), f.perm + (int64_t)Kperm * Pmax, 2 * Pmax, lane);
        cp_async_commit();
      };
      // B buffer `cur` <- staged tile q (scaled by s) once the tile has landed and the buffer's last
      // group is done; then the slot's refill for the next step goes out.  `later` = groups of the
      // previous step staged after tile q, `cnt` = groups this step has staged so far.
      auto put_tile = [&](int q, int later, int& cnt, float s, const float2* refill, int Kperm) -> bool {
        cp_async_wait_pending(later - q + cnt);
        __syncwarp();
        const int b = cur;
        if (uses[b] > 0 && !wwait(bar(kBarEmpty0 + b), uses[b])) return false;
        TileRegs tr;
        tile_from_slot<TRANS == 1>(tr, slot(q));
        write_b(Bof(b), tr, s, boff);
        proxy_fence();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kBarFull0 + b));
        uses[b] += 1;
        cur ^= 1;
        if (refill) {
          stage(q, refill, Kperm);
          ++cnt;
        }
        return true;
      };
      // A <- this thread's 64 values, then handed to the MMA warp (with every TMEM access before it)
      auto put_a = [&](const float (&a)[64]) {
        write_a_row(Abuf, t, a);
        proxy_fence();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kBarAFull));
      };
      auto wait_step = [&]() -> bool {
        if (nstep > 0 && !wwait(bar(kBarStep), nstep)) return false;
        tc_fence_after();
        return true;
      };
      auto wait_x = [&]() -> bool {
        if (!wwait(bar(kBarX), ++nx)) return false;
        tc_fence_after();
        return true;
      };

      if (TRANS == 0) {
        // ======================= forward: P, L =======================
        const int n0 = min(bt, Nb - 1);
        stage(0, f.inv, 0);  // step 0: Linv_0 with P_0, then L(q, 0), one group each
        for (int q = 1; q <= n0; ++q) stage(q, tile_of(q, 0), -1);
        for (int q = 0; q <= n0; ++q) {
          blk_from_global(v, Y, n, (int64_t)q * kTile, valid);
          blk_to_tm(v, tb + (uint32_t)(64 * (q % ringw)));
        }
        for (int K = 0; K < Nb && ok; ++K) {
          const int nbb = min(bt, Nb - 1 - K);
          const int nb1 = K + 1 < Nb ? min(bt, Nb - 2 - K) : -1;  // the next step's update count
          const int kmod = K % ringw;
          auto bcol = [&](int j) -> uint32_t {  // TMEM column of window block j (0 <= j <= bt)
            const int sl = kmod + j;
            return (uint32_t)(64 * (sl >= ringw ? sl - ringw : sl));
          };
          const uint32_t top = (uint32_t)(64 * kmod);
          int cnt = 0;
          // Linv_K into B while the previous step's last products run (with P_K; refilled with
          // Linv_{K+1} and P_{K+1})
          if (!put_tile(0, nbb, cnt, 1.f, nb1 >= 0 ? f.inv + (int64_t)(2 * (K + 1)) * te : nullptr, K + 1)) {
            ok = false;
            break;
          }
          if (K + 2 < Nb) {  // step K+2's tiles and permutation, step K+1's entering block toward L2
            l2_prefetch_tile(f.inv + (int64_t)(2 * (K + 2)) * te, warp, lane);
            for (int q = 1; q <= min(bt, Nb - 3 - K); ++q) l2_prefetch_tile(tile_of(K + 2 + q, K + 2), warp, lane);
            if (warp == 0 && 128 * lane < 2 * Pmax)
              asm volatile("prefetch.global.L2 [%0];" ::"l"((const char*)(f.perm + (int64_t)(K + 2) * Pmax) + 128 * lane));
            l2_prefetch_rows(Y, n, (int64_t)(K + bt + 2) * kTile, valid);
          }
          if (!wait_step()) { ok = false; break; }
          // P_K on the window, in TMEM: new row r = old row perm[r].  The top rows gather (lane r
          // holds perm[r]); a row below the top changes only by receiving an old top row.
          const int16_t* pm = permbuf(K);
          const int pl = pm[lane];
          const unsigned moved = __ballot_sync(~0u, pl != lane);
          blk_from_tm(v, tb + top);
          if (moved) {
            uint32_t ur[32], ui[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) {
              const int sr = __shfl_sync(~0u, pl, r);
              ur[r] = ui[r] = 0u;
              if ((moved >> r) & 1u) {
                const uint32_t a = tb + bcol(sr >> 5) + (uint32_t)(sr & 31);
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
            for (int r = 0; r < 32; ++r)
              if ((moved >> r) & 1u) {
                v[r] = __uint_as_float(ur[r]);
                v[32 + r] = __uint_as_float(ui[r]);
              }
          }
          for (int j = 1; j <= nbb; ++j) {  // rows 32 j + l that receive old top row perm[32 j + l]
            const int pj = pm[32 * j + lane];
            unsigned m = __ballot_sync(~0u, pj < 32);
            const uint32_t dcol = tb + bcol(j);
            while (m) {  // up to 8 rows per batch (m is warp-uniform)
              uint32_t va[16];
              int dl[8], nb = 0;
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                va[u] = va[8 + u] = 0u;
                dl[u] = 0;
                if (m) {
                  const int l = __ffs(m) - 1;
                  m &= m - 1;
                  const int sr = __shfl_sync(~0u, pj, l);
                  dl[u] = l;
                  va[u] = tm_ld1(tb + top + (uint32_t)sr);
                  va[8 + u] = tm_ld1(tb + top + 32u + (uint32_t)sr);
                  nb = u + 1;
                }
              }
              tm_wait_ld();
              reg_fence16(va);
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (u < nb) {
                  tm_st1(dcol + (uint32_t)dl[u], va[u]);
                  tm_st1(dcol + 32u + (uint32_t)dl[u], va[8 + u]);
                }
            }
          }
          tm_wait_st();
          put_a(v);  // g = P_K rows of the top block; x_K = Linv_K g goes to the scratch block
          if (nbb >= 1 && !put_tile(1, nbb, cnt, -1.f, 1 <= nb1 ? tile_of(K + 2, K + 1) : nullptr, -1)) {
            ok = false;
            break;
          }
          // block K+bt+1 of Y enters the slot block K leaves (no product of this step writes it); its
          // loads are in flight during the products
          const bool enter = K + bt + 1 < Nb;
          if (enter) blk_from_global(v, Y, n, (int64_t)(K + bt + 1) * kTile, valid);
          if (!wait_x()) { ok = false; break; }
          blk_from_tm(x, tb + scratch);
          if (nbb >= 1) put_a(x);
          const int parts = nbb - 1;
          for (int q = 2; q <= nbb; ++q) {
            if (!put_tile(q, nbb, cnt, -1.f, q <= nb1 ? tile_of(K + 1 + q, K + 1) : nullptr, -1)) {
              ok = false;
              break;
            }
            blk_to_global(x, X, n, (int64_t)K * kTile, valid, 16 * (q - 2) / parts, 16 * (q - 1) / parts);
          }
          if (!ok) break;
          if (parts <= 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid, 0, 16);
          if (enter) blk_to_tm(v, tb + top);
          ++nstep;
        }
        if (ok) {
          // ======================= backward: U =======================
          const int n0b = min(rings, Nb - 1);
          if (!wait_step()) ok = false;
          if (ok) {
            stage(0, f.inv + (int64_t)(2 * (Nb - 1) + 1) * te, -1);  // step Nb-1: Uinv, U(Nb-1-q, Nb-1)
            for (int q = 1; q <= n0b; ++q) stage(q, tile_of(Nb - 1 - q, Nb - 1), -1);
            for (int J = Nb - 1; J >= max(0, Nb - rings); --J) {  // pending blocks start as the forward result
              blk_from_global(v, X, n, (int64_t)J * kTile, valid);
              blk_to_tm(v, tb + (uint32_t)(64 * (J % rings)));
            }
          }
          for (int K = Nb - 1; K >= 0 && ok; --K) {
            const int nq = min(rings, K);
            const int nq1 = K >= 1 ? min(rings, K - 1) : -1;
            const uint32_t sk = (uint32_t)(64 * (K % rings));
            int cnt = 0;
            if (!put_tile(0, nq, cnt, 1.f, nq1 >= 0 ? f.inv + (int64_t)(2 * (K - 1) + 1) * te : nullptr, -1)) {
              ok = false;
              break;
            }
            if (K >= 2) {  // step K-2's tiles, step K-1's entering block toward L2
              l2_prefetch_tile(f.inv + (int64_t)(2 * (K - 2) + 1) * te, warp, lane);
              for (int q = 1; q <= min(rings, K - 2); ++q) l2_prefetch_tile(tile_of(K - 2 - q, K - 2), warp, lane);
              if (K - 1 - rings >= 0) l2_prefetch_rows(X, n, (int64_t)(K - 1 - rings) * kTile, valid);
            }
            if (!wait_step()) { ok = false; break; }
            blk_from_tm(v, tb + sk);  // acc_K is complete
            put_a(v);
            if (nq >= 1 && !put_tile(1, nq, cnt, -1.f, 1 <= nq1 ? tile_of(K - 2, K - 1) : nullptr, -1)) {
              ok = false;
              break;
            }
            // block K-2bt enters the slot K leaves; the last update (q = 2bt) accumulates into it
            const bool enter = K - rings >= 0;
            if (enter) blk_from_global(v, X, n, (int64_t)(K - rings) * kTile, valid);
            if (!wait_x()) { ok = false; break; }
            blk_from_tm(x, tb + sk);
            if (nq >= 1) put_a(x);
            const int parts = nq - 1;
            for (int q = 2; q <= nq; ++q) {
              if (enter && q == nq) blk_to_tm(v, tb + sk);
              if (!put_tile(q, nq, cnt, -1.f, q <= nq1 ? tile_of(K - 1 - q, K - 1) : nullptr, -1)) {
                ok = false;
                break;
              }
              blk_to_global(x, X, n, (int64_t)K * kTile, valid, 16 * (q - 2) / parts, 16 * (q - 1) / parts);
            }
            if (!ok) break;
            if (parts <= 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid, 0, 16);
            ++nstep;
          }
        }
      } else {
        // ======================= adjoint forward: U^H =======================
        const int n0 = min(rings, Nb - 1);
        stage(0, f.inv + te, -1);  // step 0: Uinv_0^H, then U(0, q)^H
        for (int q = 1; q <= n0; ++q) stage(q, tile_of(0, q), -1);
        for (int J = 0; J < min(rings, Nb); ++J) {  // pending blocks start as y
          blk_from_global(v, Y, n, (int64_t)J * kTile, valid);
          blk_to_tm(v, tb + (uint32_t)(64 * (J % rings)));
        }
        for (int K = 0; K < Nb && ok; ++K) {
          const int nq = min(rings, Nb - 1 - K);
          const int nq1 = K + 1 < Nb ? min(rings, Nb - 2 - K) : -1;
          const uint32_t sk = (uint32_t)(64 * (K % rings));
          int cnt = 0;
          if (!put_tile(0, nq, cnt, 1.f, nq1 >= 0 ? f.inv + (int64_t)(2 * (K + 1) + 1) * te : nullptr, -1)) {
            ok = false;
            break;
          }
          if (K + 2 < Nb) {  // step K+2's tiles, step K+1's entering block toward L2
            l2_prefetch_tile(f.inv + (int64_t)(2 * (K + 2) + 1) * te, warp, lane);
            for (int q = 1; q <= min(rings, Nb - 3 - K); ++q) l2_prefetch_tile(tile_of(K + 2, K + 2 + q), warp, lane);
            if (K + 1 + rings < Nb) l2_prefetch_rows(Y, n, (int64_t)(K + 1 + rings) * kTile, valid);
          }
          if (!wait_step()) { ok = false; break; }
          blk_from_tm(v, tb + sk);
          put_a(v);
          if (nq >= 1 && !put_tile(1, nq, cnt, -1.f, 1 <= nq1 ? tile_of(K + 1, K + 2) : nullptr, -1)) {
            ok = false;
            break;
          }
          // block K+2bt enters the slot K leaves; the last update (q = 2bt) accumulates into it
          const bool enter = K + rings < Nb;
          if (enter) blk_from_global(v, Y, n, (int64_t)(K + rings) * kTile, valid);
          if (!wait_x()) { ok = false; break; }
          blk_from_tm(x, tb + sk);
          if (nq >= 1) put_a(x);
          const int parts = nq - 1;
          for (int q = 2; q <= nq; ++q) {
            if (enter && q == nq) blk_to_tm(v, tb + sk);
            if (!put_tile(q, nq, cnt, -1.f, q <= nq1 ? tile_of(K + 1, K + 1 + q) : nullptr, -1)) {
              ok = false;
              break;
            }
            blk_to_global(x, X, n, (int64_t)K * kTile, valid, 16 * (q - 2) / parts, 16 * (q - 1) / parts);
          }
          if (!ok) break;
          if (parts <= 0) blk_to_global(x, X, n, (int64_t)K * kTile, valid, 0, 16);
          ++nstep;
        }
      }
      // the item's last products are complete before the next item reuses TMEM
      if (ok && !wait_step()) ok = false;
      cp_async_wait_pending(0);
    }
    // item end: every warp, successful or not, meets here (a failure is in sh_bad)
    __syncthreads();
  }
  // drain: every product issued is complete (bounded wait) before TMEM is released
  if (warp == 4) {
    if (lane == 0) tc_commit(bar(kBarDrain));
    __syncwarp();
    wait_k(bar(kBarDrain), 1, &sh_bad, false);
    __syncwarp();
  }
  cp_async_wait_pending(0);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(512u));
}

// ---------------------------------------------------------------------------
// The adjoint backward sweep (L^H with the inverse interchanges), left-looking:
//   v_K = w_K + sum_q (-L(K+q, K)^H) w_{K+q}    (q = 1..bt, the window's current blocks)
//   x_K = Linv_K^H v_K,  then P_K^T on the window (blocks K..K+bt)
// Every product is a bf16x6 MMA group into a fresh TMEM accumulator (the sum of the step's
// update products, then x_K), so the window blocks themselves are only written by the compute
// warps (round-to-nearest add of the sum to w_K).  A and B of each group go together into one of
// two operand pairs (full/empty mbarriers).  Factor tiles of the next step are staged per warp by
// cp.async in consumption order (the update tiles, then Linv with the permutation).
// ---------------------------------------------------------------------------
constexpr int kPairBytes = 3 * kABytes + 3 * kBBytes;  // A and B, three bf16 parts each: 72 KiB
enum { kQFull0 = 0, kQFull1, kQEmpty0, kQEmpty1, kQX, kQStep, kQDrain, kQNumBars };

__global__ void __launch_bounds__(kTcThreads, 1)
    solve_tca_kernel(FactorGeom g, const SysDesc* sys, const char* arena, float2* out, const int2* items,
                     int nitems, int* counter) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  auto pairA = [&](int p) { return sm + (size_t)p * kPairBytes; };
  auto pairB = [&](int p) { return sm + (size_t)p * kPairBytes + 3 * kABytes; };
  unsigned char* slots = sm + 2 * (size_t)kPairBytes;        // bt + 1 staged tiles: Linv, L(K+q, K)
  const int Pmax = (g.bt + 1) * kTile;
  int16_t* perm_base = (int16_t*)(slots + (size_t)(g.bt + 1) * kSlotBytes);  // [warp][2][Pmax]
  int16_t* invp_base = perm_base + 8 * Pmax;                                  // [warp][32]
  uint64_t* bars = (uint64_t*)(((uintptr_t)(invp_base + 4 * 32) + 7) & ~(uintptr_t)7);
  __shared__ uint32_t tslot;
  __shared__ int sh_item;
  __shared__ volatile int sh_bad;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto bar = [&](int i) { return smem_u32(bars + i); };
  const int polls = g_tc_solve_polls;
  auto wwait = [&](uint32_t b, int k) -> bool { return __all_sync(~0u, wait_k(b, k, &sh_bad, true, polls)) != 0; };
  if (t == 0) {
    for (int i = 0; i < kQNumBars; ++i) mbar_init(bar(i), (i == kQFull0 || i == kQFull1) ? 4u : 1u);
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
  const uint32_t tbase = tslot;
  const uint32_t tb = tslot + ((uint32_t)(32 * (warp & 3)) << 16);
  const int bt = g.bt, Nb = g.Nb;
  const int64_t n = g.n, te = g.tile_elems;
  const int ringw = bt + 1;
  const uint32_t scratch = (uint32_t)(64 * ringw);  // the step's accumulator
  int uses[2] = {0, 0};                              // groups issued on operand pair p
  int cur = 0;                                       // operand pair of the next group
  int nx = 0, nstep = 0;

  for (;;) {
    if (t == 0) sh_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sh_item;
    if (item >= nitems || sh_bad) break;
    const int2 w = items[item];
    const SysDesc d = sys[w.x];
    const FactorPtr<float2> f = factor_ptr<float2>(g, (char*)arena + d.factor_off);

    if (warp == 4) {
      // ================= the MMA warp =================
      auto group = [&](bool accumulate, bool commit_x, bool commit_step) -> bool {
        const int p = cur;
        if (!wwait(bar(kQFull0 + p), uses[p] + 1)) return false;
        tc_fence_after();
        if (lane == 0) {
          uint64_t da[3], db[3];
          for (int q = 0; q < 3; ++q) {
            da[q] = sw64_desc(smem_u32(pairA(p) + q * kABytes));
            db[q] = sw64_desc(smem_u32(pairB(p) + q * kBBytes));
          }
          mma_group(tbase + scratch, da, db, accumulate);
          tc_commit(bar(kQEmpty0 + p));
          if (commit_x) tc_commit(bar(kQX));
          if (commit_step) tc_commit(bar(kQStep));
        }
        __syncwarp();
        uses[p] += 1;
        cur ^= 1;
        return true;
      };
      bool ok = true;
      for (int K = Nb - 1; K >= 0 && ok; --K) {
        const int nb = min(bt, Nb - 1 - K);
        for (int q = 1; q <= nb && ok; ++q) ok = group(q > 1, q == nb, false);
        if (ok) ok = group(false, false, true);
      }
    } else {
      // ================= compute warps =================
      const int col = w.y + t;
      const bool valid = col < d.ncols;
      float2* X = out + d.out2_off + (int64_t)(valid ? col : 0) * n;
      auto tile_of = [&](int I, int J) { return f.tiles + g.tile_index(I, J) * te; };
      auto slot = [&](int q) { return slots + (size_t)q * kSlotBytes; };
      auto permbuf = [&](int K) { return perm_base + (size_t)(2 * warp + (K & 1)) * Pmax; };
      int16_t* invp = invp_base + 32 * warp;
      BOffsets boff;
      boff.init();
      float v[64], x[64];
      bool ok = true;
      auto scol = [&](int J) { return (uint32_t)(64 * (J % ringw)); };
      auto stage = [&](int q, const float2* T, int Kperm) {
        stage_tile_warp<true>(smem_u32(slot(q)), T, warp, lane);
        if (Kperm >= 0) stage_bytes_warp(smem_u32(permbuf(Kperm)), f.perm + (int64_t)Kperm * Pmax, 2 * Pmax, lane);
        cp_async_commit();
      };
      // operand pair `cur` <- A (this thread's 64 values) and B (staged tile q scaled by s), once
      // the pair's last group is done; the MMA warp takes it when all four warps arrived
      auto put_pair = [&](const float (&a)[64], int q, float s) -> bool {
        const int p = cur;
        if (uses[p] > 0 && !wwait(bar(kQEmpty0 + p), uses[p])) return false;
        write_a_row(pairA(p), t, a);
        TileRegs tr;
        tile_from_slot<true>(tr, slot(q));
        write_b(pairB(p), tr, s, boff);
        proxy_fence();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(kQFull0 + p));
        uses[p] += 1;
        cur ^= 1;
        return true;
      };
      // the first step (K = Nb-1, no updates): Linv_{Nb-1} with P_{Nb-1}
      stage(0, f.inv + (int64_t)(2 * (Nb - 1)) * te, Nb - 1);
      for (int K = Nb - 1; K >= 0 && ok; --K) {
        const int nb = min(bt, Nb - 1 - K);
        const int nbp = K + 1 < Nb ? min(bt, Nb - 2 - K) : 0;  // tiles the previous step consumed
        const int nbn = K >= 1 ? min(bt, Nb - K) : -1;         // the next step's update count
        const uint32_t sk = scol(K);
        int cnt = 0;
        // the next step's update tile that this step does not use goes out first
        for (int q = nb + 1; q <= nbn; ++q) {
          stage(q, tile_of(K - 1 + q, K - 1), -1);
          ++cnt;
        }
        // block K+bt+1 leaves the window (final); w_K enters its slot
        if (K + bt + 1 < Nb) {
          blk_from_tm(x, tb + sk);
          blk_to_global(x, X, n, (int64_t)(K + bt + 1) * kTile, valid, 0, 16);
        }
        blk_from_global(v, X, n, (int64_t)K * kTile, valid);
        // the update products: A = window block K+q, B = -L(K+q, K)^H
        for (int q = 1; q <= nb && ok; ++q) {
          cp_async_wait_pending(max(nbp - q, 0) + 1 + cnt);
          __syncwarp();
          blk_from_tm(x, tb + scol(K + q));
          if (!put_pair(x, q, -1.f)) { ok = false; break; }
          if (q <= nbn) {
            stage(q, tile_of(K - 1 + q, K - 1), -1);
            ++cnt;
          }
        }
        if (!ok) break;
        if (nb >= 1) {  // v_K = w_K + the products' sum (round to nearest)
          if (!wwait(bar(kQX), ++nx)) { ok = false; break; }
          tc_fence_after();
          blk_from_tm(x, tb + scratch);
#pragma unroll
          for (int i = 0; i < 64; ++i) v[i] += x[i];
        }
        // x_K = Linv_K^H v_K
        cp_async_wait_pending(cnt);
        __syncwarp();
        if (!put_pair(v, 0, 1.f)) { ok = false; break; }
        if (K >= 1) {
          stage(0, f.inv + (int64_t)(2 * (K - 1)) * te, K - 1);
          ++cnt;
        }
        if (!wwait(bar(kQStep), ++nstep)) { ok = false; break; }
        tc_fence_after();
        blk_from_tm(x, tb + scratch);
        blk_to_tm(x, tb + sk);
        // P_K^T on the window (blocks K..K+nb): new row t = old row invp[t]; the rows below that
        // receive (old top rows perm[r] >= 32) are exactly those whose values move up
        const int16_t* pm = permbuf(K);
        const int P = (nb + 1) * kTile;
        for (int r = lane; r < P; r += 32) {
          const int dst = pm[r];
          if (dst < 32) invp[dst] = (int16_t)r;
        }
        __syncwarp();
        const int pl = invp[lane], pr = pm[lane];
        const unsigned moved = __ballot_sync(~0u, pl != lane);
        const unsigned down = __ballot_sync(~0u, pr >= 32);
        auto bcol = [&](int j) { return scol(K + j); };
        if (moved) {
          uint32_t ur[32], ui[32];
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int sr = __shfl_sync(~0u, pl, r);
            ur[r] = ui[r] = 0u;
            if ((moved >> r) & 1u) {
              const uint32_t a = tb + bcol(sr >> 5) + (uint32_t)(sr & 31);
              ur[r] = tm_ld1(a);
              ui[r] = tm_ld1(a + 32);
            }
          }
          tm_wait_ld();
          reg_fence16(*(uint32_t(*)[16])&ur[0]);
          reg_fence16(*(uint32_t(*)[16])&ur[16]);
          reg_fence16(*(uint32_t(*)[16])&ui[0]);
          reg_fence16(*(uint32_t(*)[16])&ui[16]);
          // rows below receive old top rows (from x, still in registers as the old top block)
          unsigned m = down;
          while (m) {  // up to 8 rows per batch (warp-uniform)
            uint32_t va[16];
            int dr[8], nbt = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              va[u] = va[8 + u] = 0u;
              dr[u] = 0;
              if (m) {
                const int r = __ffs(m) - 1;
                m &= m - 1;
                dr[u] = __shfl_sync(~0u, pr, r);
                va[u] = tm_ld1(tb + sk + (uint32_t)r);
                va[8 + u] = tm_ld1(tb + sk + 32u + (uint32_t)r);
                nbt = u + 1;
              }
            }
            tm_wait_ld();
            reg_fence16(va);
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (u < nbt) {
                const uint32_t a = tb + bcol(dr[u] >> 5) + (uint32_t)(dr[u] & 31);
                tm_st1(a, va[u]);
                tm_st1(a + 32, va[8 + u]);
              }
          }
#pragma unroll
          for (int r = 0; r < 32; ++r)
            if ((moved >> r) & 1u) {
              x[r] = __uint_as_float(ur[r]);
              x[32 + r] = __uint_as_float(ui[r]);
            }
          tm_wait_st();
          blk_to_tm(x, tb + sk);
        }
        __syncwarp();
      }
      if (ok) {  // the blocks left in the window are final
        for (int J = 0; J <= min(bt, Nb - 1); ++J) {
          blk_from_tm(x, tb + scol(J));
          blk_to_global(x, X, n, (int64_t)J * kTile, valid, 0, 16);
        }
      }
      cp_async_wait_pending(0);
    }
    __syncthreads();
  }
  if (warp == 4) {
    if (lane == 0) tc_commit(bar(kQDrain));
    __syncwarp();
    wait_k(bar(kQDrain), 1, &sh_bad, false);
    __syncwarp();
  }
  cp_async_wait_pending(0);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(512u));
}

}  // namespace

size_t solve_tc_smem_bytes(const FactorGeom& g) {
  const int Pmax = (g.bt + 1) * kTile;
  return 1024 + 3 * (size_t)kABytes + 6 * (size_t)kBBytes + (size_t)(2 * g.bt + 1) * kSlotBytes +
         8 * (size_t)Pmax * sizeof(int16_t) + 8 * kNumBars + 8;
}

size_t solve_tca_smem_bytes(const FactorGeom& g) {
  const int Pmax = (g.bt + 1) * kTile;
  return 1024 + 2 * (size_t)kPairBytes + (size_t)(g.bt + 1) * kSlotBytes + 8 * (size_t)Pmax * sizeof(int16_t) +
         4 * 32 * sizeof(int16_t) + 8 * kQNumBars + 8;
}

bool solve_tc_supported(const FactorGeom& g) {
  return g.bt >= 1 && 64 * 2 * g.bt <= 512 && 64 * (g.bt + 2) <= 512 && solve_tc_smem_bytes(g) <= 227 * 1024 &&
         solve_tca_smem_bytes(g) <= 227 * 1024;
}

int solve_tc_set_wait_polls(int polls) {
  const int v = polls > 0 ? polls : kPollLimit;
  PD_CK(cudaMemcpyToSymbol(g_tc_solve_polls, &v, sizeof(v)));
  return 0;
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
  if (((uintptr_t)factor_arena & 15) != 0) {  // the staged tile copies are 16-byte cp.async
    set_last_error_msg("factor workspace not 16-byte aligned");
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
    // the adjoint backward sweep (L^H with the inverse interchanges), left-looking
    const size_t smem2 = solve_tca_smem_bytes(g);
    PD_CK(cudaMemsetAsync(counter, 0, sizeof(int), st));
    PD_CK(cudaFuncSetAttribute(solve_tca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    solve_tca_kernel<<<grid, kTcThreads, smem2, st>>>(g, d_sys, factor_arena, out_arena, d_items, nitems, counter);
    PD_CK_LAUNCH();
    return 0;
  }
  PD_CK(cudaFuncSetAttribute(solve_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  solve_tc_kernel<0><<<grid, kTcThreads, smem, st>>>(g, d_sys, factor_arena, rhs_arena, out_arena, d_items, nitems,
                                                     counter);
  PD_CK_LAUNCH();
  return 0;
}

}  // namespace pdeshep
