// band_lu.cuh -- tiled layout of the shifted band LU factors and the host
// entry points of the factor / solve / accumulate kernels (band_lu.cu).
#pragma once
#include "common.cuh"

namespace pdeshep {

constexpr int kTile = 32;  // T: tile edge of the block-banded factor

// Factor of z I - B for one shift, in T x T tiles.  With bt = ceil(b/T)
// (block semi-bandwidth) and Nb = ceil(n/T) block rows, block row I keeps
// the 3bt+1 tiles (I, J), J in [I-bt, I+2bt], at tile index
// I*(3bt+1) + (J - I + bt), each column-major T x T.  After factorization the
// tiles left of the diagonal hold L multipliers, the diagonal tile holds the
// packed unit-L\U of the panel's top block, right of it U (fill to 2b).
// Per block row K also: the inverse of the unit lower diagonal block (Linv),
// of the upper diagonal block (Uinv), and the composed row permutation of the
// panel (perm[r] = original window row now at window row r, r < (bt+1)T).
struct FactorGeom {
  int64_t n;
  int b, T, bt, Nb, nslot;
  int64_t tile_elems;  // T*T
  int64_t tiles;       // Nb * nslot
  int64_t perm_len;    // Nb * (bt+1)*T
  __host__ __device__ int64_t tile_index(int I, int J) const { return (int64_t)I * nslot + (J - I + bt); }
};

inline FactorGeom make_geom(int64_t n, int b) {
  FactorGeom g;
  g.n = n;
  g.b = b;
  g.T = kTile;
  g.bt = b > 0 ? (int)ceil_div(b, kTile) : 1;
  g.Nb = (int)ceil_div(n, kTile);
  g.nslot = 3 * g.bt + 1;
  g.tile_elems = (int64_t)kTile * kTile;
  g.tiles = (int64_t)g.Nb * g.nslot;
  g.perm_len = (int64_t)g.Nb * (g.bt + 1) * kTile;
  return g;
}

// Byte size of one factor (tiles + Linv/Uinv + permutation) for element size es.
inline size_t factor_bytes(const FactorGeom& g, size_t es) {
  size_t t = (size_t)(g.tiles * g.tile_elems) * es;
  size_t inv = (size_t)g.Nb * 2 * g.tile_elems * es;
  size_t perm = (size_t)g.perm_len * sizeof(int16_t);
  return ((t + 255) & ~size_t(255)) + ((inv + 255) & ~size_t(255)) + ((perm + 255) & ~size_t(255));
}

// Device-side pointers of one factor inside a contiguous factor block.
template <typename C>
struct FactorPtr {
  C* tiles;
  C* inv;  // block K: Linv at inv + 2K*T*T, Uinv at inv + (2K+1)*T*T
  int16_t* perm;
};

template <typename C>
__host__ __device__ inline FactorPtr<C> factor_ptr(const FactorGeom& g, char* base) {
  FactorPtr<C> f;
  size_t t = (size_t)(g.tiles * g.tile_elems) * sizeof(C);
  size_t inv = (size_t)g.Nb * 2 * g.tile_elems * sizeof(C);
  f.tiles = (C*)base;
  f.inv = (C*)(base + ((t + 255) & ~size_t(255)));
  f.perm = (int16_t*)(base + ((t + 255) & ~size_t(255)) + ((inv + 255) & ~size_t(255)));
  return f;
}

// One linear system of a batch: factor block, shift, right-hand sides and output.
struct SysDesc {
  int64_t factor_off;  // byte offset of the factor in the factor arena
  double zre, zim;     // shift
  int64_t rhs_off;     // element offset of Y (n x ncols, ld n) in the rhs arena
  int64_t out_off;     // element offset of X = (zI-B)^{-1} Y in the output arena
  int64_t out2_off;    // element offset of X = (zI-B)^{-H} Y in the output arena
  int32_t ncols;
  int32_t pad;
};

// Kernel launchers (async on `st`).  C is float2 (mixed) or double2 (fp64).
// band: FP64 lower band (double or double2 if cplx).  status: int per system,
// set to k+1 on an exactly zero pivot at column k.  ipiv: optional nsys x n.
template <typename C>
int launch_factor(const FactorGeom& g, int cplx, const void* band, int64_t ldab, int nsys,
                  const SysDesc* d_sys, char* factor_arena, int* d_status, int32_t* d_ipiv,
                  cudaStream_t st);

// trans = 0: X = (zI-B)^{-1} Y;  trans = 1: X = (zI-B)^{-H} Y.  Y and X hold C.
// h_sys: the same descriptors on the host (their column counts build the work
// list).  chunk: right-hand sides per work item (16, 32 or 64; 0 = 32; 128 = the
// tensor-memory kernel of solve_tm.cu, complex64 only).
// queue: device scratch of solve_queue_bytes(nsys, max columns).
template <typename C>
int launch_solve(const FactorGeom& g, int trans, int nsys, const SysDesc* h_sys, const SysDesc* d_sys,
                 const char* factor_arena, const C* rhs_arena, C* out_arena, int chunk, void* queue,
                 cudaStream_t st);

// The same in two steps: the work list is uploaded once (a host-to-device
// copy, outside any stream capture), then launches replay it (capturable).
int upload_solve_items(int nsys, const SysDesc* h_sys, int chunk, void* queue, cudaStream_t st, int* nitems);
template <typename C>
int launch_solve_queued(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                        const C* rhs_arena, C* out_arena, int chunk, void* queue, cudaStream_t st);

size_t solve_smem_bytes(const FactorGeom& g, int chunk, size_t es, int trans);
size_t solve_queue_bytes(int nsys, int max_cols);

// complex64 solves with one thread per right-hand side and the window in tensor memory
// (solve_tm.cu): work items of kTmChunk columns; bands with bt <= 4 (b <= 128).
constexpr int kTmChunk = 128;
bool solve_tm_supported(const FactorGeom& g);
size_t solve_tm_smem_bytes(const FactorGeom& g);
// complex64 solves with the tile products on the tcgen05 tensor cores (solve_tc.cu; bf16x6):
// work items of kTmChunk columns, selected as the column block kTcChunk; b <= 128.
constexpr int kTcChunk = 256;
bool solve_tc_supported(const FactorGeom& g);
size_t solve_tc_smem_bytes(const FactorGeom& g);
int launch_solve_tc(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                    const float2* rhs_arena, float2* out_arena, void* queue, cudaStream_t st);
// the error word of the tensor-core solve (a bounded wait gave up): read into *h_err (synchronous) and/or clear
int solve_tc_error(int* h_err, int clear, cudaStream_t st);
int solve_tc_set_wait_polls(int polls);  // 0: the default
// sweep0/sweep1: the sweeps [sweep0, sweep1) of each item (0: forward, 1: backward; default both)
int launch_solve_tm(const FactorGeom& g, int trans, int nitems, const SysDesc* d_sys, const char* factor_arena,
                    const float2* rhs_arena, float2* out_arena, void* queue, cudaStream_t st, int sweep0 = 0,
                    int sweep1 = 2);

}  // namespace pdeshep
