// common.cuh -- device/host helpers shared by the sm_103a kernels of the
// banded FEAST library: complex arithmetic on float2/double2, a bump
// allocator over the caller's workspace, CUDA error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <type_traits>

#include "../../include/pdeshep.h"

namespace pdeshep {

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
void set_last_error(const char* where, cudaError_t e);
void set_last_error_msg(const char* msg);
// process-wide count of kernels launched by this library
void count_launch();
void count_launches(long long k);  // k kernels run by a graph launch (or -k captured but not run)
unsigned long long launches_so_far();

#define PD_CK(...)                                    \
  do {                                                \
    cudaError_t _e = (__VA_ARGS__);                   \
    if (_e != cudaSuccess) {                          \
      ::pdeshep::set_last_error(#__VA_ARGS__, _e);    \
      return PDESHEP_CUDA_ERROR;                      \
    }                                                 \
  } while (0)

#define PD_CK_LAUNCH()                                \
  do {                                                \
    ::pdeshep::count_launch();                        \
    cudaError_t _e = cudaGetLastError();              \
    if (_e != cudaSuccess) {                          \
      ::pdeshep::set_last_error("kernel launch", _e); \
      return PDESHEP_CUDA_ERROR;                      \
    }                                                 \
  } while (0)

#define PD_TRY(...)             \
  do {                          \
    int _st = (__VA_ARGS__);    \
    if (_st != 0) return _st;   \
  } while (0)

// ----------------------------------------------------------------------------
// workspace arena: carves 256-byte aligned sub-buffers out of the caller's
// device workspace.  With base == nullptr it only measures.
// ----------------------------------------------------------------------------
// SplitMix64 (Vigna): the state advanced by the golden-ratio increment, then
// mixed.  Counter-based use: value k of a stream is splitmix64(seed + k).
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Uniform double in [-1, 1) from the top 53 bits of a 64-bit word (exact: the
// 53-bit integer times 2^-52 minus 1 rounds nowhere).
__host__ __device__ inline double uniform_pm1(uint64_t v) {
  return (double)(int64_t)(v >> 11) * 0x1p-52 - 1.0;
}

struct Arena {
  char* base;
  size_t cap;
  size_t off;
  explicit Arena(void* b = nullptr, size_t c = 0) : base((char*)b), cap(c), off(0) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? (T*)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  bool fits() const { return off <= cap; }
  size_t used() const { return (off + 255) & ~size_t(255); }
};

// ----------------------------------------------------------------------------
// complex helpers on float2 / double2
// ----------------------------------------------------------------------------
template <typename R>
struct cx_of;
template <>
struct cx_of<float> {
  using type = float2;
};
template <>
struct cx_of<double> {
  using type = double2;
};

template <typename C>
struct real_of;
template <>
struct real_of<float2> {
  using type = float;
};
template <>
struct real_of<double2> {
  using type = double;
};

template <typename C>
__host__ __device__ __forceinline__ C cmk(typename real_of<C>::type re, typename real_of<C>::type im) {
  C r;
  r.x = re;
  r.y = im;
  return r;
}
template <typename C>
__host__ __device__ __forceinline__ C cadd(C a, C b) {
  return cmk<C>(a.x + b.x, a.y + b.y);
}
template <typename C>
__host__ __device__ __forceinline__ C csub(C a, C b) {
  return cmk<C>(a.x - b.x, a.y - b.y);
}
template <typename C>
__host__ __device__ __forceinline__ C cmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C>
__host__ __device__ __forceinline__ C cmulcj(C a, C b) {
  return cmk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C>
__host__ __device__ __forceinline__ C cconj(C a) {
  return cmk<C>(a.x, -a.y);
}
template <typename C>
__host__ __device__ __forceinline__ C cscale(C a, typename real_of<C>::type s) {
  return cmk<C>(a.x * s, a.y * s);
}
// acc += a * b
template <typename C>
__host__ __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b
template <typename C>
__host__ __device__ __forceinline__ void cfms(C& acc, C a, C b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C>
__host__ __device__ __forceinline__ void cfmacj(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= conj(a) * b
template <typename C>
__host__ __device__ __forceinline__ void cfmscj(C& acc, C a, C b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
template <typename C>
__host__ __device__ __forceinline__ typename real_of<C>::type cabs1(C a) {
  return fabs(a.x) + fabs(a.y);
}
// 1 / a with Smith's scaling
template <typename C>
__host__ __device__ __forceinline__ C crecip(C a) {
  using R = typename real_of<C>::type;
  if (fabs(a.x) >= fabs(a.y)) {
    R r = a.y / a.x, den = a.x + a.y * r;
    return cmk<C>(R(1) / den, -r / den);
  } else {
    R r = a.x / a.y, den = a.x * r + a.y;
    return cmk<C>(r / den, R(-1) / den);
  }
}

__host__ __device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }

// scalar-generic helpers for the FP64 dense kernels (double or double2)
template <typename S>
struct sc;
template <>
struct sc<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double conj(double a) { return a; }
  static __device__ __forceinline__ void fma_(double& acc, double a, double b) { acc = fma(a, b, acc); }
  // acc += conj(a) b
  static __device__ __forceinline__ void fmacj(double& acc, double a, double b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ double abs2(double a) { return a * a; }
  static __device__ __forceinline__ double absv(double a) { return fabs(a); }
  static __device__ __forceinline__ double re(double a) { return a; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double scale(double a, double s) { return a * s; }
  static __device__ __forceinline__ double from_re(double r) { return r; }
};
template <>
struct sc<double2> {
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 conj(double2 a) { return make_double2(a.x, -a.y); }
  static __device__ __forceinline__ void fma_(double2& acc, double2 a, double2 b) { cfma(acc, a, b); }
  static __device__ __forceinline__ void fmacj(double2& acc, double2 a, double2 b) { cfmacj(acc, a, b); }
  static __device__ __forceinline__ double abs2(double2 a) { return a.x * a.x + a.y * a.y; }
  static __device__ __forceinline__ double absv(double2 a) { return hypot(a.x, a.y); }
  static __device__ __forceinline__ double re(double2 a) { return a.x; }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) { return cmul(a, b); }
  static __device__ __forceinline__ double2 sub(double2 a, double2 b) { return csub(a, b); }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return cadd(a, b); }
  static __device__ __forceinline__ double2 scale(double2 a, double s) { return cscale(a, s); }
  static __device__ __forceinline__ double2 from_re(double r) { return make_double2(r, 0.0); }
};

template <>
struct sc<float> {
  static __device__ __forceinline__ float zero() { return 0.0f; }
  static __device__ __forceinline__ float conj(float a) { return a; }
  static __device__ __forceinline__ void fma_(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
  static __device__ __forceinline__ float abs2(float a) { return a * a; }
  static __device__ __forceinline__ float absv(float a) { return fabsf(a); }
  static __device__ __forceinline__ float re(float a) { return a; }
  static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float scale(float a, float s) { return a * s; }
  static __device__ __forceinline__ float from_re(float r) { return r; }
};
template <>
struct sc<float2> {
  static __device__ __forceinline__ float2 zero() { return make_float2(0.0f, 0.0f); }
  static __device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
  static __device__ __forceinline__ void fma_(float2& acc, float2 a, float2 b) { cfma(acc, a, b); }
  static __device__ __forceinline__ float abs2(float2 a) { return a.x * a.x + a.y * a.y; }
  static __device__ __forceinline__ float absv(float2 a) { return hypotf(a.x, a.y); }
  static __device__ __forceinline__ float re(float2 a) { return a.x; }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return cmul(a, b); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return csub(a, b); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return cadd(a, b); }
  static __device__ __forceinline__ float2 scale(float2 a, float s) { return cscale(a, s); }
  static __device__ __forceinline__ float2 from_re(float r) { return make_float2(r, 0.0f); }
};

// real type of a scalar (double for double/double2, float for float/float2)
template <typename S>
struct real_t {
  using type = double;
};
template <>
struct real_t<float> {
  using type = float;
};
template <>
struct real_t<float2> {
  using type = float;
};
// single-precision counterpart of an FP64 scalar type
template <typename S>
struct lowp;
template <>
struct lowp<double> {
  using type = float;
};
template <>
struct lowp<double2> {
  using type = float2;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace pdeshep
