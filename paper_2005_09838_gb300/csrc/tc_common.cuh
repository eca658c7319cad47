// Shared device types and helpers of the TCTF2R CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

// Complex value in (re, im) order; layout-compatible with float2 / double2.
template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cconjmul(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += a * conj(b)
template <typename T>
__host__ __device__ __forceinline__ void cfmac(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(-a.re, b.im, acc.im);
}
// acc += conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ void cfmaconj(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// Read-only cached load of a complex value.
__device__ __forceinline__ cx<float> ldg_cx(const cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Device error word (first error wins).  Kernels record a code and return
// instead of trapping, so the context stays usable.
enum DevErr : int {
  DEV_OK = 0,
  DEV_BAD_LAUNCH = 1,   // launch shape does not match the sizes
  DEV_BAD_SIZE = 2,     // size outside what a kernel instance supports
  DEV_NONFINITE = 3,    // a non-finite value where a finite one is required
};

__device__ __forceinline__ void set_err(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kMaxRank = 32;

// ---------------------------------------------------------------------------
// Double-float arithmetic: an unevaluated sum hi + lo of two floats carries
// about 48 significant bits at FP32 instruction rates (GB300's FP64 rate is a
// small fraction of its FP32 rate).  Error-free transformations: TwoSum
// (Knuth), TwoProduct through the fused multiply-add.  The _rn intrinsics keep
// the compiler from contracting or reassociating these sequences.
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ dfl df_norm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return dfl{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}

// acc += x * y with the product formed exactly
__device__ __forceinline__ void df_fma(dfl& acc, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);
  float s, e;
  two_sum(acc.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(acc.lo, pe));
  acc = df_norm(s, e);
}

// acc += a * y with a double-float a
__device__ __forceinline__ void df_fma(dfl& acc, dfl a, float y) {
  const float p = __fmul_rn(a.hi, y);
  float pe = __fmaf_rn(a.hi, y, -p);
  pe = __fmaf_rn(a.lo, y, pe);
  float s, e;
  two_sum(acc.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(acc.lo, pe));
  acc = df_norm(s, e);
}

__device__ __forceinline__ dfl df_shfl_xor(dfl v, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

__device__ __forceinline__ dfl df_warp_sum(dfl v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

__device__ __forceinline__ dfl df_from_double(double x) {
  const float hi = (float)x;
  return dfl{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double df_to_double(dfl v) { return (double)v.hi + (double)v.lo; }

// Complex double-float accumulator.
struct cdfl {
  dfl re, im;
};

}  // namespace tc
