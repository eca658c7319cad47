// Shared device types and helpers of the TCTF2R CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace tc {

// Static shared memory the library's kernels declare (block reductions) is at
// most this; sizes of dynamic shared memory are checked against the opt-in
// limit less it.
constexpr int kStaticSmemReserve = 2048;

// The dynamic shared-memory limit is an attribute of the kernel itself, shared
// by every live context that launches it: raise it to `bytes` if it is lower,
// never lower it (a smaller context created later must not break the launches
// of a larger one).
inline cudaError_t allow_dynamic_smem(const void* f, size_t bytes) {
  static std::mutex m;
  std::lock_guard<std::mutex> g(m);
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, f);
  if (e != cudaSuccess) return e;
  if ((size_t)a.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

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

// |a|
template <typename T>
__host__ __device__ __forceinline__ T cabs(cx<T> a) {
  return sqrt(a.re * a.re + a.im * a.im);
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
  DEV_TIMEOUT = 4,      // a bounded wait on the tensor core gave up
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

// Asynchronous 4-, 8- or 16-byte global -> shared copy (cp.async, L1-allocating);
// both addresses aligned to the element size.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async element size");
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(gsrc) : "memory");
  else if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(gsrc) : "memory");
}

// Wait for every cp.async of this thread (the block still needs a barrier).
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace tc
