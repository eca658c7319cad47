// Device state of the TCTF2R hot path (arXiv 2005.09838, Sec. 4.1) and the
// kernel headers.
//
// State kept on the device between iterations (residual form):
//   R~ = DFT3(W - Z) for the floor(n3/2)+1 solved slices and the half spectra
//   X~, Y~ of the factors that produced Z.  Since W~ = X~Y~ + R~, every term
//   of Eq. (updataXYW1) that involves W~ is formed from X~, Y~ and R~:
//   W~Y~^H = X~A + R~Y~^H and X~'^H W~ = X~'^H X~ Y~ + X~'^H R~.
//
// Layouts (last index fastest):
//   G    [n1][n3][n2]  real, observed values (0 off the mask), row-major
//   mask [n1][n3][mw]  mw = ceil(n2/32); bit i2 % 32 of word i2 / 32 of
//                        row (i1, :, i3) = entry (i1, i2, i3) observed
//   Rt   [n1][S][n2]   complex
//   Xt   [S][r][n1]    complex
//   Yt   [S][r][n2]    complex
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"
#include "tc_common.cuh"

namespace tc {

template <typename T>
struct Dev {
  int n1, n2, n3, S, r, mw;
  T mu, rho1, rho2;
  const T* G;
  const uint32_t* mask;
  cx<T>* Rt;
  cx<T>* Zt;        // [n1][S][n2] Z~ = X~Y~ of the current factors (written by k_ystep)
  cx<T>* Xt;
  cx<T>* Yt;
  cx<double>* Ag;   // [S][ytiles][r(r+1)/2] partial Grams Y~Y~^H over 32-column tiles
  int ytiles;       // ceil(n2 / 32)
  cx<T>* Dg;        // [S][r][r] E - G of the Y-step (k_xstep)
  cx<T>* Gp;        // [S][r][r] G^+
  cx<double>* Gp64; // [2][r][r] t G^+ of the real slices (DC, Nyquist) in FP64; FP32 engines only
  double rtol64;    // pseudo-inverse cutoff of the FP64-accurate real-slice solves
  cx<T>* Tb;        // [S][3][r][n1] X-step work arrays when shared memory is too small
  const T* winv;    // [6][n2] W-step run tables (wstep_tables)
  const T* hinv;    // [2][n1] H_rho1 = I + rho1 H^T H: inverse pivots and rho1 * inverse pivots
  const cx<T>* twg; // [n3] exp(-2 pi i m / n3) for the generic transform
  T* scratch;       // per-CTA slabs when shared memory is too small
  double* part;     // [n1][4] objective partial sums
  double* part_k;   // [S][kRhoChunks] rho1-term partial sums per slice
  int* err;
  double rtol;
  // step control (Eq. (updataXYW1) step sizes; Algorithm step 6)
  int scaled;        // 0: unit steps; 1: steps alpha / L1, beta / L2 (L from lambda_max)
  T alpha, beta;
  T hnorm;           // ||H_rho1||_2
  unsigned long long* conv;  // stopping test (null when off): [0] max |X~' - X~|, [1] max |Y~' - Y~|
                             // (non-negative doubles as bits), [2] stop flag, [3] iterations done,
                             // [4..6] last ||dX~||_inf, ||dY~||_inf, ||dW||_F as double bits
  double* part_dw;   // [n1] partial sums of ||W~^{l+1} - W~^l||^2 over the half spectrum (weighted)
  cx<T>* dZt;        // [n1][S][n2] Z~^{l+1} - Z~^l (written by k_ystep while the test is on)
  double eps;
  int yx_global;     // 1: k_ystep reads X~ of the slice from global memory (r n1 too large to stage)
  cx<T>* Dpart;      // [S][ksplit][r][n2] partial D = X~'^H R~ of the tensor-core Y-step
  int ksplit;
  // X-step of large ranks spread over five kernels (k_xa, k_xbg, k_xbc, k_xg, k_xc)
  cx<T>* Apg;        // [S][r][r] A^+
  cx<T>* Pg;         // [S][r][r] P = A A^+
  int* certA;        // [S] 1 when A^+ = A^-1 (P = I)
  T* tstep;          // [S] step t1 along d_X
  cx<T>* Gpart;      // [S][gch][3][r][r] partial Grams over kXgRows rows
  int gch;
  int apre;          // 1: A^+, P, certA, tstep of the one-CTA X-step come from k_xa (run on a
                     // graph branch after each Y-step) instead of being formed in k_xstep
  // step 5 of the Algorithm (rank vector), when the rule is on (rk != nullptr)
  int* rk;           // [S] rank of each solved slice: columns rk..r-1 of X~_k and rows of Y~_k are zero
  int* rcnt;         // [S] consecutive iterations with a Gram eigenvalue at or below rank_tol lambda_max
  cx<T>* rscr;       // [S][r][n1 + n2] work of k_rank (X~ v_d and v_d^H Y~ of the dropped directions)
  double rank_tol;
  int rank_patience;
};

// True once the stopping test has fired: the iteration kernels return at once.
template <typename T>
__device__ __forceinline__ bool converged(const Dev<T>& d) {
  return d.conv != nullptr && *reinterpret_cast<volatile const unsigned long long*>(d.conv + 2) != 0ull;
}

// atomic max of a non-negative double (its bit pattern orders like the value)
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Largest index < j whose mask bit is set in the row, or -1.
__device__ __forceinline__ int prev_observed(const uint32_t* __restrict__ row, int j) {
  if (j <= 0) return -1;
  const int b = j - 1;
  int w = b >> 5;
  const int sh = b & 31;
  uint32_t bits = __ldg(row + w) & (sh == 31 ? 0xffffffffu : ((2u << sh) - 1u));
  while (bits == 0u && w > 0) {
    --w;
    bits = __ldg(row + w);
  }
  if (bits == 0u) return -1;
  return w * 32 + 31 - __clz(bits);
}

__device__ __forceinline__ bool bit_at(const uint32_t* __restrict__ row, int j) {
  return (__ldg(row + (j >> 5)) >> (j & 31)) & 1u;
}

// Block-wide fixed-order sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
    red[2 * wid] = a;
    red[2 * wid + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int w = 0; w < nw; ++w) {
      sa += red[2 * w];
      sb += red[2 * w + 1];
    }
    a = sa;
    b = sb;
  }
  __syncthreads();
}

}  // namespace tc

#include "k_slab.cuh"
#include "k_slab_f.cuh"
#include "k_slice.cuh"
#include "k_xsplit.cuh"
#include "k_aux.cuh"
#include "k_grad.cuh"
