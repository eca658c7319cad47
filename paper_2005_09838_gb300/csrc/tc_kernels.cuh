// Device kernels of the TCTF2R hot path (arXiv 2005.09838, Sec. 4.1).
//
// State kept on the device between iterations (the residual form):
//   R~ = DFT3(W - Z) for the floor(n3/2)+1 solved slices, X~, Y~ (half
//   spectra) and Q = R~ Y~^H (the X-step contraction, produced by the slab
//   kernel of the previous iteration).  Since W~ = X~Y~ + R~ with the factors
//   that produced Z, every quantity of Eq. (updataXYW1) that involves W~ is
//   formed from X~, Y~ and R~ without storing W.
//
// Layouts (column index fastest):
//   G    [n1][n3][n2]  real, observed values (0 off the mask)
//   mask [n1][n3][words] bit j of row (i1, i3) = (i1, j, i3) observed
//   Rt   [n1][S][n2]   complex
//   Xt   [S][r][n1]    complex
//   Yt   [S][r][n2]    complex
//   Q    [S][r][n1]    complex
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_reg.cuh"
#include "tc_common.cuh"

namespace tc {

template <typename T>
struct Dev {
  int n1, n2, n3, S, r, words;
  T mu, rho1, rho2;
  const T* G;
  const uint32_t* mask;
  cx<T>* Rt;
  cx<T>* Xt;
  cx<T>* Yt;
  cx<T>* Q;
  cx<T>* Tb;        // [S][r][n1] work buffer of the X-step
  cx<T>* Mm;        // [S][r][r] Y-step matrix I - G^+ G + G^+ E
  cx<T>* Gp;        // [S][r][r] G^+
  const T* winv;    // [2][n2] inverse pivots of the W-step rows
  const T* hinv;    // [n1] inverse pivots of H_rho1 = I + rho1 H^T H
  const cx<T>* twg; // [n3] exp(-2 pi i m / n3) for the generic transform
  T* scratch;       // per-CTA slabs when they do not fit in shared memory
  double* part;     // [n1][4] objective partial sums
  double* part_k;   // [S] rho1-term per slice
  int* err;
  double rtol;
  int pinv_fallbacks_enabled;
};

enum SlabMode : int { MODE_ITER = 0, MODE_INIT = 1, MODE_W = 2, MODE_R = 3 };

constexpr int kSlabMaxThreads = 288;

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of the slab kernel.
struct SlabLayout {
  size_t xrow, wtab, spec, spat, red, total;  // byte offsets, total bytes
  size_t slab_bytes;                          // bytes of spec (+ spat) per CTA
  bool inplace;
};

template <typename T>
__host__ __device__ inline SlabLayout slab_layout(int n2, int n3, int r, bool specialised, bool slabs_in_smem) {
  SlabLayout L{};
  const int S = n3 / 2 + 1;
  size_t off = 0;
  L.xrow = off;
  off = align_up(off + sizeof(cx<T>) * S * r, 16);
  L.wtab = off;
  off = align_up(off + sizeof(T) * 2 * n2, 16);
  L.red = off;
  off = align_up(off + sizeof(double) * 4 * 32, 16);
  L.inplace = specialised;
  const size_t spec_bytes = align_up(sizeof(cx<T>) * (size_t)S * n2, 16);
  const size_t spat_bytes = specialised ? 0 : align_up(sizeof(T) * (size_t)n3 * n2, 16);
  L.slab_bytes = spec_bytes + spat_bytes;
  if (slabs_in_smem) {
    L.spec = off;
    L.spat = specialised ? off : off + spec_bytes;
    off += spec_bytes + spat_bytes;
  } else {
    L.spec = 0;
    L.spat = specialised ? 0 : spec_bytes;
  }
  L.total = off;
  return L;
}

// Largest index < j whose mask bit is set in the row, or -1.
__device__ __forceinline__ int prev_observed(const uint32_t* __restrict__ row, int j) {
  if (j <= 0) return -1;
  int b = j - 1;
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

// Block-wide fixed-order sum of 2 doubles; result valid in thread 0.
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

// ---------------------------------------------------------------------------
// W-step of one spatial row (i1, i3) in residual form.
//
// Eq. (subquKKT): for a missing (i, j), (W K_{mu rho2})_ij = Z_ij with
// K_{mu rho2} = (1+mu) I + rho2 K^T K (tridiagonal), and W_ij = G_ij on the
// mask.  Writing W = Z + R, the unknown R solves the same tridiagonal system
// with right-hand side  -(mu + rho2 deg_j) z_j + rho2 (z_{j-1} + z_{j+1})  on
// missing entries and g_j - z_j on observed ones (identity rows).  Observed
// entries decouple the row into runs; the LU pivots of a run depend only on
// the position in the run and on whether it starts at j = 0, so their inverses
// come from a table (winv) and the sweeps carry only the right-hand side.
// On return row[j] holds r_j = w_j - z_j.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void wstep_row_tridiag(T* row, int stride, const T* __restrict__ g, const uint32_t* __restrict__ m,
                                  int n2, T mu, T rho2, const T* __restrict__ wtab) {
  const T* tab1 = wtab;       // runs starting at j = 0
  const T* tab0 = wtab + n2;  // runs starting at j > 0
  const T rho2sq = rho2 * rho2;
  // forward sweep
  T dprev = T(0);
  T zprev = T(0);
  T zcur = row[0];
  int p = -1;
  bool start0 = false;
  T invprev = T(0);
  for (int j = 0; j < n2; ++j) {
    const T znext = (j + 1 < n2) ? row[(j + 1) * stride] : T(0);
    const bool obs = bit_at(m, j);
    T dp;
    if (obs) {
      dp = __ldg(g + j) - zcur;
      p = -1;
    } else {
      if (p < 0) start0 = (j == 0);
      ++p;
      const int deg = (j > 0) + (j + 1 < n2);
      T inv;
      if (j == n2 - 1 && n2 > 1) {
        const T den = T(1) + mu + rho2 - ((p > 0) ? rho2sq * invprev : T(0));
        inv = T(1) / den;
      } else {
        inv = (start0 ? tab1 : tab0)[p];
      }
      const T rhs = -(mu + rho2 * T(deg)) * zcur + rho2 * (zprev + znext);
      dp = (rhs + rho2 * dprev) * inv;
      invprev = inv;
    }
    row[j * stride] = dp;
    dprev = dp;
    zprev = zcur;
    zcur = znext;
  }
  // backward sweep
  T rnext = T(0);
  int runstart = 0;
  int pb = -1;
  for (int j = n2 - 1; j >= 0; --j) {
    const bool obs = bit_at(m, j);
    T rj = row[j * stride];
    if (!obs) {
      if (pb < 0) {  // entering a run from its right end
        runstart = prev_observed(m, j) + 1;
        pb = j - runstart;
      }
      if (j < n2 - 1) {
        T inv;
        inv = (runstart == 0 ? tab1 : tab0)[pb];
        rj = rj + rho2 * inv * rnext;
      }
      --pb;
      row[j * stride] = rj;
    } else {
      pb = -1;
    }
    rnext = rj;
  }
}

// ---------------------------------------------------------------------------
// Generic (any n3) direct transforms of one tube, used when no register FFT
// is specialised for n3.  Eq. (bar BA-k) / Eq. (barAAk) written as sums.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void generic_irdft(const cx<T>* spec, int sstride, T* spat, int pstride, int n3,
                              const cx<T>* __restrict__ twg) {
  const int S = n3 / 2 + 1;
  const bool even = (n3 % 2) == 0;
  const int kmax = even ? S - 2 : S - 1;  // slices with a conjugate partner
  const T inv = T(1) / T(n3);
  for (int l = 0; l < n3; ++l) {
    T acc = spec[0].re;
    for (int k = 1; k <= kmax; ++k) {
      const cx<T> w = twg[(int)(((long long)k * l) % n3)];
      const cx<T> v = spec[k * sstride];
      // 2 Re(v * conj(w))
      acc += T(2) * (v.re * w.re + v.im * w.im);
    }
    if (even) acc += ((l & 1) ? -spec[(S - 1) * sstride].re : spec[(S - 1) * sstride].re);
    spat[l * pstride] = acc * inv;
  }
}

template <typename T>
__device__ void generic_rdft(const T* spat, int pstride, cx<T>* spec, int sstride, int n3,
                             const cx<T>* __restrict__ twg) {
  const int S = n3 / 2 + 1;
  for (int k = 0; k < S; ++k) {
    cx<T> acc = {T(0), T(0)};
    for (int l = 0; l < n3; ++l) {
      const cx<T> w = twg[(int)(((long long)k * l) % n3)];
      const T x = spat[l * pstride];
      acc.re += x * w.re;
      acc.im += x * w.im;
    }
    if (k == 0 || (2 * k == n3)) acc.im = T(0);
    spec[k * sstride] = acc;
  }
}

// ---------------------------------------------------------------------------
// Slab kernel: one CTA per mode-1 index i1 (one OD pair): all tubes (i1, :, :)
// and all rows (i1, :, i3).
//
// MODE_ITER: Z~ = X~Y~ (step 3), C2R (Eq. (barAAk)), W-step in residual form
//            (step 4), R2C of R = W - Z (step 7), store R~, Q = R~ Y~^H.
// MODE_INIT: same with W = P_Omega(G) in place of the W-step.
// MODE_W   : W = iDFT(X~Y~ + R~), optional copy to Wout (column-major), and
//            the partial sums ||W||^2, ||K unfold(W,2)||^2.
// MODE_R   : R = iDFT(R~), partial sums ||R||^2 and ||P_Omega R||^2.
// ---------------------------------------------------------------------------
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kSlabMaxThreads, 1) k_slab(Dev<T> d, T* __restrict__ Wout, int slabs_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int i1 = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r;
  const int n3 = (L > 0) ? L : d.n3;
  const int S = n3 / 2 + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (L > 0 && (d.n3 != L || n2 > nt)) {
    if (tid == 0) set_err(d.err, DEV_BAD_LAUNCH);
    return;
  }
  const SlabLayout lay = slab_layout<T>(n2, n3, r, L > 0, slabs_in_smem != 0);
  cx<T>* xrow = reinterpret_cast<cx<T>*>(smem + lay.xrow);
  T* wtab = reinterpret_cast<T*>(smem + lay.wtab);
  double* red = reinterpret_cast<double*>(smem + lay.red);
  unsigned char* slab_base = slabs_in_smem ? smem : reinterpret_cast<unsigned char*>(d.scratch) + (size_t)i1 * lay.slab_bytes;
  cx<T>* spec = reinterpret_cast<cx<T>*>(slab_base + lay.spec);
  T* spat = reinterpret_cast<T*>(slab_base + lay.spat);

  const bool synth = (MODE != MODE_R);
  if (synth) {
    for (int idx = tid; idx < S * r; idx += nt) {
      const int k = idx / r, s = idx - k * r;
      xrow[idx] = d.Xt[(size_t)(k * r + s) * n1 + i1];
    }
  }
  if (MODE == MODE_ITER) {
    for (int j = tid; j < 2 * n2; j += nt) wtab[j] = d.winv[j];
  }
  __syncthreads();

  // ---- phase A: spectrum of the tube and inverse transform -----------------
  if constexpr (L > 0) {
    const int t = tid;
    if (t < n2) {
      cx<T> X[L / 2 + 1];
#pragma unroll
      for (int k = 0; k < L / 2 + 1; ++k) {
        cx<T> acc = {T(0), T(0)};
        if (MODE == MODE_W || MODE == MODE_R) acc = d.Rt[((size_t)i1 * S + k) * n2 + t];
        if (synth) {
          const cx<T>* yk = d.Yt + (size_t)k * r * n2 + t;
          const cx<T>* xk = xrow + k * r;
          for (int s = 0; s < r; ++s) cfma(acc, xk[s], yk[(size_t)s * n2]);
        }
        X[k] = acc;
      }
      T x[L];
      fft::irfft<T, L>(X, x);
#pragma unroll
      for (int l = 0; l < L; ++l) spat[l * n2 + t] = x[l];
    }
  } else {
    for (int t = tid; t < n2; t += nt) {
      for (int k = 0; k < S; ++k) {
        cx<T> acc = {T(0), T(0)};
        if (MODE == MODE_W || MODE == MODE_R) acc = d.Rt[((size_t)i1 * S + k) * n2 + t];
        if (synth) {
          const cx<T>* yk = d.Yt + (size_t)k * r * n2 + t;
          const cx<T>* xk = xrow + k * r;
          for (int s = 0; s < r; ++s) cfma(acc, xk[s], yk[(size_t)s * n2]);
        }
        spec[k * n2 + t] = acc;
      }
    }
    __syncthreads();
    for (int t = tid; t < n2; t += nt) generic_irdft<T>(spec + t, n2, spat + t, n2, n3, d.twg);
  }
  __syncthreads();

  // ---- phase B: rows ------------------------------------------------------
  if (MODE == MODE_W || MODE == MODE_R) {
    double a = 0.0, b = 0.0;
    for (int e = tid; e < n3 * n2; e += nt) {
      const int l = e / n2, j = e - l * n2;
      const T v = spat[e];
      if (MODE == MODE_W) {
        a += (double)v * (double)v;
        if (j + 1 < n2) {
          const double dv = (double)v - (double)spat[e + 1];
          b += dv * dv;
        }
        if (Wout) Wout[(size_t)i1 + (size_t)n1 * ((size_t)j + (size_t)n2 * l)] = v;
      } else {
        a += (double)v * (double)v;
        const uint32_t* mrow = d.mask + ((size_t)i1 * n3 + l) * d.words;
        if (bit_at(mrow, j)) b += (double)v * (double)v;
      }
    }
    block_sum2(a, b, red);
    if (tid == 0) {
      const int o = (MODE == MODE_W) ? 2 : 0;
      d.part[(size_t)i1 * 4 + o] = a;
      d.part[(size_t)i1 * 4 + o + 1] = b;
    }
    return;
  }

  if (MODE == MODE_INIT || d.rho2 == T(0)) {
    // W = P_Omega(G) (init) or the entry-wise closed form of Eq. (Wkiom) with
    // rho2 = 0: W = Z / (1 + mu) off the mask.
    const T shrink = -d.mu / (T(1) + d.mu);
    for (int e = tid; e < n3 * n2; e += nt) {
      const int l = e / n2, j = e - l * n2;
      const size_t rowi = (size_t)i1 * n3 + l;
      const T z = spat[e];
      const bool obs = bit_at(d.mask + rowi * d.words, j);
      T rr;
      if (obs) rr = __ldg(d.G + rowi * n2 + j) - z;
      else rr = (MODE == MODE_INIT) ? -z : shrink * z;
      spat[e] = rr;
    }
  } else {
    for (int l = tid; l < n3; l += nt) {
      const size_t rowi = (size_t)i1 * n3 + l;
      wstep_row_tridiag<T>(spat + (size_t)l * n2, 1, d.G + rowi * n2, d.mask + rowi * d.words, n2, d.mu, d.rho2,
                           wtab);
    }
  }
  __syncthreads();

  // ---- phase C: forward transform, store R~ --------------------------------
  if constexpr (L > 0) {
    const int t = tid;
    T x[L];
    if (t < n2) {
#pragma unroll
      for (int l = 0; l < L; ++l) x[l] = spat[l * n2 + t];
    }
    __syncthreads();  // the spectrum overwrites the spatial slab in place
    if (t < n2) {
      cx<T> X[L / 2 + 1];
      fft::rfft<T, L>(x, X);
      cx<T>* rt = d.Rt + (size_t)i1 * S * n2 + t;
#pragma unroll
      for (int k = 0; k < L / 2 + 1; ++k) {
        spec[k * n2 + t] = X[k];
        rt[(size_t)k * n2] = X[k];
      }
    }
  } else {
    for (int t = tid; t < n2; t += nt) {
      generic_rdft<T>(spat + t, n2, spec + t, n2, n3, d.twg);
      cx<T>* rt = d.Rt + (size_t)i1 * S * n2 + t;
      for (int k = 0; k < S; ++k) rt[(size_t)k * n2] = spec[k * n2 + t];
    }
  }
  __syncthreads();

  // ---- phase D: Q(i1, :, k) = R~_k(i1, :) Y~_k^H ---------------------------
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k = wid; k < S; k += nw) {
    const cx<T>* yk = d.Yt + (size_t)k * r * n2;
    for (int s0 = 0; s0 < r; s0 += 4) {
      cx<T> acc[4] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
      for (int t = lane; t < n2; t += 32) {
        const cx<T> v = spec[k * n2 + t];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (s0 + q < r) cfmac(acc[q], v, yk[(size_t)(s0 + q) * n2 + t]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q].re = warp_sum(acc[q].re);
        acc[q].im = warp_sum(acc[q].im);
      }
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (s0 + q < r) d.Q[(size_t)(k * r + s0 + q) * n1 + i1] = acc[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 pseudo-inverse of a Hermitian PSD r x r matrix by one warp
// (Lemma "SVPMPI": A^+ = V diag(1/lambda) V^* over the eigenvalues above the
// cutoff rtol * lambda_max).
//
// Fast path: Gauss-Jordan inverse without pivoting (stable for Hermitian
// positive definite A), accepted only when ||A||_1 ||A^-1||_1 < 1/(10 rtol),
// which certifies lambda_min > rtol * lambda_max, i.e. no eigenvalue is cut
// and A^+ = A^-1 (then the projector A A^+ is exactly I).  Otherwise a cyclic
// Jacobi eigendecomposition applies the cutoff rule literally.
//
// A, Ap, P, V: r*r row-major complex doubles in shared memory; W: 2*r*r work.
// Returns (lane-uniform) 1 if the inverse path was taken.
// ---------------------------------------------------------------------------
__device__ inline int warp_pinv_herm(const cx<double>* A, cx<double>* Ap, cx<double>* P, cx<double>* V,
                                     cx<double>* W, int r, double rtol) {
  const int lane = threadIdx.x & 31;
  const int n2c = 2 * r;  // augmented columns [A | I]
  // W holds the augmented matrix row-major r x 2r
  for (int e = lane; e < r * n2c; e += 32) {
    const int i = e / n2c, j = e - i * n2c;
    W[e] = (j < r) ? A[i * r + j] : cx<double>{(j - r == i) ? 1.0 : 0.0, 0.0};
  }
  __syncwarp();
  double anorm = 0.0;
  for (int j = lane; j < r; j += 32) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += hypot(A[i * r + j].re, A[i * r + j].im);
    anorm = fmax(anorm, s);
  }
  for (int o = 16; o > 0; o >>= 1) anorm = fmax(anorm, __shfl_xor_sync(0xffffffffu, anorm, o));
  int ok = (anorm > 0.0) && isfinite(anorm);
  for (int p = 0; p < r && ok; ++p) {
    const double piv = W[p * n2c + p].re;
    ok = (piv > 1e-300) && isfinite(piv);
    if (!ok) break;
    const double ip = 1.0 / piv;
    // copy the pivot column first: its entries are overwritten below by the
    // lane that owns column p
    for (int i = lane; i < r; i += 32) V[i] = W[i * n2c + p];
    __syncwarp();
    for (int j = lane; j < n2c; j += 32) W[p * n2c + j] = W[p * n2c + j] * ip;
    __syncwarp();
    // eliminate column p from every other row; each lane owns columns
    for (int j = lane; j < n2c; j += 32) {
      const cx<double> wpj = W[p * n2c + j];
      for (int i = 0; i < r; ++i) {
        if (i == p) continue;
        W[i * n2c + j] = W[i * n2c + j] - cmul(V[i], wpj);
      }
    }
    __syncwarp();
  }
  __syncwarp();
  if (ok) {
    double inorm = 0.0;
    for (int j = lane; j < r; j += 32) {
      double s = 0.0;
      for (int i = 0; i < r; ++i) s += hypot(W[i * n2c + r + j].re, W[i * n2c + r + j].im);
      inorm = fmax(inorm, s);
    }
    for (int o = 16; o > 0; o >>= 1) inorm = fmax(inorm, __shfl_xor_sync(0xffffffffu, inorm, o));
    ok = isfinite(inorm) && (anorm * inorm < 0.1 / rtol);
  }
  if (ok) {
    for (int e = lane; e < r * r; e += 32) {
      const int i = e / r, j = e - i * r;
      // symmetrise: A^-1 of a Hermitian matrix is Hermitian
      const cx<double> a = W[i * n2c + r + j];
      const cx<double> b = W[j * n2c + r + i];
      Ap[e] = cx<double>{0.5 * (a.re + b.re), 0.5 * (a.im - b.im)};
      P[e] = cx<double>{(i == j) ? 1.0 : 0.0, 0.0};
    }
    __syncwarp();
    return 1;
  }
  // ---- cyclic Jacobi on a copy of A (stored in W, row-major r x r) ----------
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    W[e] = A[e];
    const int i = e / r, j = e - i * r;
    V[e] = cx<double>{(i == j) ? 1.0 : 0.0, 0.0};
  }
  __syncwarp();
  double fro = 0.0;
  for (int e = lane; e < r * r; e += 32) fro += W[e].re * W[e].re + W[e].im * W[e].im;
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  const double tol = 1e-30 * fro + 1e-300;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int e = lane; e < r * r; e += 32) {
      const int i = e / r, j = e - i * r;
      if (i != j) off += W[e].re * W[e].re + W[e].im * W[e].im;
    }
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (off <= tol) break;
    for (int p = 0; p < r - 1; ++p) {
      for (int q = p + 1; q < r; ++q) {
        const cx<double> c = W[p * r + q];
        const double ac = hypot(c.re, c.im);
        if (ac <= 1e-300) continue;
        const double a = W[p * r + p].re, b = W[q * r + q].re;
        const cx<double> u = {c.re / ac, c.im / ac};
        const double tau = (b - a) / (2.0 * ac);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        __syncwarp();
        // columns: A J with J = [[cs, sn u], [-sn conj(u), cs]]
        for (int i = lane; i < r; i += 32) {
          const cx<double> aip = W[i * r + p], aiq = W[i * r + q];
          W[i * r + p] = aip * cs - cmulc(aiq, u) * sn;
          W[i * r + q] = cmul(aip, u) * sn + aiq * cs;
          const cx<double> vip = V[i * r + p], viq = V[i * r + q];
          V[i * r + p] = vip * cs - cmulc(viq, u) * sn;
          V[i * r + q] = cmul(vip, u) * sn + viq * cs;
        }
        __syncwarp();
        // rows: J^H (A J)
        for (int j = lane; j < r; j += 32) {
          const cx<double> apj = W[p * r + j], aqj = W[q * r + j];
          W[p * r + j] = apj * cs - cmul(aqj, u) * sn;
          W[q * r + j] = cmulc(apj, u) * sn + aqj * cs;
        }
        __syncwarp();
      }
    }
  }
  // eigenvalues on the diagonal; cutoff relative to lambda_max
  double lmax = 0.0;
  for (int i = 0; i < r; ++i) lmax = fmax(lmax, W[i * r + i].re);
  const double cut = rtol * lmax;
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int i = e / r, j = e - i * r;
    cx<double> sa = {0.0, 0.0}, sp = {0.0, 0.0};
    for (int m = 0; m < r; ++m) {
      const double lam = W[m * r + m].re;
      if (lmax > 0.0 && lam > cut) {
        const cx<double> vv = cmulc(V[i * r + m], V[j * r + m]);  // V_im conj(V_jm)
        sa = sa + vv * (1.0 / lam);
        sp = sp + vv;
      }
    }
    Ap[e] = sa;
    P[e] = sp;
  }
  __syncwarp();
  return 0;
}

// ---------------------------------------------------------------------------
// X-step of one slice k (step 1 with the exact step of Eq. (updataXYW1)),
// followed by the r x r preparation of the Y-step (step 2):
//   A  = Y~Y~^H,  A^+, P = A A^+                                  (FP64)
//   X~' = X~ - X~P + H_rho1^{-1} (X~P + Q A^+)     [Q = R~Y~^H]
//   G  = X~'^H H_rho1 X~',  E = X~'^H X~,  G^+                      (FP64)
//   M  = I - G^+ G + G^+ E   (Y~' = M Y~ + G^+ X~'^H R~ in the Y-step kernel)
// One CTA per slice; the n1 x r work uses d.Tb.
// ---------------------------------------------------------------------------
constexpr int kSliceThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kSliceThreads) k_xstep(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem);
  cx<double>* Ap = A + rr;
  cx<double>* P = Ap + rr;
  cx<double>* V = P + rr;
  cx<double>* Wk = V + rr;          // 2 rr
  cx<double>* Gm = Wk + 2 * rr;
  cx<double>* E = Gm + rr;
  cx<T>* Pt = reinterpret_cast<cx<T>*>(E + rr);
  cx<T>* Apt = Pt + rr;
  int* flag = reinterpret_cast<int*>(Apt + rr);

  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  cx<T>* X = d.Xt + (size_t)k * r * n1;
  const cx<T>* Qk = d.Q + (size_t)k * r * n1;
  cx<T>* Tb = d.Tb + (size_t)k * r * n1;
  const bool realslice = (k == 0) || (2 * k == d.n3);

  // ---- A = Y Y^H (upper triangle, then mirrored) ---------------------------
  for (int task = wid; task < r * (r + 1) / 2; task += nw) {
    int s = 0, rem = task;
    while (rem >= r - s) {
      rem -= r - s;
      ++s;
    }
    const int u = s + rem;
    cx<T> acc = {T(0), T(0)};
    for (int j = lane; j < n2; j += 32) cfmac(acc, Y[(size_t)s * n2 + j], Y[(size_t)u * n2 + j]);
    acc.re = warp_sum(acc.re);
    acc.im = warp_sum(acc.im);
    if (lane == 0) {
      A[s * r + u] = cx<double>{(double)acc.re, (double)acc.im};
      A[u * r + s] = cx<double>{(double)acc.re, -(double)acc.im};
      if (s == u) A[s * r + s].im = 0.0;
    }
  }
  __syncthreads();
  if (wid == 0) {
    warp_pinv_herm(A, Ap, P, V, Wk, r, d.rtol);
  }
  __syncthreads();
  for (int e = tid; e < rr; e += blockDim.x) {
    Pt[e] = cx<T>{(T)P[e].re, (T)P[e].im};
    Apt[e] = cx<T>{(T)Ap[e].re, (T)Ap[e].im};
  }
  __syncthreads();

  // ---- T = X P + Q A^+ -------------------------------------------------------
  for (int e = tid; e < r * n1; e += blockDim.x) {
    const int s = e / n1, i = e - s * n1;
    cx<T> acc = {T(0), T(0)};
    for (int u = 0; u < r; ++u) {
      cfma(acc, X[(size_t)u * n1 + i], Pt[u * r + s]);
      cfma(acc, Qk[(size_t)u * n1 + i], Apt[u * r + s]);
    }
    Tb[e] = acc;
  }
  __syncthreads();
  // ---- U = H_rho1^{-1} T (tridiagonal along mode 1, one column per thread) ---
  if (d.rho1 != T(0) && n1 > 1) {
    const T rho1 = d.rho1;
    for (int s = tid; s < r; s += blockDim.x) {
      cx<T>* col = Tb + (size_t)s * n1;
      cx<T> prev = {T(0), T(0)};
      for (int i = 0; i < n1; ++i) {
        const T inv = __ldg(d.hinv + i);
        const cx<T> v = col[i];
        prev = cx<T>{(v.re + rho1 * prev.re) * inv, (v.im + rho1 * prev.im) * inv};
        col[i] = prev;
      }
      cx<T> next = col[n1 - 1];
      for (int i = n1 - 2; i >= 0; --i) {
        const T c = rho1 * __ldg(d.hinv + i);
        const cx<T> v = col[i];
        next = cx<T>{v.re + c * next.re, v.im + c * next.im};
        col[i] = next;
      }
    }
    __syncthreads();
  }
  // ---- X' = X - X P + U  (kept in Tb; X still holds the old factor) ---------
  for (int e = tid; e < r * n1; e += blockDim.x) {
    const int s = e / n1, i = e - s * n1;
    cx<T> xp = {T(0), T(0)};
    for (int u = 0; u < r; ++u) cfma(xp, X[(size_t)u * n1 + i], Pt[u * r + s]);
    cx<T> v = X[e] - xp + Tb[e];
    if (realslice) v.im = T(0);
    Tb[e] = v;
  }
  __syncthreads();

  // ---- G = X'^H H_rho1 X',  E = X'^H X_old ------------------------------------
  const int ntask_g = r * (r + 1) / 2;
  for (int task = wid; task < ntask_g + rr; task += nw) {
    if (task < ntask_g) {
      int s = 0, rem = task;
      while (rem >= r - s) {
        rem -= r - s;
        ++s;
      }
      const int u = s + rem;
      cx<T> acc = {T(0), T(0)};
      cx<T> acc2 = {T(0), T(0)};
      const cx<T>* xs = Tb + (size_t)s * n1;
      const cx<T>* xu = Tb + (size_t)u * n1;
      for (int i = lane; i < n1; i += 32) {
        const cx<T> a = xs[i], b = xu[i];
        cfmaconj(acc, a, b);
        if (i + 1 < n1) cfmaconj(acc2, a - xs[i + 1], b - xu[i + 1]);
      }
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      acc2.re = warp_sum(acc2.re);
      acc2.im = warp_sum(acc2.im);
      if (lane == 0) {
        const double gre = (double)acc.re + (double)d.rho1 * (double)acc2.re;
        const double gim = (double)acc.im + (double)d.rho1 * (double)acc2.im;
        Gm[s * r + u] = cx<double>{gre, gim};
        Gm[u * r + s] = cx<double>{gre, -gim};
        if (s == u) Gm[s * r + s].im = 0.0;
      }
    } else {
      const int e = task - ntask_g;
      const int s = e / r, u = e - s * r;
      cx<T> acc = {T(0), T(0)};
      const cx<T>* xs = Tb + (size_t)s * n1;
      const cx<T>* xu = X + (size_t)u * n1;
      for (int i = lane; i < n1; i += 32) cfmaconj(acc, xs[i], xu[i]);
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
      if (lane == 0) E[s * r + u] = cx<double>{(double)acc.re, (double)acc.im};
    }
  }
  __syncthreads();
  // ---- G^+ and M = I - G^+ G + G^+ E ---------------------------------------------
  if (wid == 0) {
    const int inv_path = warp_pinv_herm(Gm, Ap, P, V, Wk, r, d.rtol);
    if (lane == 0) flag[0] = inv_path;
  }
  __syncthreads();
  cx<T>* Mk = d.Mm + (size_t)k * rr;
  cx<T>* Gpk = d.Gp + (size_t)k * rr;
  for (int e = tid; e < rr; e += blockDim.x) {
    const int s = e / r, u = e - s * r;
    cx<double> m = {0.0, 0.0};
    for (int v = 0; v < r; ++v) m = m + cmul(Ap[s * r + v], E[v * r + u]);
    // I - G^+ G = I - P (P = G^+ G, the projector onto the range)
    m.re += ((s == u) ? 1.0 : 0.0) - P[e].re;
    m.im -= P[e].im;
    if (realslice) m.im = 0.0;
    cx<double> gp = Ap[e];
    if (realslice) gp.im = 0.0;
    Mk[e] = cx<T>{(T)m.re, (T)m.im};
    Gpk[e] = cx<T>{(T)gp.re, (T)gp.im};
  }
  // ---- X <- X' ------------------------------------------------------------------
  for (int e = tid; e < r * n1; e += blockDim.x) X[e] = Tb[e];
}

template <typename T>
__host__ inline size_t xstep_smem_bytes(int r) {
  const size_t rr = (size_t)r * r;
  return rr * sizeof(cx<double>) * 8 + rr * sizeof(cx<T>) * 2 + 16;
}

// ---------------------------------------------------------------------------
// Y-step of slice k on a tile of 32 columns (step 2 with the exact step):
//   D  = X~'^H R~_k(:, tile)           (contraction over n1, reads R~ once)
//   Y~' = M Y~ + G^+ D
// where M, G^+ come from k_xstep.  Grid (S, ceil(n2/32)), 8 warps; warp w
// accumulates the rows i = w, w+8, ...
// ---------------------------------------------------------------------------
constexpr int kYThreads = 256;

template <typename T, int RP>
__global__ void __launch_bounds__(kYThreads) k_ystep(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * 32;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* red = reinterpret_cast<cx<T>*>(smem);  // [nw][RP][32]
  cx<T>* Ds = red + nw * RP * 32;               // [RP][32]
  cx<T>* Yo = Ds + RP * 32;                     // [RP][32]
  const int j = j0 + lane;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  cx<T> acc[RP];
#pragma unroll
  for (int s = 0; s < RP; ++s) acc[s] = cx<T>{T(0), T(0)};
  if (j < n2) {
    for (int i = wid; i < n1; i += nw) {
      const cx<T> v = d.Rt[((size_t)i * S + k) * n2 + j];
#pragma unroll
      for (int s = 0; s < RP; ++s)
        if (s < r) cfmaconj(acc[s], X[(size_t)s * n1 + i], v);
    }
  }
#pragma unroll
  for (int s = 0; s < RP; ++s) red[(wid * RP + s) * 32 + lane] = acc[s];
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    Yo[s * 32 + c] = (j0 + c < n2) ? d.Yt[((size_t)k * r + s) * n2 + j0 + c] : cx<T>{T(0), T(0)};
  }
  __syncthreads();
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    cx<T> sum = {T(0), T(0)};
    for (int w = 0; w < nw; ++w) sum = sum + red[(w * RP + s) * 32 + c];
    Ds[s * 32 + c] = sum;
  }
  __syncthreads();
  const cx<T>* Mk = d.Mm + (size_t)k * r * r;
  const cx<T>* Gpk = d.Gp + (size_t)k * r * r;
  const bool realslice = (k == 0) || (2 * k == d.n3);
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    if (j0 + c >= n2) continue;
    cx<T> y = {T(0), T(0)};
    for (int u = 0; u < r; ++u) {
      cfma(y, Mk[s * r + u], Yo[u * 32 + c]);
      cfma(y, Gpk[s * r + u], Ds[u * 32 + c]);
    }
    if (realslice) y.im = T(0);
    d.Yt[((size_t)k * r + s) * n2 + j0 + c] = y;
  }
}

// ---------------------------------------------------------------------------
// Initialisation and read-back helpers (not on the per-iteration path).
// ---------------------------------------------------------------------------

// G (column-major, i1 fastest) and the byte mask -> internal row layout and
// mask bits.  One CTA per (i1, i3) row.
template <typename T>
__global__ void k_pack(const T* __restrict__ Gin, const uint8_t* __restrict__ Min, T* __restrict__ Gout,
                       uint32_t* __restrict__ Mout, int n1, int n2, int n3, int words) {
  const int row = blockIdx.x;  // i1 * n3 + i3
  const int i1 = row / n3, i3 = row - i1 * n3;
  for (int j0 = 0; j0 < words * 32; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool obs = false;
    T g = T(0);
    if (j < n2) {
      const size_t src = (size_t)i1 + (size_t)n1 * ((size_t)j + (size_t)n2 * i3);
      obs = Min[src] != 0;
      g = obs ? Gin[src] : T(0);
      Gout[(size_t)row * n2 + j] = g;
    }
    const unsigned bits = __ballot_sync(0xffffffffu, obs);
    if ((threadIdx.x & 31) == 0 && j < words * 32) Mout[(size_t)row * words + (j >> 5)] = bits;
  }
}

// Direct DFT (Eq. (bar BA-k), forward sign convention of the library) of a
// real factor along mode 3, written to the half spectrum [S][r][n]:
//   transposed = 0: input n x r x n3 (X0: i fastest, then s)
//   transposed = 1: input r x n x n3 (Y0: s fastest, then i)
template <typename T>
__global__ void k_factor_dft(const T* __restrict__ in, cx<T>* __restrict__ out, int n, int r, int n3, int transposed) {
  const int S = n3 / 2 + 1;
  const size_t total = (size_t)S * r * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const int s = (int)((e / n) % r);
    const int k = (int)(e / ((size_t)n * r));
    double re = 0.0, im = 0.0;
    for (int l = 0; l < n3; ++l) {
      const size_t src = transposed ? ((size_t)s + (size_t)r * ((size_t)i + (size_t)n * l))
                                    : ((size_t)i + (size_t)n * ((size_t)s + (size_t)r * l));
      const double v = (double)in[src];
      double sn, cs;
      sincospi(2.0 * (double)((long long)k * l % n3) / (double)n3, &sn, &cs);
      re += v * cs;
      im -= v * sn;
    }
    if (k == 0 || 2 * k == n3) im = 0.0;
    out[e] = cx<T>{(T)re, (T)im};
  }
}

// Inverse of k_factor_dft (Eq. (barAAk)) back to the caller's layout.
template <typename T>
__global__ void k_factor_idft(const cx<T>* __restrict__ in, T* __restrict__ out, int n, int r, int n3, int transposed) {
  const int S = n3 / 2 + 1;
  const bool even = (n3 % 2) == 0;
  const int kmax = even ? S - 2 : S - 1;
  const size_t total = (size_t)n * r * n3;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i, s, l;
    if (transposed) {
      s = (int)(e % r);
      i = (int)((e / r) % n);
      l = (int)(e / ((size_t)r * n));
    } else {
      i = (int)(e % n);
      s = (int)((e / n) % r);
      l = (int)(e / ((size_t)n * r));
    }
    double acc = (double)in[((size_t)0 * r + s) * n + i].re;
    for (int k = 1; k <= kmax; ++k) {
      const cx<T> v = in[((size_t)k * r + s) * n + i];
      double sn, cs;
      sincospi(2.0 * (double)((long long)k * l % n3) / (double)n3, &sn, &cs);
      // 2 Re(v * exp(+i theta))
      acc += 2.0 * ((double)v.re * cs - (double)v.im * sn);
    }
    if (even) {
      const double nyq = (double)in[((size_t)(S - 1) * r + s) * n + i].re;
      acc += (l & 1) ? -nyq : nyq;
    }
    out[e] = (T)(acc / (double)n3);
  }
}

// rho1 term of f0 per slice: tr((X~^H H^T H X~)(Y~ Y~^H)) in FP64.
template <typename T>
__global__ void k_rho1_term(Dev<T> d) {
  __shared__ double part[32];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  double tot = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int s = e / r, u = e - s * r;
    double hre = 0.0, him = 0.0;  // (HX)^H (HX) [s][u]
    for (int i = 0; i + 1 < n1; ++i) {
      const cx<T> a0 = X[(size_t)s * n1 + i], a1 = X[(size_t)s * n1 + i + 1];
      const cx<T> b0 = X[(size_t)u * n1 + i], b1 = X[(size_t)u * n1 + i + 1];
      const double ar = (double)a0.re - (double)a1.re, ai = (double)a0.im - (double)a1.im;
      const double br = (double)b0.re - (double)b1.re, bi = (double)b0.im - (double)b1.im;
      hre += ar * br + ai * bi;
      him += ar * bi - ai * br;
    }
    double yre = 0.0, yim = 0.0;  // (Y Y^H)[u][s]
    for (int j = 0; j < n2; ++j) {
      const cx<T> a = Y[(size_t)u * n2 + j], b = Y[(size_t)s * n2 + j];
      yre += (double)a.re * (double)b.re + (double)a.im * (double)b.im;
      yim += (double)a.im * (double)b.re - (double)a.re * (double)b.im;
    }
    tot += hre * yre - him * yim;
  }
  tot = warp_sum(tot);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    d.part_k[k] = s;
  }
}

}  // namespace tc
