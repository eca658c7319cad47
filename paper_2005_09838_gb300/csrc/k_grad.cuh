// Differentiation form: the adjoint of the masked t-product loss of the factor
// model,
//   L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2
// (the factor terms of f0, Eq. (TETP-optim), with W held at G on the mask).
// With E = P_Omega(Z - G) + rho1 (H^T H) x_1 Z, Z = X*Y, the gradients are the
// t-products dL/dX = E * Y^* and dL/dY = X^* * E (conjugate transpose of
// Sec. 2), i.e. per slice of the half spectrum
//   dL/dX~_k = E~_k Y~_k^H = R~_k Y~_k^H + rho1 H^T H X~_k (Y~_k Y~_k^H),
//   dL/dY~_k = X~_k^H E~_k = X~_k^H R~_k + rho1 (X~_k^H H^T H X~_k) Y~_k,
// with R~ = DFT(P_Omega(Z - G)) from the slab kernel (MODE_GRAD); the
// inverse mode-3 DFT brings them back to the spatial factors.
#pragma once

namespace tc {

// D = X~^H R~ per slice (r x n2), over a tile of 32 columns: grid
// (S, ceil(n2/32)); warp w accumulates rows i = w, w + 8, ...
template <typename T, int RP>
__global__ void __launch_bounds__(kYThreads) k_dcon(Dev<T> d, cx<T>* __restrict__ Dout) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * 32;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* red = reinterpret_cast<cx<T>*>(smem);  // [nw][RP][32]
  const cx<T>* Xg = d.Xt + (size_t)k * r * n1;
  const cx<T>* Xs = Xg;                         // [r][n1], staged when it fits
  if (!d.yx_global) {
    cx<T>* xs = red + nw * RP * 32;
    for (int e = tid; e < r * n1; e += blockDim.x) xs[e] = Xg[e];
    Xs = xs;
  }
  __syncthreads();
  const int j = j0 + lane;
  cx<T> acc[RP];
#pragma unroll
  for (int s = 0; s < RP; ++s) acc[s] = cx<T>{T(0), T(0)};
  if (j < n2) {
    int i = wid;
    for (; i + 3 * nw < n1; i += 4 * nw) {
      cx<T> v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = ldg_cx(d.Rt + ((size_t)(i + q * nw) * S + k) * n2 + j);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int s = 0; s < RP; ++s)
          if (s < r) cfmaconj(acc[s], Xs[(size_t)s * n1 + i + q * nw], v[q]);
    }
    for (; i < n1; i += nw) {
      const cx<T> v = ldg_cx(d.Rt + ((size_t)i * S + k) * n2 + j);
#pragma unroll
      for (int s = 0; s < RP; ++s)
        if (s < r) cfmaconj(acc[s], Xs[(size_t)s * n1 + i], v);
    }
  }
#pragma unroll
  for (int s = 0; s < RP; ++s) red[(wid * RP + s) * 32 + lane] = acc[s];
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    if (j0 + c >= n2) continue;
    cx<T> v = {T(0), T(0)};
    for (int w = 0; w < nw; ++w) v = v + red[(w * RP + s) * 32 + c];
    if (realslice) v.im = T(0);
    Dout[((size_t)k * r + s) * n2 + j0 + c] = v;
  }
}

template <typename T>
__host__ inline size_t dcon_smem_bytes(int n1, int r, int rp, bool x_in_smem = true) {
  return ((size_t)(kYThreads / 32) * rp * 32 + (x_in_smem ? (size_t)r * n1 : 0)) * sizeof(cx<T>);
}

// The rho1 terms, one CTA per slice, added in place:
//   GX (= R~Y~^H, [S][r][n1]) += rho1 (H^T H X~) A,   A = Y~ Y~^H
//   GY (= X~^H R~, [S][r][n2]) += rho1 B Y~,          B = (H X~)^H (H X~)
// Shared memory: A and B (2 r^2 complex).
template <typename T>
__global__ void __launch_bounds__(kSliceThreads) k_grad_rho1(Dev<T> d, cx<T>* __restrict__ GX, cx<T>* __restrict__ GY) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, rr = r * r;
  const int tid = threadIdx.x;
  const T rho1 = d.rho1;
  cx<T>* A = reinterpret_cast<cx<T>*>(smem);
  cx<T>* B = A + rr;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  // Grams: tp adjacent threads per (s, u) pair, partial sums combined by shuffles
  int tp = 1;
  while (tp < 32 && tp * 2 * rr <= (int)blockDim.x) tp *= 2;
  const int per_pass = blockDim.x / tp;
  for (int base = 0; base < rr; base += per_pass) {
    const int task = base + tid / tp, q = tid & (tp - 1);
    const bool has = task < rr;
    const int s = has ? task / r : 0, u = has ? task - s * r : 0;
    cx<T> a = {T(0), T(0)}, b = {T(0), T(0)};
    if (has) {
      for (int j = q; j < n2; j += tp) cfmac(a, Y[(size_t)s * n2 + j], Y[(size_t)u * n2 + j]);
      for (int i = q; i + 1 < n1; i += tp)
        cfmaconj(b, X[(size_t)s * n1 + i] - X[(size_t)s * n1 + i + 1], X[(size_t)u * n1 + i] - X[(size_t)u * n1 + i + 1]);
    }
    for (int o = tp >> 1; o > 0; o >>= 1) {
      a.re += __shfl_xor_sync(0xffffffffu, a.re, o);
      a.im += __shfl_xor_sync(0xffffffffu, a.im, o);
      b.re += __shfl_xor_sync(0xffffffffu, b.re, o);
      b.im += __shfl_xor_sync(0xffffffffu, b.im, o);
    }
    if (has && q == 0) {
      A[s * r + u] = a;
      B[s * r + u] = b;
    }
  }
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  for (int e = tid; e < r * n1; e += blockDim.x) {
    const int s = e / n1, i = e - s * n1;
    cx<T> acc = {T(0), T(0)};
    for (int u = 0; u < r; ++u) cfma(acc, hth_at(X + (size_t)u * n1, i, n1), A[u * r + s]);
    cx<T> v = GX[(size_t)k * r * n1 + e] + acc * rho1;
    if (realslice) v.im = T(0);
    GX[(size_t)k * r * n1 + e] = v;
  }
  for (int e = tid; e < r * n2; e += blockDim.x) {
    const int s = e / n2, j = e - s * n2;
    cx<T> acc = {T(0), T(0)};
    for (int u = 0; u < r; ++u) cfma(acc, B[s * r + u], Y[(size_t)u * n2 + j]);
    cx<T> v = GY[(size_t)k * r * n2 + e] + acc * rho1;
    if (realslice) v.im = T(0);
    GY[(size_t)k * r * n2 + e] = v;
  }
}

}  // namespace tc
