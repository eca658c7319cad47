// Differentiation form: the adjoint of the masked t-product loss of the factor
// model,
//   L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2
// (the factor terms of f0, Eq. (TETP-optim), with W held at G on the mask).
// With E = P_Omega(Z - G) + rho1 (H^T H) x_1 Z, Z = X*Y, the gradients are the
// t-products dL/dX = E * Y^* and dL/dY = X^* * E (conjugate transpose of
// Sec. 2), i.e. per slice of the half spectrum
//   dL/dX~_k = E~_k Y~_k^H,  dL/dY~_k = X~_k^H E~_k,
// E~_k = R~_k + rho1 H^T H Z~_k with R~ = DFT(P_Omega(Z - G)) from the slab
// kernel (MODE_GRAD) and the stencil k_grad_hth adding the rho1 part in
// place; the inverse mode-3 DFT brings the gradients back to the spatial
// factors.
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

// rho1 part of the gradient: with E = P_Omega(Z - G) + rho1 (H^T H) x_1 Z the
// spectrum R~ holds DFT3(P_Omega(Z - G)) after the slab kernel; adding
// rho1 (H^T H Z~)_k to every slice makes the contractions R~Y~^H and X~^H R~
// that follow give the whole gradient.  (H^T H z)_i = deg_i z_i - z_{i-1} -
// z_{i+1} along mode 1.  One thread per entry of R~ ([n1][S][n2]).
template <typename T>
__global__ void k_grad_hth(Dev<T> d) {
  const int n1 = d.n1, n2 = d.n2, S = d.S;
  const size_t rs = (size_t)S * n2, tot = (size_t)n1 * rs;
  const T rho1 = d.rho1;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / rs);
    const cx<T> z = d.Zt[e];
    cx<T> h = {T(0), T(0)};
    if (i > 0) h = h + (z - d.Zt[e - rs]);
    if (i + 1 < n1) h = h + (z - d.Zt[e + rs]);
    const int k = (int)((e / n2) % S);
    cx<T> v = d.Rt[e] + h * rho1;
    if (k == 0 || 2 * k == d.n3) v.im = T(0);
    d.Rt[e] = v;
  }
}

}  // namespace tc
