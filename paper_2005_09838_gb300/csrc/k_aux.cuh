// Initialisation, read-back and objective helpers of the TCTF2R library (not
// on the per-iteration path).
#pragma once

namespace tc {


// G (column-major, i1 fastest) and the byte mask -> the internal layouts:
// G row-major [i1][i3][i2] and mask words row-major [i1][i3][ceil(n2/32)]
// (bit i2 % 32 of word i2 / 32).  One CTA per row (i1, :, i3).
template <typename T>
__global__ void k_pack(const T* __restrict__ Gin, const uint8_t* __restrict__ Min, T* __restrict__ Gout,
                       uint32_t* __restrict__ Mout, int n1, int n2, int n3, int mw) {
  const int row = blockIdx.x;  // i1 * n3 + i3
  const int i1 = row / n3, l = row - i1 * n3;
  for (int t0 = 0; t0 < mw * 32; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    bool obs = false;
    if (t < n2) {
      const size_t src = (size_t)i1 + (size_t)n1 * ((size_t)t + (size_t)n2 * l);
      obs = Min[src] != 0;
      Gout[(size_t)row * n2 + t] = obs ? Gin[src] : T(0);
    }
    const unsigned bits = __ballot_sync(0xffffffffu, obs);
    if ((threadIdx.x & 31) == 0 && t < mw * 32) Mout[(size_t)row * mw + (t >> 5)] = bits;
  }
}

// Direct DFT (Eq. (bar BA-k), forward sign convention of the library) of a
// real factor along mode 3, written to the half spectrum [S][r][n]:
//   transposed = 0: input n x r x n3 (X0: i fastest, then s)
//   transposed = 1: input r x n x n3 (Y0: s fastest, then i)
// twg[m] = exp(-2 pi i m / n3); four interleaved partial sums.
template <typename T>
__global__ void k_factor_dft(const T* __restrict__ in, cx<T>* __restrict__ out, int n, int r, int n3, int transposed,
                             const cx<T>* __restrict__ twg) {
  const int S = n3 / 2 + 1;
  const size_t total = (size_t)S * r * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n);
    const int s = (int)((e / n) % r);
    const int k = (int)(e / ((size_t)n * r));
    cx<T> acc[4] = {};
    int m = 0;  // k * l mod n3
    for (int l = 0; l < n3; ++l) {
      const size_t src = transposed ? ((size_t)s + (size_t)r * ((size_t)i + (size_t)n * l))
                                    : ((size_t)i + (size_t)n * ((size_t)s + (size_t)r * l));
      const T v = in[src];
      const cx<T> w = twg[m];
      acc[l & 3].re = fma(v, w.re, acc[l & 3].re);
      acc[l & 3].im = fma(v, w.im, acc[l & 3].im);
      m += k;
      if (m >= n3) m -= n3;
    }
    cx<T> v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    if (k == 0 || 2 * k == n3) v.im = T(0);
    out[e] = v;
  }
}

// Inverse of k_factor_dft (Eq. (barAAk)) back to the caller's layout.
template <typename T>
__global__ void k_factor_idft(const cx<T>* __restrict__ in, T* __restrict__ out, int n, int r, int n3, int transposed,
                              const cx<T>* __restrict__ twg) {
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
    T acc[2] = {in[((size_t)0 * r + s) * n + i].re, T(0)};
    int m = 0;  // k * l mod n3
    for (int k = 1; k <= kmax; ++k) {
      m += l;
      if (m >= n3) m -= n3;
      const cx<T> v = in[((size_t)k * r + s) * n + i];
      const cx<T> w = twg[m];
      // 2 Re(v exp(+i 2 pi k l / n3)) = 2 (v.re w.re + v.im w.im)
      acc[k & 1] = fma(T(2) * v.re, w.re, fma(T(2) * v.im, w.im, acc[k & 1]));
    }
    if (even) {
      const T nyq = in[((size_t)(S - 1) * r + s) * n + i].re;
      acc[0] += (l & 1) ? -nyq : nyq;
    }
    out[e] = (acc[0] + acc[1]) / T(n3);
  }
}

// Stopping test of the Algorithm (step 6), one warp after each iteration:
// stop once ||X~^{l+1} - X~^l||_inf <= eps, ||Y~^{l+1} - Y~^l||_inf <= eps and
// ||W^{l+1} - W^l||_F <= eps.  ||.||_inf is the largest modulus of an entry;
// ||dW||_F comes from the half spectrum by Parseval (sum over all n3 slices of
// |dW~_k|^2 divided by n3).  Counts the iterations run and resets the maxima.
template <typename T>
__global__ void k_check(Dev<T> d) {
  unsigned long long* c = d.conv;
  if (c[2] != 0ull) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < d.n1; i += 32) s += d.part_dw[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    const double dx = __longlong_as_double((long long)c[0]);
    const double dy = __longlong_as_double((long long)c[1]);
    const double dw = sqrt(s / (double)d.n3);
    c[3] += 1ull;
    c[4] = (unsigned long long)__double_as_longlong(dx);
    c[5] = (unsigned long long)__double_as_longlong(dy);
    c[6] = (unsigned long long)__double_as_longlong(dw);
    if (dx <= d.eps && dy <= d.eps && dw <= d.eps) c[2] = 1ull;
    c[0] = 0ull;
    c[1] = 0ull;
  }
}

// rho1 term of f0 per slice, tr(B A) with B = (H X~)^H (H X~) and A = Y~ Y~^H
// (||H Z~_k||_F^2 for Z~_k = X~_k Y~_k, Eq. (HunfZ2)).  One CTA per slice; each
// upper-triangle pair (s, u) of the two r x r Grams is summed by tp adjacent
// threads that split the rows, with products in the working precision
// accumulated error-free (dot2: about twice the working precision) and the
// partial sums combined in FP64; the trace is accumulated in FP64 as
// sum_s B_ss A_ss + 2 sum_{s<u} Re(B_su A_us).
template <typename T>
__device__ __forceinline__ void cdot2_acc(T (&acc)[4], cx<T> a, cx<T> b) {
  // conj(a) b = (ar br + ai bi) + i (ar bi - ai br), four error-free running sums
  dot2(acc[0], acc[2], a.re, b.re);
  dot2(acc[0], acc[2], a.im, b.im);
  dot2(acc[1], acc[3], a.re, b.im);
  dot2(acc[1], acc[3], -a.im, b.re);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rho1_term(Dev<T> d) {
  __shared__ double part[32];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r;
  const int ntask = r * (r + 1) / 2;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  int tp = 1;
  while (tp < 32 && tp * 2 * ntask <= (int)blockDim.x) tp *= 2;
  const int per_pass = blockDim.x / tp, q = threadIdx.x & (tp - 1);
  double tot = 0.0;
  for (int base = 0; base < ntask; base += per_pass) {  // every thread runs the same passes
    const int task = base + (int)threadIdx.x / tp;
    double bre = 0.0, bim = 0.0, are = 0.0, aim = 0.0;
    int s = 0, u = 0;
    if (task < ntask) {
      tri_index(task, r, s, u);
      T b[4] = {T(0), T(0), T(0), T(0)}, a[4] = {T(0), T(0), T(0), T(0)};
      const cx<T>* xs = X + (size_t)s * n1;
      const cx<T>* xu = X + (size_t)u * n1;
      for (int i = q; i + 1 < n1; i += tp) cdot2_acc(b, xs[i] - xs[i + 1], xu[i] - xu[i + 1]);  // B_su
      const cx<T>* ys = Y + (size_t)s * n2;
      const cx<T>* yu = Y + (size_t)u * n2;
      for (int j = q; j < n2; j += tp) cdot2_acc(a, ys[j], yu[j]);  // conj(y_s) y_u summed: A_us
      bre = (double)b[0] + (double)b[2];
      bim = (double)b[1] + (double)b[3];
      are = (double)a[0] + (double)a[2];
      aim = (double)a[1] + (double)a[3];
    }
    for (int o = tp >> 1; o > 0; o >>= 1) {
      bre += __shfl_xor_sync(0xffffffffu, bre, o);
      bim += __shfl_xor_sync(0xffffffffu, bim, o);
      are += __shfl_xor_sync(0xffffffffu, are, o);
      aim += __shfl_xor_sync(0xffffffffu, aim, o);
    }
    // B_su = sum_i conj(Hx_s) Hx_u = (bre, bim); A_us = sum_j y_u conj(y_s) = (are, aim)
    if (task < ntask && q == 0) tot += (s == u ? 1.0 : 2.0) * (bre * are - bim * aim);
  }
  tot = warp_sum(tot);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += part[w];
    d.part_k[k] = sum;
  }
}

// Initial Z~ = X~Y~ (step 3 at the initial point; during the iteration the
// Y-step kernel writes Z~).  One thread per output.
template <typename T>
__global__ void k_synth_init(Dev<T> d) {
  const size_t total = (size_t)d.n1 * d.S * d.n2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % d.n2);
    const int k = (int)((e / d.n2) % d.S);
    const int i = (int)(e / ((size_t)d.n2 * d.S));
    cx<T> z = {T(0), T(0)};
    for (int s = 0; s < d.r; ++s)
      cfma(z, d.Xt[((size_t)k * d.r + s) * d.n1 + i], d.Yt[((size_t)k * d.r + s) * d.n2 + j]);
    d.Zt[e] = z;
  }
}

// Initial tile Grams of Y~ (the X-step's A for the first iteration).  Grid
// (S, ytiles), one warp per upper-triangle entry.
template <typename T>
__global__ void k_gram_tiles(Dev<T> d) {
  const int k = blockIdx.x, tile = blockIdx.y;
  const int r = d.r, n2 = d.n2, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ntask = r * (r + 1) / 2;
  const int j = tile * 32 + lane;
  for (int task = wid; task < ntask; task += nw) {
    int s, u;
    tri_index(task, r, s, u);
    cx<T> g = {T(0), T(0)};  // the same arithmetic as the tile Grams of k_ystep
    if (j < n2) cfmac(g, d.Yt[((size_t)k * r + s) * n2 + j], d.Yt[((size_t)k * r + u) * n2 + j]);
    g.re = warp_sum(g.re);
    g.im = warp_sum(g.im);
    if (lane == 0) d.Ag[((size_t)k * d.ytiles + tile) * ntask + task] = cx<double>{(double)g.re, (double)g.im};
  }
}

}  // namespace tc
