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
// twg[m] = exp(-2 pi i m / n3).  Each work item is one tube (s, i) and kFT
// consecutive slices k, so every input value read feeds kFT outputs; the
// items run along the input's fastest index (coalesced loads).
constexpr int kFT = 4;

__device__ __forceinline__ void factor_item(size_t e, int n, int r, int transposed, int& i, int& s, size_t& blk) {
  if (transposed) {
    s = (int)(e % r);
    i = (int)((e / r) % n);
    blk = e / ((size_t)r * n);
  } else {
    i = (int)(e % n);
    s = (int)((e / n) % r);
    blk = e / ((size_t)n * r);
  }
}

template <typename T>
__global__ void k_factor_dft(const T* __restrict__ in, cx<T>* __restrict__ out, int n, int r, int n3, int transposed,
                             const cx<T>* __restrict__ twg) {
  const int S = n3 / 2 + 1;
  const size_t total = (size_t)((S + kFT - 1) / kFT) * r * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i, s;
    size_t blk;
    factor_item(e, n, r, transposed, i, s, blk);
    const int k0 = (int)blk * kFT;
    cx<T> acc[kFT];
    int m[kFT], inc[kFT];  // (k0 + j) l mod n3, advanced by (k0 + j) mod n3
#pragma unroll
    for (int j = 0; j < kFT; ++j) {
      acc[j] = cx<T>{T(0), T(0)};
      m[j] = 0;
      inc[j] = (k0 + j) % n3;
    }
    for (int l = 0; l < n3; ++l) {
      const size_t src = transposed ? ((size_t)s + (size_t)r * ((size_t)i + (size_t)n * l))
                                    : ((size_t)i + (size_t)n * ((size_t)s + (size_t)r * l));
      const T v = in[src];
#pragma unroll
      for (int j = 0; j < kFT; ++j) {
        const cx<T> w = twg[m[j]];
        acc[j].re = fma(v, w.re, acc[j].re);
        acc[j].im = fma(v, w.im, acc[j].im);
        m[j] += inc[j];
        if (m[j] >= n3) m[j] -= n3;
      }
    }
#pragma unroll
    for (int j = 0; j < kFT; ++j) {
      const int k = k0 + j;
      if (k >= S) break;
      cx<T> v = acc[j];
      if (k == 0 || 2 * k == n3) v.im = T(0);
      out[((size_t)k * r + s) * n + i] = v;
    }
  }
}

// Inverse of k_factor_dft (Eq. (barAAk)) back to the caller's layout: each work
// item is one tube (s, i) and kFT consecutive positions l.
template <typename T>
__global__ void k_factor_idft(const cx<T>* __restrict__ in, T* __restrict__ out, int n, int r, int n3, int transposed,
                              const cx<T>* __restrict__ twg) {
  const int S = n3 / 2 + 1;
  const bool even = (n3 % 2) == 0;
  const int kmax = even ? S - 2 : S - 1;
  const size_t total = (size_t)((n3 + kFT - 1) / kFT) * r * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int i, s;
    size_t blk;
    factor_item(e, n, r, 0, i, s, blk);  // i fastest: the spectrum [S][r][n] is read coalesced
    const int l0 = (int)blk * kFT;
    T acc[kFT];
    const T s0 = in[(size_t)s * n + i].re;
#pragma unroll
    for (int j = 0; j < kFT; ++j) acc[j] = s0;
    int base = 0;  // k l0 mod n3
    for (int k = 1; k <= kmax; ++k) {
      base += l0;
      if (base >= n3) base -= n3;
      const cx<T> v = in[((size_t)k * r + s) * n + i];
      int idx = base;  // k (l0 + j) mod n3
#pragma unroll
      for (int j = 0; j < kFT; ++j) {
        const cx<T> w = twg[idx];
        // 2 Re(v exp(+i 2 pi k l / n3)) = 2 (v.re w.re + v.im w.im)
        acc[j] = fma(T(2) * v.re, w.re, fma(T(2) * v.im, w.im, acc[j]));
        idx += k;
        if (idx >= n3) idx -= n3;
      }
    }
    const T nyq = even ? in[((size_t)(S - 1) * r + s) * n + i].re : T(0);
#pragma unroll
    for (int j = 0; j < kFT; ++j) {
      const int l = l0 + j;
      if (l >= n3) break;
      T a = acc[j];
      if (even) a += (l & 1) ? -nyq : nyq;
      const size_t dst = transposed ? ((size_t)s + (size_t)r * ((size_t)i + (size_t)n * l))
                                    : ((size_t)i + (size_t)n * ((size_t)s + (size_t)r * l));
      out[dst] = a / T(n3);
    }
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

// rho1 term of f0 per slice: ||H Z~_k||_F^2 (Eq. (HunfZ2)), the sum over rows of
// |Z~_k(i+1, :) - Z~_k(i, :)|^2 of the stored spectrum Z~ = X~Y~ of the current
// factors; equal to tr((H X~)^H (H X~) Y~ Y~^H).  Grid (S, kRhoChunks): CTA
// (k, c) streams chunk c of the slice's row differences (coalesced along n2)
// and writes part_k[k kRhoChunks + c]; squares are summed error-free per thread
// (dot2) and the thread totals added in FP64 in a fixed order.
constexpr int kRhoChunks = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_rho1_term(Dev<T> d) {
  __shared__ double part[32];
  const int k = blockIdx.x, ch = blockIdx.y;
  const int n1 = d.n1, n2 = d.n2;
  const size_t rs = (size_t)d.S * n2;  // distance between rows i and i + 1 of slice k
  const cx<T>* Z = d.Zt + (size_t)k * n2;
  T s = T(0), c = T(0);
  const int nd = n1 > 1 ? n1 - 1 : 0, per = (nd + kRhoChunks - 1) / kRhoChunks;
  const int i0 = min(ch * per, nd), i1 = min(i0 + per, nd);
  // a thread walks down column j through the chunk's rows, keeping the previous
  // row's value, so each entry is read once; four rows are loaded at a time
  for (int j = threadIdx.x; j < n2 && i0 < i1; j += blockDim.x) {
    cx<T> prev = Z[(size_t)i0 * rs + j];
    int i = i0;
    for (; i + 4 <= i1; i += 4) {
      cx<T> nx[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) nx[q] = Z[(size_t)(i + 1 + q) * rs + j];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const cx<T> a = nx[q] - prev;
        dot2(s, c, a.re, a.re);
        dot2(s, c, a.im, a.im);
        prev = nx[q];
      }
    }
    for (; i < i1; ++i) {
      const cx<T> cur = Z[(size_t)(i + 1) * rs + j];
      const cx<T> a = cur - prev;
      dot2(s, c, a.re, a.re);
      dot2(s, c, a.im, a.im);
      prev = cur;
    }
  }
  double tot_d = warp_sum((double)s + (double)c);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) part[wid] = tot_d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += part[w];
    d.part_k[(size_t)k * kRhoChunks + ch] = sum;
  }
}

// ---------------------------------------------------------------------------
// Step 5 of the TCTF2R Algorithm: adjust the rank vector (the Algorithm leaves
// the rule open; this library's reading).  After the W-update of an
// iteration, every solved slice k takes the eigendecomposition G_k = V diag(lambda) V^*
// of its Y-step Gram G_k = X~_k^* H_rho1 X~_k; while at least one eigenvalue of
// the slice's active directions is <= rank_tol lambda_max, a counter grows
// (else it restarts), and when it reaches rank_patience the slice keeps only
// the directions above that level: X~_k <- X~_k V_keep and Y~_k <- V_keep^* Y~_k,
// ordered by decreasing eigenvalue, the rest of the r columns / rows set to
// zero (r_k shrinks; slices past floor(n3/2) follow by conjugate symmetry).
// W~ does not change: the part of Z~_k = X~_k Y~_k that is dropped,
// dZ = sum_d (X~_k v_d)(v_d^* Y~_k), moves from the stored Z~ to the residual
// R~ = W~ - Z~.  Zero columns stay zero through the updates (their Gram rows
// and columns are exactly zero and the pseudo-inverse cuts them).
// One CTA per slice; G is summed error-free in the working precision (FP64
// values) and its eigendecomposition is the block Jacobi in FP64.  Shared
// memory: rank_smem_bytes(r).
// ---------------------------------------------------------------------------
// s/c running sums of conj(a) b = (ar br + ai bi) + i (ar bi - ai br): acc[0],
// acc[1] the real and imaginary sums, acc[2], acc[3] their error terms (dot2).
template <typename T>
__device__ __forceinline__ void cdot2_acc(T (&acc)[4], cx<T> a, cx<T> b) {
  dot2(acc[0], acc[2], a.re, b.re);
  dot2(acc[0], acc[2], a.im, b.im);
  dot2(acc[1], acc[3], a.re, b.im);
  dot2(acc[1], acc[3], -a.im, b.re);
}

__host__ __device__ inline size_t rank_smem_bytes(int r) {
  return (7 * (size_t)r * r + 3 * (size_t)r + 2) * sizeof(cx<double>) + 2 * 32 * sizeof(int);
}

template <typename T>
__global__ void __launch_bounds__(256) k_rank(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, n1 = d.n1, n2 = d.n2, r = d.r, rr = r * r;
  const int tid = threadIdx.x, nt = blockDim.x;
  cx<double>* Gm = reinterpret_cast<cx<double>*>(smem);
  cx<double>* Ap = Gm + rr;
  cx<double>* P = Ap + rr;
  cx<double>* V = P + rr;
  cx<double>* Wk = V + rr;  // 2 r^2
  cx<double>* piv = Wk + 2 * rr;  // 3 r
  double* lmx = reinterpret_cast<double*>(piv + 3 * r);  // 2
  int* perm = reinterpret_cast<int*>(lmx + 4);            // [32] kept then dropped directions
  int* ctl = perm + 32;                                   // [0] directions kept (0: no change)
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const double rho1 = (double)d.rho1;
  cx<T>* X = d.Xt + (size_t)k * r * n1;
  cx<T>* Y = d.Yt + (size_t)k * r * n2;
  // ---- G = X~^* X~ + rho1 (H X~)^* (H X~), upper triangle, error-free sums --------------
  {
    const int ntask = r * (r + 1) / 2;
    int tp = 1;
    while (tp < 32 && tp * 2 * ntask <= nt) tp *= 2;
    const int per_pass = nt / tp, q = tid & (tp - 1);
    for (int base = 0; base < ntask; base += per_pass) {
      const int task = base + tid / tp;
      double re = 0.0, im = 0.0;
      int s = 0, u = 0;
      if (task < ntask) {
        tri_index(task, r, s, u);
        T a[4] = {T(0), T(0), T(0), T(0)}, h[4] = {T(0), T(0), T(0), T(0)};
        const cx<T>* xs = X + (size_t)s * n1;
        const cx<T>* xu = X + (size_t)u * n1;
        for (int i = q; i < n1; i += tp) {
          cdot2_acc(a, xs[i], xu[i]);
          if (i + 1 < n1) cdot2_acc(h, xs[i] - xs[i + 1], xu[i] - xu[i + 1]);
        }
        re = ((double)a[0] + (double)a[2]) + rho1 * ((double)h[0] + (double)h[2]);
        im = ((double)a[1] + (double)a[3]) + rho1 * ((double)h[1] + (double)h[3]);
      }
      for (int o = tp >> 1; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (task < ntask && q == 0) {
        if (s == u || realslice) im = 0.0;
        Gm[s * r + u] = cx<double>{re, im};
        Gm[u * r + s] = cx<double>{re, -im};
      }
    }
  }
  __syncthreads();
  // ---- eigendecomposition: eigenvalues on the diagonal of Wk, eigenvectors in V --------
  block_jacobi_pinv<double>(Gm, Ap, P, V, Wk, piv, r, 0.0, lmx);
  __syncthreads();
  if (tid == 0) {
    const int ra = d.rk[k];
    const double lmax = lmx[0];
    int nsmall = 0;
    for (int c = 0; c < r; ++c) nsmall += (Wk[c * r + c].re <= d.rank_tol * lmax) ? 1 : 0;
    // the r - ra inactive directions have eigenvalue 0 exactly
    const bool small = lmax > 0.0 && ra > 1 && nsmall > r - ra;
    int cnt = small ? d.rcnt[k] + 1 : 0;
    int keep = 0;
    if (cnt >= d.rank_patience && small) {
      // kept directions by decreasing eigenvalue, then the dropped ones
      bool used[32] = {};
      for (int c = 0; c < r; ++c) {
        int best = -1;
        for (int e = 0; e < r; ++e)
          if (!used[e] && (best < 0 || Wk[e * r + e].re > Wk[best * r + best].re)) best = e;
        used[best] = true;
        perm[c] = best;
        if (Wk[best * r + best].re > d.rank_tol * lmax) ++keep;
      }
      cnt = 0;
      d.rk[k] = keep;
    }
    d.rcnt[k] = cnt;
    ctl[0] = keep;
  }
  __syncthreads();
  const int keep = ctl[0];
  if (keep == 0) return;
  const int nd = r - keep;
  // ---- dropped part of Z~_k: a_d = X~ v_d (n1), b_d = v_d^* Y~ (n2), before rotating ----
  cx<T>* ad = d.rscr + (size_t)k * r * (n1 + n2);
  cx<T>* bd = ad + (size_t)r * n1;
  for (int e = tid; e < nd * n1; e += nt) {
    const int dd = e / n1, i = e - dd * n1, v = perm[keep + dd];
    cx<double> acc = {0.0, 0.0};
    for (int u = 0; u < r; ++u) {
      const cx<T> x = X[(size_t)u * n1 + i];
      acc = acc + cmul(cx<double>{(double)x.re, (double)x.im}, V[u * r + v]);
    }
    ad[(size_t)dd * n1 + i] = cx<T>{(T)acc.re, (T)acc.im};
  }
  for (int e = tid; e < nd * n2; e += nt) {
    const int dd = e / n2, j = e - dd * n2, v = perm[keep + dd];
    cx<double> acc = {0.0, 0.0};
    for (int u = 0; u < r; ++u) {
      const cx<T> y = Y[(size_t)u * n2 + j];
      acc = acc + cmulc(cx<double>{(double)y.re, (double)y.im}, V[u * r + v]);  // conj(V_uv) y
    }
    bd[(size_t)dd * n2 + j] = cx<T>{(T)acc.re, (T)acc.im};
  }
  __syncthreads();
  // ---- rotate: X~ <- X~ V_perm (kept columns, the rest zero), Y~ <- V_perm^* Y~ ---------
  for (int i = tid; i < n1; i += nt) {
    cx<double> x[kMaxRank];
    for (int u = 0; u < r; ++u) {
      const cx<T> v = X[(size_t)u * n1 + i];
      x[u] = cx<double>{(double)v.re, (double)v.im};
    }
    for (int c = 0; c < r; ++c) {
      cx<double> acc = {0.0, 0.0};
      if (c < keep)
        for (int u = 0; u < r; ++u) acc = acc + cmul(x[u], V[u * r + perm[c]]);
      if (realslice) acc.im = 0.0;
      X[(size_t)c * n1 + i] = cx<T>{(T)acc.re, (T)acc.im};
    }
  }
  for (int j = tid; j < n2; j += nt) {
    cx<double> y[kMaxRank];
    for (int u = 0; u < r; ++u) {
      const cx<T> v = Y[(size_t)u * n2 + j];
      y[u] = cx<double>{(double)v.re, (double)v.im};
    }
    for (int c = 0; c < r; ++c) {
      cx<double> acc = {0.0, 0.0};
      if (c < keep)
        for (int u = 0; u < r; ++u) acc = acc + cmulc(y[u], V[u * r + perm[c]]);
      if (realslice) acc.im = 0.0;
      Y[(size_t)c * n2 + j] = cx<T>{(T)acc.re, (T)acc.im};
    }
  }
  // ---- W~ unchanged: R~ += dZ, Z~ -= dZ on slice k ------------------------------------
  for (size_t e = tid; e < (size_t)n1 * n2; e += nt) {
    const int i = (int)(e / n2), j = (int)(e - (size_t)i * n2);
    cx<T> dz = {T(0), T(0)};
    for (int dd = 0; dd < nd; ++dd) cfma(dz, ad[(size_t)dd * n1 + i], bd[(size_t)dd * n2 + j]);
    if (realslice) dz.im = T(0);
    const size_t o = ((size_t)i * d.S + k) * n2 + j;
    d.Rt[o] = d.Rt[o] + dz;
    d.Zt[o] = d.Zt[o] - dz;
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
