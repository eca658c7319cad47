// The X-step of large ranks (r > 16) spread over the GPU: one CTA per slice
// for a whole X-step (k_xstep) leaves most SMs idle and runs r^2 n1 Gram
// products on one SM.  Here the same step (Eq. (updataXYW1) with the gradients
// of Eq. (hkXYDer), formed as in k_xstep) is four kernels:
//   k_xa   (S CTAs)               A = Y~Y~^H from the tile Grams, A^+, P, step t1; run
//                                 after every change of Y~ (initialisation, each
//                                 Y-step), beside the rest of that iteration
//   k_xb1  (S CTAs) or            one warp per column s: B = Q A^+ - rho1 (H^T H X~) P,
//   k_xb   (S x ceil(r/8) CTAs)   d_X = H_rho1^{-1} B, X~' = X~ + t1 d_X (to d.Tb); k_xb1
//                                 stages the slice's Q in shared memory, k_xb (n1 too
//                                 large for that) reads it through L1
//   k_xg   (S x ceil(n1/64) CTAs) partial Grams over 64 rows: X~'^H X~', (H X~')^H (H X~'),
//                                 X~'^H (X~' - X~)
//   k_xc   (S CTAs)               the partials summed in a fixed order, G, Dg, t2 G^+ for
//                                 k_ystep; X~ <- X~'
#pragma once

namespace tc {

constexpr int kXaThreads = 1024;
constexpr int kXgRows = 64;
constexpr int kXgLd = kXgRows + 1;  // odd row pitch: conflict-free column reads

template <typename TS>
__host__ __device__ inline size_t xa_smem_bytes(int r) {
  const size_t rr = (size_t)r * r;
  return align_up((rr * 7 + 3 * (size_t)r) * sizeof(cx<TS>) + 4 * sizeof(TS), 16);
}

template <typename T>
__host__ __device__ inline size_t xb_smem_bytes(int n1) {
  return align_up(2 * (size_t)n1 * sizeof(T), 16) + (8 * (size_t)n1 + 2 * 8 * 32) * sizeof(cx<T>);
}

template <typename T>
__host__ __device__ inline size_t xg_smem_bytes(int r) {
  return 2 * (size_t)r * kXgLd * sizeof(cx<T>);
}

// ---- A^+ and P of every slice ----------------------------------------------------------
template <typename T, typename TS>
__global__ void __launch_bounds__(kXaThreads) k_xa(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, r = d.r, rr = r * r, tid = threadIdx.x;
  cx<TS>* A = reinterpret_cast<cx<TS>*>(smem);
  cx<TS>* Ap = A + rr;
  cx<TS>* P = Ap + rr;
  cx<TS>* V = P + rr;
  cx<TS>* Wk = V + rr;
  cx<TS>* pivbuf = Wk + 2 * rr;  // 3 r
  TS* sred = reinterpret_cast<TS*>(pivbuf + 3 * r);
  {
    const int ntask = r * (r + 1) / 2;
    const cx<double>* ag = d.Ag + (size_t)k * d.ytiles * ntask;
    for (int task = tid; task < ntask; task += blockDim.x) {
      int s, u;
      tri_index(task, r, s, u);
      cx<double> acc[4] = {};
      int t = 0;
      for (; t + 3 < d.ytiles; t += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = acc[q] + ag[(size_t)(t + q) * ntask + task];
      }
      for (; t < d.ytiles; ++t) acc[0] = acc[0] + ag[(size_t)t * ntask + task];
      cx<double> v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      if (s == u) v.im = 0.0;
      A[s * r + u] = cx<TS>{(TS)v.re, (TS)v.im};
      A[u * r + s] = cx<TS>{(TS)v.re, (TS)(-v.im)};
    }
  }
  __syncthreads();
  constexpr bool kDF = sizeof(T) == 4 && sizeof(TS) == 8;
  const bool cert = block_pinv_herm<TS, 32, kDF>(A, Ap, P, V, Wk, pivbuf, sred, r, (TS)d.rtol, d.scaled != 0) != 0;
  const T t1 = d.scaled ? ((sred[2] > TS(0)) ? d.alpha / (d.hnorm * (T)sred[2]) : T(0)) : T(1);
  for (int e = tid; e < rr; e += blockDim.x) {
    d.Apg[(size_t)k * rr + e] = cvt<T>(Ap[e]);
    d.Pg[(size_t)k * rr + e] = cvt<T>(P[e]);
  }
  if (tid == 0) {
    d.certA[k] = cert ? 1 : 0;
    d.tstep[k] = t1;
  }
}

// ---- B, d_X = H_rho1^{-1} B and X~' per column ----------------------------------------
// One CTA per 8 columns, Q read through L1 (n1 too large for k_xb1).
template <typename T>
__global__ void __launch_bounds__(256) k_xb(Dev<T> d, const cx<T>* __restrict__ Qin) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, n1 = d.n1, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int s = blockIdx.y * 8 + wid;
  T* hinv = reinterpret_cast<T*>(smem);
  T* ha = hinv + n1;
  cx<T>* cols = reinterpret_cast<cx<T>*>(smem + align_up(2 * (size_t)n1 * sizeof(T), 16));  // [8][n1]
  cx<T>* apc = cols + 8 * (size_t)n1;  // [8][32] column s of A^+
  cx<T>* pc = apc + 8 * 32;            // [8][32] column s of P
  for (int i = tid; i < 2 * n1; i += blockDim.x) hinv[i] = d.hinv[i];
  if (s < r) {
    apc[wid * 32 + lane] = lane < r ? d.Apg[(size_t)k * rr + lane * r + s] : cx<T>{T(0), T(0)};
    pc[wid * 32 + lane] = lane < r ? d.Pg[(size_t)k * rr + lane * r + s] : cx<T>{T(0), T(0)};
  }
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const T rho1 = d.rho1;
  double dmax = 0.0;
  if (s < r) {
    const bool certA = d.certA[k] != 0;
    const T t1 = d.tstep[k];
    const cx<T>* Q = Qin + (size_t)k * r * n1;
    const cx<T>* X = d.Xt + (size_t)k * r * n1;
    const cx<T>* ap = apc + wid * 32;
    const cx<T>* pp = pc + wid * 32;
    cx<T>* col = cols + (size_t)wid * n1;
    for (int i = lane; i < n1; i += 32) {
      cx<T> acc = {T(0), T(0)};
      cx<T> q[32];  // all r loads of the row in flight, then the products in order
#pragma unroll
      for (int u = 0; u < 32; ++u) q[u] = u < r ? ldg_cx(Q + (size_t)u * n1 + i) : cx<T>{T(0), T(0)};
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (u < r) cfma(acc, q[u], ap[u]);
      if (rho1 != T(0)) {
        cx<T> hx = {T(0), T(0)};
        if (certA) {
          hx = hth_at(X + (size_t)s * n1, i, n1);  // P = I
        } else {
          for (int u = 0; u < r; ++u) cfma(hx, hth_at(X + (size_t)u * n1, i, n1), pp[u]);
        }
        acc = acc - hx * rho1;
      }
      col[i] = acc;
    }
    __syncwarp();
    if (rho1 != T(0) && n1 > 1) warp_tridiag_solve<T>(col, n1, hinv, ha);
    __syncwarp();
    cx<T>* Xp = d.Tb + (size_t)k * r * n1 + (size_t)s * n1;
    for (int i = lane; i < n1; i += 32) {
      const cx<T> x0 = X[(size_t)s * n1 + i];
      cx<T> v = d.scaled ? x0 + col[i] * t1 : x0 + col[i];
      if (realslice) v.im = T(0);
      Xp[i] = v;
      if (d.conv) dmax = fmax(dmax, (double)cabs(v - x0));
    }
  }
  if (d.conv) block_max_to(dmax, d.conv + 0);
}

// ---- the same per slice: one CTA of 1024 threads, warp s forms column s ---------------
// Q of the slice is staged once; each warp writes its column of B to the
// slice's work array (L2-resident) and, once every warp has read Q, copies it
// back into its own row of the staged Q for the tridiagonal solve.

template <typename T>
__host__ __device__ inline size_t xb1_smem_bytes(int n1, int r) {
  return align_up(2 * (size_t)n1 * sizeof(T), 16) + (2 * 32 * 32 + (size_t)r * n1) * sizeof(cx<T>);
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_xb1(Dev<T> d, const cx<T>* __restrict__ Qin) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, n1 = d.n1, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, s = tid >> 5;
  T* hinv = reinterpret_cast<T*>(smem);
  T* ha = hinv + n1;
  cx<T>* apc = reinterpret_cast<cx<T>*>(smem + align_up(2 * (size_t)n1 * sizeof(T), 16));  // [32][32]
  cx<T>* pc = apc + 32 * 32;
  cx<T>* qs = pc + 32 * 32;  // [r][n1]
  for (int i = tid; i < 2 * n1; i += blockDim.x) hinv[i] = d.hinv[i];
  if (s < r) {
    apc[s * 32 + lane] = lane < r ? d.Apg[(size_t)k * rr + lane * r + s] : cx<T>{T(0), T(0)};
    pc[s * 32 + lane] = lane < r ? d.Pg[(size_t)k * rr + lane * r + s] : cx<T>{T(0), T(0)};
  }
  {
    const cx<T>* Qk = Qin + (size_t)k * r * n1;
    const int nq = r * n1, nt = blockDim.x;
    int e = tid;
    for (; e + 3 * nt < nq; e += 4 * nt) {
      cx<T> v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = ldg_cx(Qk + e + q * nt);
#pragma unroll
      for (int q = 0; q < 4; ++q) qs[e + q * nt] = v[q];
    }
    for (; e < nq; e += nt) qs[e] = ldg_cx(Qk + e);
  }
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const T rho1 = d.rho1;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  cx<T>* Bw = d.Tb + (size_t)k * r * n1 + (size_t)s * n1;  // column s of B, then of X~'
  if (s < r) {
    const bool certA = d.certA[k] != 0;
    const cx<T>* ap = apc + s * 32;
    const cx<T>* pp = pc + s * 32;
    for (int i = lane; i < n1; i += 32) {
      cx<T> acc = {T(0), T(0)};
      for (int u = 0; u < r; ++u) cfma(acc, qs[(size_t)u * n1 + i], ap[u]);
      if (rho1 != T(0)) {
        cx<T> hx = {T(0), T(0)};
        if (certA) {
          hx = hth_at(X + (size_t)s * n1, i, n1);  // P = I
        } else {
          for (int u = 0; u < r; ++u) cfma(hx, hth_at(X + (size_t)u * n1, i, n1), pp[u]);
        }
        acc = acc - hx * rho1;
      }
      Bw[i] = acc;
    }
  }
  __syncthreads();  // every warp has read Q (and its own B stores are visible to it)
  double dmax = 0.0;
  if (s < r) {
    cx<T>* col = qs + (size_t)s * n1;
    for (int i = lane; i < n1; i += 32) col[i] = Bw[i];
    __syncwarp();
    if (rho1 != T(0) && n1 > 1) warp_tridiag_solve<T>(col, n1, hinv, ha);
    __syncwarp();
    const T t1 = d.tstep[k];
    const cx<T>* xs = X + (size_t)s * n1;
    auto update = [&](int i, cx<T> x0) {
      cx<T> v = d.scaled ? x0 + col[i] * t1 : x0 + col[i];
      if (realslice) v.im = T(0);
      Bw[i] = v;
      if (d.conv) dmax = fmax(dmax, (double)cabs(v - x0));
    };
    int i = lane;
    for (; i + 96 < n1; i += 128) {  // four loads in flight per lane
      cx<T> x0[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x0[q] = xs[i + 32 * q];
#pragma unroll
      for (int q = 0; q < 4; ++q) update(i + 32 * q, x0[q]);
    }
    for (; i < n1; i += 32) update(i, xs[i]);
  }
  if (d.conv) block_max_to(dmax, d.conv + 0);
}

// ---- partial Grams over kXgRows rows -----------------------------------------------------
// The real slices (DC and, for even n3, Nyquist) hold real factors; their
// Grams are the ill-conditioned ones (the DC slice carries the mean traffic),
// so they are accumulated with dot2 and the partial is stored as (sum,
// compensation) in the (re, im) fields.
template <typename T>
__global__ void __launch_bounds__(256) k_xg(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, c = blockIdx.y, n1 = d.n1, r = d.r, rr = r * r;
  const int tid = threadIdx.x, i0 = c * kXgRows;
  cx<T>* gx = reinterpret_cast<cx<T>*>(smem);  // [r][kXgLd] rows i0 .. i0 + kXgRows of X~'
  cx<T>* go = gx + (size_t)r * kXgLd;          // [r][kXgLd] rows i0 .. of X~
  const cx<T>* Xp = d.Tb + (size_t)k * r * n1;
  const cx<T>* X = d.Xt + (size_t)k * r * n1;
  const int nrow = min(kXgRows + 1, n1 - i0);
  for (int e = tid; e < r * kXgLd; e += blockDim.x) {
    const int s = e / kXgLd, ii = e - s * kXgLd;
    if (ii < nrow) {
      gx[e] = Xp[(size_t)s * n1 + i0 + ii];
      if (ii < kXgRows) go[e] = X[(size_t)s * n1 + i0 + ii];
    }
  }
  __syncthreads();
  const int iend = min(kXgRows, n1 - i0);
  cx<T>* out = d.Gpart + ((size_t)k * d.gch + c) * 3 * rr;
  const bool realslice = (k == 0) || (2 * k == d.n3);
  if (realslice) {
    for (int task = tid; task < rr; task += blockDim.x) {
      const int s = task / r, u = task - s * r;
      const cx<T>* xs = gx + s * kXgLd;
      const cx<T>* xu = gx + u * kXgLd;
      const cx<T>* ou = go + u * kXgLd;
      T s0 = T(0), c0 = T(0), s1 = T(0), c1 = T(0), s2 = T(0), c2 = T(0);
      for (int ii = 0; ii < iend; ++ii) {
        const T a = xs[ii].re, b = xu[ii].re;
        dot2(s0, c0, a, b);
        dot2(s2, c2, a, b - ou[ii].re);
        if (i0 + ii + 1 < n1) dot2(s1, c1, a - xs[ii + 1].re, b - xu[ii + 1].re);
      }
      out[task] = cx<T>{s0, c0};
      out[rr + task] = cx<T>{s1, c1};
      out[2 * rr + task] = cx<T>{s2, c2};
    }
    return;
  }
  // a thread takes the pairs {s0, s0 + rb} x {u0, u0 + rb} (rb = ceil(r / 2)):
  // 10 loads per row feed 12 products, and consecutive threads (consecutive
  // u0) read consecutive rows of odd pitch, so a half-warp hits distinct banks
  const int rb = (r + 1) / 2;
  for (int blk = tid; blk < rb * rb; blk += blockDim.x) {
    const int s0 = blk / rb, u0 = blk % rb;
    const int s1 = min(s0 + rb, r - 1), u1 = min(u0 + rb, r - 1);
    const cx<T>* xs[2] = {gx + s0 * kXgLd, gx + s1 * kXgLd};
    const cx<T>* xu[2] = {gx + u0 * kXgLd, gx + u1 * kXgLd};
    const cx<T>* ou[2] = {go + u0 * kXgLd, go + u1 * kXgLd};
    cx<T> a0[2][2], hh[2][2], dd[2][2];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) a0[x][y] = hh[x][y] = dd[x][y] = cx<T>{T(0), T(0)};
    for (int ii = 0; ii < iend; ++ii) {
      const bool nb = i0 + ii + 1 < n1;
      cx<T> a[2], da[2], b[2], db[2], e[2];
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        a[x] = xs[x][ii];
        da[x] = nb ? a[x] - xs[x][ii + 1] : cx<T>{T(0), T(0)};
        b[x] = xu[x][ii];
        db[x] = nb ? b[x] - xu[x][ii + 1] : cx<T>{T(0), T(0)};
        e[x] = b[x] - ou[x][ii];
      }
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          cfmaconj(a0[x][y], a[x], b[y]);
          cfmaconj(dd[x][y], a[x], e[y]);
          cfmaconj(hh[x][y], da[x], db[y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int s = s0 + x * rb, u = u0 + y * rb;
        if (s < r && u < r) {
          const int task = s * r + u;
          out[task] = a0[x][y];
          out[rr + task] = hh[x][y];
          out[2 * rr + task] = dd[x][y];
        }
      }
  }
}

// Sums of the k_xg partials of one Gram entry in a fixed order: in df64 on the
// FP32 pipes for float partials (real slices: the (sum, compensation) pairs
// are added as df64 values), in FP64 for double ones.
__device__ __forceinline__ void sum_partials(const cx<float>* part, int rr, int gch, int task, bool realslice,
                                             cx<double>& a0, cx<double>& hh, cx<double>& dd) {
  df s[6] = {};
  auto add = [&](int q, cx<float> v) {
    if (realslice) {
      s[2 * q] = df_add(s[2 * q], df_norm(v.re, v.im));
    } else {
      s[2 * q] = df_add(s[2 * q], df{v.re, 0.f});
      s[2 * q + 1] = df_add(s[2 * q + 1], df{v.im, 0.f});
    }
  };
  int c = 0;
  for (; c + 2 <= gch; c += 2) {  // six loads in flight, added in chunk order
    cx<float> v[2][3];
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[w][q] = part[((size_t)(c + w) * 3 + q) * rr + task];
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) add(q, v[w][q]);
  }
  for (; c < gch; ++c)
#pragma unroll
    for (int q = 0; q < 3; ++q) add(q, part[((size_t)c * 3 + q) * rr + task]);
  a0 = cx<double>{df_to(s[0]), df_to(s[1])};
  hh = cx<double>{df_to(s[2]), df_to(s[3])};
  dd = cx<double>{df_to(s[4]), df_to(s[5])};
}
__device__ __forceinline__ void sum_partials(const cx<double>* part, int rr, int gch, int task, bool realslice,
                                             cx<double>& a0, cx<double>& hh, cx<double>& dd) {
  a0 = hh = dd = cx<double>{0.0, 0.0};
  for (int c = 0; c < gch; ++c) {
    const cx<double>* pc = part + (size_t)c * 3 * rr;
    a0 = a0 + pc[task];
    hh = hh + pc[rr + task];
    dd = dd + pc[2 * rr + task];
  }
  if (realslice) {  // (sum, compensation) pairs of k_xg
    a0 = cx<double>{a0.re + a0.im, 0.0};
    hh = cx<double>{hh.re + hh.im, 0.0};
    dd = cx<double>{dd.re + dd.im, 0.0};
  }
}

// ---- G, Dg from the partials, t2 G^+; X~ <- X~' -------------------------------------------
template <typename T, typename TS>
__global__ void __launch_bounds__(kXaThreads) k_xc(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, n1 = d.n1, r = d.r, rr = r * r, tid = threadIdx.x;
  cx<TS>* Gm = reinterpret_cast<cx<TS>*>(smem);
  cx<TS>* Ap = Gm + rr;
  cx<TS>* P = Ap + rr;
  cx<TS>* V = P + rr;
  cx<TS>* Wk = V + rr;
  cx<TS>* Dgm = Wk + 2 * rr;
  cx<TS>* pivbuf = Dgm + rr;  // 3 r
  TS* sred = reinterpret_cast<TS*>(pivbuf + 3 * r);
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const double rho1 = (double)d.rho1;
  const cx<T>* part = d.Gpart + (size_t)k * d.gch * 3 * rr;
  const cx<T>* Xp = d.Tb + (size_t)k * r * n1;
  cx<T>* X = d.Xt + (size_t)k * r * n1;
  const int nx = r * n1, nt = blockDim.x;
  if (sizeof(T) == 4 && realslice) {
    // FP64 G^+ of a real slice (real_gram_solve_store); the partials are the
    // compensated sums of k_xg
    cx<double>* M64 = reinterpret_cast<cx<double>*>(smem);
    for (int task = tid; task < rr; task += blockDim.x) {
      cx<double> a0, hh, dd;
      sum_partials(part, rr, d.gch, task, true, a0, hh, dd);
      real_gram_G(M64, rr)[task] = cx<double>{a0.re + rho1 * hh.re, 0.0};
      real_gram_Dg(M64, rr)[task] = cx<double>{-(dd.re + rho1 * hh.re), 0.0};
    }
    __syncthreads();
    real_gram_solve_store<T, 32>(d, k, M64);
    for (int e = tid; e < nx; e += nt) X[e] = Xp[e];
    return;
  }
  for (int task = tid; task < rr; task += blockDim.x) {
    const int s = task / r, u = task - s * r;
    cx<double> a0, hh, dd;
    sum_partials(part, rr, d.gch, task, realslice, a0, hh, dd);
    cx<double> dg = {-(dd.re + rho1 * hh.re), -(dd.im + rho1 * hh.im)};
    if (realslice) dg.im = 0.0;
    Dgm[task] = cvt<TS>(dg);
    if (s <= u) {
      cx<double> g = {a0.re + rho1 * hh.re, a0.im + rho1 * hh.im};
      if (s == u || realslice) g.im = 0.0;
      Gm[s * r + u] = cvt<TS>(g);
      Gm[u * r + s] = cx<TS>{(TS)g.re, (TS)(-g.im)};
    }
  }
  __syncthreads();
  constexpr bool kDF = sizeof(T) == 4 && sizeof(TS) == 8;
  block_pinv_herm<TS, 32, kDF>(Gm, Ap, P, V, Wk, pivbuf, sred, r, (TS)d.rtol, d.scaled != 0);
  const TS t2 = d.scaled ? ((sred[2] > TS(0)) ? (TS)d.beta / sred[2] : TS(0)) : TS(1);
  for (int e = tid; e < rr; e += blockDim.x) {
    cx<T> gp = cvt<T>(Ap[e] * t2);
    if (realslice) gp.im = T(0);
    d.Dg[(size_t)k * rr + e] = cvt<T>(Dgm[e]);
    d.Gp[(size_t)k * rr + e] = gp;
  }
  int e = tid;
  for (; e + 3 * nt < nx; e += 4 * nt) {  // four loads in flight per thread
    cx<T> v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = Xp[e + q * nt];
#pragma unroll
    for (int q = 0; q < 4; ++q) X[e + q * nt] = v[q];
  }
  for (; e < nx; e += nt) X[e] = Xp[e];
}

}  // namespace tc
