// The X-step of large ranks (r > 16) spread over the GPU: one CTA per slice
// for a whole X-step (k_xstep) leaves most SMs idle and runs r^2 n1 Gram
// products on one SM.  Here the same step (Eq. (updataXYW1) with the gradients
// of Eq. (hkXYDer), formed as in k_xstep) is five kernels:
//   k_xa   (S CTAs)               A = Y~Y~^H from the tile Grams, A^+, P, step t1; run
//                                 after every change of Y~ (initialisation, each
//                                 Y-step), beside the rest of that iteration
//   k_xbg  (S x ceil(n1/128) CTAs) B = Q A^+ over 128-row chunks (register tiles), to d.Tb
//   k_xbc  (S x ceil(r/8) CTAs)   one warp per column: d_X = H_rho1^{-1}(B - rho1 (H^T H X~) P),
//                                 X~' = X~ + t1 d_X; with P = I written in place over X~
//                                 and X~' - X~ to d.Tb, else X~' to d.Tb
//   k_xg   (S x ceil(n1/64) CTAs) partial Grams over 64 rows: X~'^H X~', (H X~')^H (H X~'),
//                                 X~'^H (X~' - X~)
//   k_xc   (S CTAs)               the partials summed in a fixed order, G, Dg, t2 G^+ for
//                                 k_ystep; X~ <- X~' when P != I
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
  // FP64-storage solves of an FP32 engine: A also as FP32 head and tail (in V)
  // for herm_inverse_refined, whose work and result take W
  constexpr bool kDF = sizeof(T) == 4 && sizeof(TS) == 8;
  const bool refine = kDF && !d.scaled;
  cx<float>* ahf = reinterpret_cast<cx<float>*>(V);
  cx<float>* alf = ahf + rr;
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
      if (refine) {
        const cx<float> h = {(float)v.re, (float)v.im};
        const cx<float> l = {(float)(v.re - (double)h.re), (float)(v.im - (double)h.im)};
        ahf[s * r + u] = h;
        alf[s * r + u] = l;
        ahf[u * r + s] = cx<float>{h.re, -h.im};
        alf[u * r + s] = cx<float>{l.re, -l.im};
      }
    }
  }
  __syncthreads();
  if constexpr (kDF) {
    cx<float>* wf = alf + rr;  // 3 r^2
    cx<float>* xo = wf + 3 * rr;
    if (refine && herm_inverse_refined<true>(ahf, alf, xo, wf, reinterpret_cast<float*>(sred), r, d.rtol)) {
      for (int e = tid; e < rr; e += blockDim.x) {
        const int i = e / r, j = e - i * r;
        d.Apg[(size_t)k * rr + e] = cvt<T>(xo[e]);
        d.Pg[(size_t)k * rr + e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
      }
      if (tid == 0) {
        d.certA[k] = 1;
        d.tstep[k] = T(1);
      }
      return;
    }
    __syncthreads();
  }
  const bool cert =
      block_pinv_herm<TS, 32, kDF>(A, Ap, P, V, Wk, pivbuf, sred, r, (TS)d.rtol, d.scaled != 0, !refine) != 0;
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

// ---- B = Q A^+ over row chunks --------------------------------------------------------
// A CTA stages kXbRows rows of the slice's Q and A^+ (by rows) in shared
// memory; a thread forms an RT x CT tile of B, so each step over u loads RT
// values of Q and CT of A^+ for RT * CT products.  B goes to the work array
// d.Tb through shared memory (coalesced rows).
constexpr int kXbRows = 128;

template <typename T>
struct XbTile {  // rows x columns of B per thread
  static constexpr int R = sizeof(T) == 4 ? 4 : 2;
  static constexpr int C = sizeof(T) == 4 ? 4 : 2;
};

template <typename T>
__host__ __device__ inline size_t xbg_smem_bytes(int r) {
  return (32 * 32 + 2 * (size_t)r * kXbRows) * sizeof(cx<T>);
}

// N consecutive complex values from 16-byte aligned shared memory
template <int N>
__device__ __forceinline__ void ld_cxn(const cx<float>* p, cx<float> (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N / 2; ++q) {
    const float4 f = reinterpret_cast<const float4*>(p)[q];
    v[2 * q] = cx<float>{f.x, f.y};
    v[2 * q + 1] = cx<float>{f.z, f.w};
  }
}
template <int N>
__device__ __forceinline__ void ld_cxn(const cx<double>* p, cx<double> (&v)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) v[q] = p[q];
}

template <typename T>
__global__ void __launch_bounds__(256) k_xbg(Dev<T> d, const cx<T>* __restrict__ Qin) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, i0 = blockIdx.y * kXbRows, n1 = d.n1, r = d.r, rr = r * r;
  const int tid = threadIdx.x, nt = blockDim.x, nrow = min(kXbRows, n1 - i0);
  cx<T>* apr = reinterpret_cast<cx<T>*>(smem);  // [u][32] A^+ by rows
  cx<T>* qs = apr + 32 * 32;                    // [u][kXbRows] rows i0 .. of Q
  cx<T>* bsm = qs + (size_t)r * kXbRows;       // [s][kXbRows] the same rows of B
  for (int e = tid; e < 32 * 32; e += nt) {
    const int a = e >> 5, b = e & 31;
    apr[e] = (a < r && b < r) ? d.Apg[(size_t)k * rr + a * r + b] : cx<T>{T(0), T(0)};
  }
  {
    const cx<T>* Qk = Qin + (size_t)k * r * n1 + i0;
    const int nq = r * kXbRows;
    auto get = [&](int e) {
      const int u = e / kXbRows, ii = e - u * kXbRows;
      return ii < nrow ? ldg_cx(Qk + (size_t)u * n1 + ii) : cx<T>{T(0), T(0)};
    };
    int e = tid;
    for (; e + 3 * nt < nq; e += 4 * nt) {  // four loads in flight per thread
      cx<T> v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = get(e + q * nt);
#pragma unroll
      for (int q = 0; q < 4; ++q) qs[e + q * nt] = v[q];
    }
    for (; e < nq; e += nt) qs[e] = get(e);
  }
  __syncthreads();
  constexpr int RT = XbTile<T>::R, CT = XbTile<T>::C;
  const int ncg = (r > 16 ? 32 : 16) / CT;  // column groups
  const int cg = tid % ncg, s0 = cg * CT;
  const int rstep = (nt / ncg) * RT;
  for (int ii = (tid / ncg) * RT; ii < nrow; ii += rstep) {
    cx<T> acc[RT][CT];
#pragma unroll
    for (int x = 0; x < RT; ++x)
#pragma unroll
      for (int y = 0; y < CT; ++y) acc[x][y] = cx<T>{T(0), T(0)};
#pragma unroll 2
    for (int u = 0; u < r; ++u) {
      cx<T> q[RT], a[CT];
      ld_cxn<RT>(qs + (size_t)u * kXbRows + ii, q);
      ld_cxn<CT>(apr + u * 32 + s0, a);
#pragma unroll
      for (int x = 0; x < RT; ++x)
#pragma unroll
        for (int y = 0; y < CT; ++y) cfma(acc[x][y], q[x], a[y]);
    }
#pragma unroll
    for (int x = 0; x < RT; ++x)
#pragma unroll
      for (int y = 0; y < CT; ++y)
        if (s0 + y < r) bsm[(size_t)(s0 + y) * kXbRows + ii + x] = acc[x][y];
  }
  __syncthreads();
  cx<T>* Bk = d.Tb + (size_t)k * r * n1 + i0;
  for (int e = tid; e < r * kXbRows; e += nt) {
    const int s = e / kXbRows, ii = e - s * kXbRows;
    if (ii < nrow) Bk[(size_t)s * n1 + ii] = bsm[e];
  }
}

// ---- d_X = H_rho1^{-1}(B - rho1 (H^T H X~) P) and X~' per column ------------------------
// One warp per column s of slice k (grid S x ceil(r/8), 8 warps).  When A^+ =
// A^-1 (P = I) and the step is the exact one, d_X = H_rho1^{-1}(B + X~) - X~
// (H_rho1 = I + rho1 H^T H), so X~' = H_rho1^{-1}(X~ + B) needs no H^T H
// stencil.  With P = I the warp reads only its own column of X~ and writes
// X~' in place over it, with X~' - X~ over B in d.Tb; otherwise (P != I, the
// stencil reads every column) X~' goes to d.Tb and k_xc copies it back.
template <typename T>
__host__ __device__ inline size_t xbc_smem_bytes(int n1) {
  // H_rho1 tables, then per warp its column of B (then d_X) and of X~
  return align_up(2 * (size_t)n1 * sizeof(T), 16) + 2 * 8 * (size_t)n1 * sizeof(cx<T>);
}

template <typename T>
__global__ void __launch_bounds__(256) k_xbc(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x, n1 = d.n1, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int s = blockIdx.y * 8 + wid;
  T* hinv = reinterpret_cast<T*>(smem);
  T* ha = hinv + n1;
  cx<T>* col = reinterpret_cast<cx<T>*>(smem + align_up(2 * (size_t)n1 * sizeof(T), 16)) + (size_t)wid * n1;
  cx<T>* xsm = col + 8 * (size_t)n1;  // the warp's column of X~ (read once from L2)
  for (int i = tid; i < 2 * n1; i += blockDim.x) hinv[i] = d.hinv[i];
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const bool certA = d.certA[k] != 0, fast = certA && !d.scaled;
  const T rho1 = d.rho1, t1 = d.tstep[k];
  double dmax = 0.0;
  if (s < r) {
    const cx<T>* Xk = d.Xt + (size_t)k * r * n1;
    cx<T>* xs = d.Xt + (size_t)k * r * n1 + (size_t)s * n1;
    cx<T>* bs = d.Tb + (size_t)k * r * n1 + (size_t)s * n1;
    {
      int i = lane;
      for (; i + 224 < n1; i += 256) {  // eight pairs of loads in flight per lane
        cx<T> b[8], x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          b[q] = bs[i + 32 * q];
          x[q] = xs[i + 32 * q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          col[i + 32 * q] = fast ? b[q] + x[q] : b[q];
          xsm[i + 32 * q] = x[q];
        }
      }
      for (; i < n1; i += 32) {
        const cx<T> b = bs[i], x = xs[i];
        col[i] = fast ? b + x : b;
        xsm[i] = x;
      }
    }
    if (!fast && rho1 != T(0)) {
      const cx<T>* pg = d.Pg + (size_t)k * rr;
      for (int i = lane; i < n1; i += 32) {
        cx<T> hx = {T(0), T(0)};
        if (certA) {
          hx = hth_at(xs, i, n1);  // P = I
        } else {
          for (int u = 0; u < r; ++u) cfma(hx, hth_at(Xk + (size_t)u * n1, i, n1), pg[u * r + s]);
        }
        col[i] = col[i] - hx * rho1;
      }
    }
    __syncwarp();
    if (rho1 != T(0) && n1 > 1) warp_tridiag_solve<T>(col, n1, hinv, ha);
    __syncwarp();
    auto update = [&](int i, cx<T> x0) {
      cx<T> v = fast ? col[i] : (d.scaled ? x0 + col[i] * t1 : x0 + col[i]);
      if (realslice) v.im = T(0);
      if (certA) {
        xs[i] = v;
        bs[i] = v - x0;
      } else {
        bs[i] = v;
      }
      if (d.conv) dmax = fmax(dmax, (double)cabs(v - x0));
    };
    for (int i = lane; i < n1; i += 32) update(i, xsm[i]);
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
  cx<T>* go = gx + (size_t)r * kXgLd;          // [r][kXgLd] rows i0 .. of X~' - X~
  // k_xbc left X~' in d.Xt and X~' - X~ in d.Tb when P = I, else X~' in d.Tb
  const bool inplace = d.certA[k] != 0;
  const cx<T>* Xp = (inplace ? d.Xt : d.Tb) + (size_t)k * r * n1;
  const cx<T>* X2 = (inplace ? d.Tb : d.Xt) + (size_t)k * r * n1;
  const int nrow = min(kXgRows + 1, n1 - i0);
  for (int e = tid; e < r * kXgLd; e += blockDim.x) {
    const int s = e / kXgLd, ii = e - s * kXgLd;
    if (ii < nrow) {
      const cx<T> xp = Xp[(size_t)s * n1 + i0 + ii];
      gx[e] = xp;
      if (ii < kXgRows) go[e] = inplace ? X2[(size_t)s * n1 + i0 + ii] : xp - X2[(size_t)s * n1 + i0 + ii];
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
        dot2(s2, c2, a, ou[ii].re);
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
        e[x] = ou[x][ii];
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

// Sums of the k_xg partials of one Gram entry in chunk order.  FP32 engines:
// real slices add the (sum, compensation) pairs as df64 values; complex slices
// add in FP32, as the partials themselves were accumulated.  Four chunks (12
// loads) are in flight at a time.  FP64 engines: FP64.
__device__ __forceinline__ void sum_partials(const cx<float>* part, int rr, int gch, int task, bool realslice,
                                             cx<double>& a0, cx<double>& hh, cx<double>& dd) {
  df s[3] = {};
  cx<float> f[3] = {};
  auto add = [&](int q, cx<float> v) {
    if (realslice) s[q] = df_add(s[q], df_norm(v.re, v.im));
    else f[q] = f[q] + v;
  };
  int c = 0;
  for (; c + 4 <= gch; c += 4) {
    cx<float> v[4][3];
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[w][q] = part[((size_t)(c + w) * 3 + q) * rr + task];
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) add(q, v[w][q]);
  }
  if (c < gch) {
    cx<float> v[3][3];
#pragma unroll
    for (int w = 0; w < 3; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[w][q] = c + w < gch ? part[((size_t)(c + w) * 3 + q) * rr + task] : cx<float>{0.f, 0.f};
#pragma unroll
    for (int w = 0; w < 3; ++w)
      if (c + w < gch)
#pragma unroll
        for (int q = 0; q < 3; ++q) add(q, v[w][q]);
  }
  if (realslice) {
    a0 = cx<double>{df_to(s[0]), 0.0};
    hh = cx<double>{df_to(s[1]), 0.0};
    dd = cx<double>{df_to(s[2]), 0.0};
  } else {
    a0 = cx<double>{(double)f[0].re, (double)f[0].im};
    hh = cx<double>{(double)f[1].re, (double)f[1].im};
    dd = cx<double>{(double)f[2].re, (double)f[2].im};
  }
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

// FP32 sums of the partials of a complex slice (FP32 engines)
__device__ __forceinline__ void sum_partials_f32(const cx<float>* part, int rr, int gch, int task, cx<float>& a0,
                                                 cx<float>& hh, cx<float>& dd) {
  cx<float> f[3] = {};
  int c = 0;
  for (; c + 4 <= gch; c += 4) {
    cx<float> v[4][3];
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[w][q] = part[((size_t)(c + w) * 3 + q) * rr + task];
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] = f[q] + v[w][q];
  }
  if (c < gch) {
    cx<float> v[3][3];
#pragma unroll
    for (int w = 0; w < 3; ++w)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[w][q] = c + w < gch ? part[((size_t)(c + w) * 3 + q) * rr + task] : cx<float>{0.f, 0.f};
#pragma unroll
    for (int w = 0; w < 3; ++w)
      if (c + w < gch)
#pragma unroll
        for (int q = 0; q < 3; ++q) f[q] = f[q] + v[w][q];
  }
  a0 = f[0];
  hh = f[1];
  dd = f[2];
}

// ---- G, Dg from the partials, t2 G^+; X~ <- X~' when P != I -------------------------------
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
  cx<TS>* pivbuf = Wk + 3 * rr;  // 3 r (after Wk and a free r^2)
  TS* sred = reinterpret_cast<TS*>(pivbuf + 3 * r);
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const cx<T>* part = d.Gpart + (size_t)k * d.gch * 3 * rr;
  const int nx = r * n1, nt = blockDim.x;
  if (!d.certA[k]) {
    // k_xbc wrote X~' to the work array (P != I; nothing below reads X~)
    const cx<T>* Xp = d.Tb + (size_t)k * r * n1;
    cx<T>* X = d.Xt + (size_t)k * r * n1;
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
  const double rho1 = (double)d.rho1;
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
    return;
  }
  constexpr bool kDF = sizeof(T) == 4 && sizeof(TS) == 8;
  // FP64-storage solve of an FP32 engine: G in FP32 (in V) for herm_inverse_refined,
  // whose work and result take the rest of V and W; G in FP64 only if that fails
  const bool refine = kDF && !d.scaled;
  cx<float>* ghf = reinterpret_cast<cx<float>*>(V);
  for (int task = tid; task < rr; task += blockDim.x) {
    const int s = task / r, u = task - s * r;
    if constexpr (kDF) {
      cx<float> a0, hh, dd;
      sum_partials_f32(reinterpret_cast<const cx<float>*>(part), rr, d.gch, task, a0, hh, dd);
      const float rf = d.rho1;
      d.Dg[(size_t)k * rr + task] = cx<T>{-fmaf(rf, hh.re, dd.re), -fmaf(rf, hh.im, dd.im)};
      if (s <= u) {
        cx<float> g = {fmaf(rf, hh.re, a0.re), fmaf(rf, hh.im, a0.im)};
        if (s == u) g.im = 0.f;
        ghf[s * r + u] = g;
        ghf[u * r + s] = cx<float>{g.re, -g.im};
      }
    } else {
      cx<double> a0, hh, dd;
      sum_partials(part, rr, d.gch, task, realslice, a0, hh, dd);
      cx<double> dg = {-(dd.re + rho1 * hh.re), -(dd.im + rho1 * hh.im)};
      if (realslice) dg.im = 0.0;
      d.Dg[(size_t)k * rr + task] = cvt<T>(dg);
      if (s <= u) {
        cx<double> g = {a0.re + rho1 * hh.re, a0.im + rho1 * hh.im};
        if (s == u || realslice) g.im = 0.0;
        Gm[s * r + u] = cvt<TS>(g);
        Gm[u * r + s] = cx<TS>{(TS)g.re, (TS)(-g.im)};
      }
    }
  }
  __syncthreads();
  if constexpr (kDF) {
    cx<float>* wf = ghf + rr;  // 3 r^2
    cx<float>* xo = wf + 3 * rr;
    if (refine && herm_inverse_refined<false>(ghf, nullptr, xo, wf, reinterpret_cast<float*>(sred), r, d.rtol)) {
      for (int e = tid; e < rr; e += blockDim.x) d.Gp[(size_t)k * rr + e] = cvt<T>(xo[e]);
      return;
    }
    for (int e = tid; e < rr; e += blockDim.x) Gm[e] = cx<TS>{(TS)ghf[e].re, (TS)ghf[e].im};
    __syncthreads();
  }
  block_pinv_herm<TS, 32, kDF>(Gm, Ap, P, V, Wk, pivbuf, sred, r, (TS)d.rtol, d.scaled != 0, !refine);
  const TS t2 = d.scaled ? ((sred[2] > TS(0)) ? (TS)d.beta / sred[2] : TS(0)) : TS(1);
  for (int e = tid; e < rr; e += blockDim.x) {
    cx<T> gp = cvt<T>(d.scaled ? Ap[e] * t2 : Ap[e]);
    if (realslice) gp.im = T(0);
    d.Gp[(size_t)k * rr + e] = gp;
  }
}

}  // namespace tc
