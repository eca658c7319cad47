// Per-slice solvers of the TCTF2R iteration (Sec. 4.1, Eq. (updataXYW1)):
// the X-step contraction, the FP64 pseudo-inverses, the X-step and the Y-step.
#pragma once

namespace tc {

// ---------------------------------------------------------------------------
// Pseudo-inverse of a Hermitian PSD r x r matrix in the working precision T
// (Lemma "SVPMPI": A^+ = V diag(1/lambda) V^* over the eigenvalues above the
// cutoff rtol * lambda_max).
//
// Fast path (block-wide): Gauss-Jordan inverse without pivoting (stable for
// Hermitian positive definite A), accepted only when ||A||_1 ||A^-1||_1 <
// 1/(10 rtol) (1-norms bounded above through |re| + |im|), which certifies
// lambda_min > rtol * lambda_max: no eigenvalue is cut, A^+ = A^-1 and the
// projector A A^+ is exactly I.  Otherwise warp 0 runs a cyclic Jacobi
// eigendecomposition that applies the cutoff rule literally.
//
// A, Ap, P, V: r*r row-major complex values in shared memory; W: 2*r*r work;
// piv: 3*r complex values; sred: 2 values.  Every thread of the block must
// call it.  Returns (block-uniform) 1 if the inverse path was taken.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline void warp_jacobi_pinv(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, int r, T rtol);

template <typename T>
__device__ inline T warp_norm1_bound(const cx<T>* M, int ld, int col0, int r) {
  const int lane = threadIdx.x & 31;
  T nrm = T(0);
  for (int j = lane; j < r; j += 32) {
    T s = T(0);
    for (int i = 0; i < r; ++i) s += fabs(M[i * ld + col0 + j].re) + fabs(M[i * ld + col0 + j].im);
    nrm = fmax(nrm, s);
  }
  for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
  return nrm;
}

// 1/a.  FP64: a correctly rounded FP32 seed and two Newton steps
// y <- y (2 - a y) (the error squares at each step); FP64 division is slow on
// this part.  FP32: the IEEE quotient.
__device__ __forceinline__ double rcp_refined(double a) {
  const float af = (float)a;
  if (!(fabsf(af) > 1e-30f && fabsf(af) < 1e30f)) return 1.0 / a;
  double y = (double)__frcp_rn(af);
  y = y * fma(-a, y, 2.0);
  y = y * fma(-a, y, 2.0);
  return y;
}
__device__ __forceinline__ float rcp_refined(float a) { return 1.0f / a; }

// Smallest positive normal number of T, as a guard for pivots.
template <typename T>
__device__ __forceinline__ T tiny_pivot() {
  return sizeof(T) == 8 ? T(1e-300) : T(1e-37f);
}

template <typename T>
__device__ inline int block_pinv_herm(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, cx<T>* piv, T* sred,
                                      int r, T rtol) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n2c = 2 * r;  // augmented columns [A | I], row-major r x 2r
  cx<T>* colp = piv;
  cx<T>* rowp = piv + r;
  for (int e = tid; e < r * n2c; e += nt) {
    const int i = e / n2c, j = e - i * n2c;
    W[e] = (j < r) ? A[i * r + j] : cx<T>{(j - r == i) ? T(1) : T(0), T(0)};
  }
  if (tid < 32) {
    const T an = warp_norm1_bound(A, r, 0, r);
    if (tid == 0) sred[0] = an;
  }
  __syncthreads();
  const T anorm = sred[0];
  int ok = (anorm > T(0)) && isfinite(anorm);
  for (int p = 0; p < r && ok; ++p) {
    const T pv = W[p * n2c + p].re;
    if (!((pv > tiny_pivot<T>()) && isfinite(pv))) {
      ok = 0;
      break;
    }
    const T ip = rcp_refined(pv);
    for (int e = tid; e < r + n2c; e += nt) {
      if (e < r) colp[e] = W[e * n2c + p];
      else rowp[e - r] = W[p * n2c + (e - r)] * ip;
    }
    __syncthreads();
    for (int e = tid; e < r * n2c; e += nt) {
      const int i = e / n2c, j = e - i * n2c;
      W[e] = (i == p) ? rowp[j] : W[e] - cmul(colp[i], rowp[j]);
    }
    __syncthreads();
  }
  if (ok) {
    if (tid < 32) {
      const T in = warp_norm1_bound(W, n2c, r, r);
      if (tid == 0) sred[1] = in;
    }
    __syncthreads();
    const T inorm = sred[1];
    ok = isfinite(inorm) && (anorm * inorm < T(0.1) / rtol);
  }
  if (ok) {
    for (int e = tid; e < r * r; e += nt) {
      const int i = e / r, j = e - i * r;
      // symmetrise: A^-1 of a Hermitian matrix is Hermitian
      const cx<T> a = W[i * n2c + r + j];
      const cx<T> b = W[j * n2c + r + i];
      Ap[e] = cx<T>{T(0.5) * (a.re + b.re), T(0.5) * (a.im - b.im)};
      P[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
    }
    __syncthreads();
    return 1;
  }
  __syncthreads();
  if (tid < 32) warp_jacobi_pinv<T>(A, Ap, P, V, W, r, rtol);
  __syncthreads();
  return 0;
}

// Cyclic complex Jacobi eigendecomposition A = V diag(lambda) V^* by one warp,
// then A^+ and P = A A^+ with the cutoff rule.
template <typename T>
__device__ inline void warp_jacobi_pinv(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, int r, T rtol) {
  const int lane = threadIdx.x & 31;
  // ---- cyclic Jacobi on a copy of A (stored in W, row-major r x r) ----------
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    W[e] = A[e];
    const int i = e / r, j = e - i * r;
    V[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
  }
  __syncwarp();
  T fro = T(0);
  for (int e = lane; e < r * r; e += 32) fro += W[e].re * W[e].re + W[e].im * W[e].im;
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  // converged when the off-diagonal mass is below (unit roundoff)^2 of the total
  const T tol = (sizeof(T) == 8 ? T(1e-30) : T(1e-14f)) * fro + tiny_pivot<T>();
  for (int sweep = 0; sweep < 60; ++sweep) {
    T off = T(0);
    for (int e = lane; e < r * r; e += 32) {
      const int i = e / r, j = e - i * r;
      if (i != j) off += W[e].re * W[e].re + W[e].im * W[e].im;
    }
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (off <= tol) break;
    for (int p = 0; p < r - 1; ++p) {
      for (int q = p + 1; q < r; ++q) {
        const cx<T> c = W[p * r + q];
        const T ac = hypot(c.re, c.im);
        if (ac <= tiny_pivot<T>()) continue;
        const T a = W[p * r + p].re, b = W[q * r + q].re;
        const cx<T> u = {c.re / ac, c.im / ac};
        const T tau = (b - a) / (T(2) * ac);
        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
        const T cs = T(1) / sqrt(T(1) + t * t), sn = t * cs;
        __syncwarp();
        // columns: A J with J = [[cs, sn u], [-sn conj(u), cs]]
        for (int i = lane; i < r; i += 32) {
          const cx<T> aip = W[i * r + p], aiq = W[i * r + q];
          W[i * r + p] = aip * cs - cmulc(aiq, u) * sn;
          W[i * r + q] = cmul(aip, u) * sn + aiq * cs;
          const cx<T> vip = V[i * r + p], viq = V[i * r + q];
          V[i * r + p] = vip * cs - cmulc(viq, u) * sn;
          V[i * r + q] = cmul(vip, u) * sn + viq * cs;
        }
        __syncwarp();
        // rows: J^H (A J)
        for (int j = lane; j < r; j += 32) {
          const cx<T> apj = W[p * r + j], aqj = W[q * r + j];
          W[p * r + j] = apj * cs - cmul(aqj, u) * sn;
          W[q * r + j] = cmulc(apj, u) * sn + aqj * cs;
        }
        __syncwarp();
      }
    }
  }
  // eigenvalues on the diagonal; cutoff relative to lambda_max
  T lmax = T(0);
  for (int i = 0; i < r; ++i) lmax = fmax(lmax, W[i * r + i].re);
  const T cut = rtol * lmax;
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int i = e / r, j = e - i * r;
    cx<T> sa = {T(0), T(0)}, sp = {T(0), T(0)};
    for (int m = 0; m < r; ++m) {
      const T lam = W[m * r + m].re;
      if (lmax > T(0) && lam > cut) {
        const cx<T> vv = cmulc(V[i * r + m], V[j * r + m]);  // V_im conj(V_jm)
        sa = sa + vv * (T(1) / lam);
        sp = sp + vv;
      }
    }
    Ap[e] = sa;
    P[e] = sp;
  }
  __syncwarp();
}

// Upper-triangle task index -> (s, u), s <= u.
__device__ __forceinline__ void tri_index(int task, int r, int& s, int& u) {
  int rem = task;
  s = 0;
  while (rem >= r - s) {
    rem -= r - s;
    ++s;
  }
  u = s + rem;
}

constexpr int kSliceThreads = 256;

// ---------------------------------------------------------------------------
// Sum each of F values over the 32 lanes of a warp with F - 1 + (5 - log2 F)
// shuffles (butterfly that halves the live values at every level).  On return
// v[0] of lane l holds the total of value index l >> (5 - log2 F).  F <= 32.
// ---------------------------------------------------------------------------
template <typename T, int F>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[F]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int n = F, o = 16; n > 1; n >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const T send = up ? v[i] : v[i + n / 2];
      const T keep = up ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T x = v[0];
#pragma unroll
  for (int o = 16 / F; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int F>
struct Log2 {
  static constexpr int value = (F <= 1) ? 0 : 1 + Log2<F / 2>::value;
};
template <>
struct Log2<1> {
  static constexpr int value = 0;
};

// ---------------------------------------------------------------------------
// Q_k = R~_k Y~_k^H (n1 x r per slice), the W~Y~^H part of the X-gradient of
// Eq. (hkXYDer) that involves the residual.  Grid (S, ceil(n1/32)); one warp
// per row with coalesced loads along the row, Y~_k staged in shared memory.
// Reads R~ once.
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void __launch_bounds__(kSliceThreads) k_qcon(Dev<T> d, cx<T>* __restrict__ Qout) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* Ys = reinterpret_cast<cx<T>*>(smem);  // [r][n2]
  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  for (int e = tid; e < r * n2; e += blockDim.x) Ys[e] = Y[e];
  __syncthreads();
  constexpr int HALF = (RP > 16) ? 16 : RP;  // complex values per reduction pass
  for (int ii = wid; ii < 32; ii += nw) {
    const int i = blockIdx.y * 32 + ii;
    if (i >= n1) break;
    const cx<T>* row = d.Rt + ((size_t)i * S + k) * n2;
    cx<T> acc[RP];
#pragma unroll
    for (int s = 0; s < RP; ++s) acc[s] = cx<T>{T(0), T(0)};
    for (int j = lane; j < n2; j += 32) {
      const cx<T> v = ldg_cx(row + j);
#pragma unroll
      for (int s = 0; s < RP; ++s)
        if (s < r) cfmac(acc[s], v, Ys[(size_t)s * n2 + j]);
    }
#pragma unroll
    for (int h = 0; h < RP; h += HALF) {
      T f[2 * HALF];
#pragma unroll
      for (int s = 0; s < HALF; ++s) {
        f[2 * s] = acc[h + s].re;
        f[2 * s + 1] = acc[h + s].im;
      }
      const T tot = warp_reduce_scatter<T, 2 * HALF>(f);
      const int idx = lane >> (5 - Log2<2 * HALF>::value);
      const int s = h + idx / 2;
      const bool first = (lane & ((32 >> Log2<2 * HALF>::value) - 1)) == 0;
      if (first && s < r) reinterpret_cast<T*>(Qout + ((size_t)k * r + s) * n1 + i)[idx & 1] = tot;
    }
  }
}

// ---------------------------------------------------------------------------
// X-step of slice k (step 1 of the algorithm: Eq. (updataXYW1) with the
// gradients of Eq. (hkXYDer)) followed by the r x r preparation of the Y-step
// (step 2).  With W~ = X~Y~ + R~ and Q = R~Y~^H the X-gradient is
// grad_X = -Q + rho1 H^T H X~ A, so the update is
//   X~' = X~ + t d_X,  d_X = -H_rho1^{-1} grad_X A^+ = H_rho1^{-1} (Q A^+ - rho1 H^T H X~ P),
//   A = Y~Y~^H, P = A A^+, t = 1 (exact step).
// With E = X~'^H X~ and G = X~'^H H_rho1 X~', the Y-gradient at X~' is
// grad_Y = (G - E) Y~ - D, D = X~'^H R~, so k_ystep forms
//   Y~' = Y~ + t G^+ (Dg Y~ + D),  Dg = E - G = -X~'^H (X~' - X~) - rho1 (H X~')^H (H X~').
// Each new factor is the old one plus a correction that shrinks as the
// iteration converges, so rounding in the working precision T touches only
// the correction.  The pseudo-inverses are taken in T as well.
// One CTA per slice.  Work arrays in shared memory when they fit, else in the
// per-slice region of d.Tb.
// ---------------------------------------------------------------------------
struct XLayout {
  size_t mats, ht, xs, qs, ts, total;
};

template <typename T>
__host__ __device__ inline XLayout xstep_layout(int n1, int n2, int r, bool arrays_in_smem) {
  XLayout L{};
  const size_t rr = (size_t)r * r;
  size_t off = 0;
  L.mats = off;  // A, A^+, P, V, work (2), G, Dg, pivots, reductions
  off = align_up(off + (rr * 8 + 3 * (size_t)r + 2) * sizeof(cx<T>), 16);
  L.ht = off;
  off = align_up(off + sizeof(T) * 2 * n1, 16);
  if (arrays_in_smem) {
    L.xs = off;
    off = align_up(off + sizeof(cx<T>) * r * n1, 16);
    L.qs = off;
    off = align_up(off + sizeof(cx<T>) * r * n1, 16);
    L.ts = off;
    off = align_up(off + sizeof(cx<T>) * r * n1, 16);
  }
  L.total = off;
  return L;
}

// (H^T H x)_i for the first-difference matrix H of Eq. (Toeplitz) on n1 entries:
// deg_i x_i - x_{i-1} - x_{i+1} over the neighbours that exist.
template <typename T>
__device__ __forceinline__ cx<T> hth_at(const cx<T>* x, int i, int n1) {
  cx<T> v = {T(0), T(0)};
  const cx<T> xi = x[i];
  if (i > 0) v = v + (xi - x[i - 1]);
  if (i + 1 < n1) v = v + (xi - x[i + 1]);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kSliceThreads) k_xstep(Dev<T> d, const cx<T>* __restrict__ Qin, int arrays_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const XLayout lay = xstep_layout<T>(n1, n2, r, arrays_in_smem != 0);
  cx<T>* A = reinterpret_cast<cx<T>*>(smem + lay.mats);
  cx<T>* Ap = A + rr;
  cx<T>* P = Ap + rr;
  cx<T>* V = P + rr;
  cx<T>* Wk = V + rr;
  cx<T>* Gm = Wk + 2 * rr;
  cx<T>* Dgm = Gm + rr;
  cx<T>* pivbuf = Dgm + rr;  // 3 r
  T* sred = reinterpret_cast<T*>(pivbuf + 3 * r);
  T* hinv = reinterpret_cast<T*>(smem + lay.ht);
  T* ha = hinv + n1;
  cx<T>* Xs;
  cx<T>* Qs;
  cx<T>* Ts;
  cx<T>* Xg = d.Xt + (size_t)k * r * n1;
  const cx<T>* Qg = Qin + (size_t)k * r * n1;
  if (arrays_in_smem) {
    Xs = reinterpret_cast<cx<T>*>(smem + lay.xs);
    Qs = reinterpret_cast<cx<T>*>(smem + lay.qs);
    Ts = reinterpret_cast<cx<T>*>(smem + lay.ts);
    for (int e = tid; e < r * n1; e += blockDim.x) {
      Xs[e] = Xg[e];
      Qs[e] = Qg[e];
    }
  } else {
    Xs = Xg;
    Qs = const_cast<cx<T>*>(Qg);
    Ts = d.Tb + (size_t)k * r * n1;
  }
  for (int i = tid; i < 2 * n1; i += blockDim.x) hinv[i] = d.hinv[i];
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const T rho1 = d.rho1;
  const T rtol = (T)d.rtol;

  // ---- A = Y~Y~^H: FP64 sums of the 32-column tile Grams written by k_ystep ----------
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
      A[s * r + u] = cx<T>{(T)v.re, (T)v.im};
      A[u * r + s] = cx<T>{(T)v.re, (T)(-v.im)};
    }
  }
  __syncthreads();
  const bool certA = block_pinv_herm<T>(A, Ap, P, V, Wk, pivbuf, sred, r, rtol) != 0;

  // ---- B = Q A^+ - rho1 (H^T H X~) P ------------------------------------------------------
  for (int e = tid; e < r * n1; e += blockDim.x) {
    const int s = e / n1, i = e - s * n1;
    cx<T> acc = {T(0), T(0)};
    for (int u = 0; u < r; ++u) cfma(acc, Qs[(size_t)u * n1 + i], Ap[u * r + s]);
    if (rho1 != T(0)) {
      cx<T> hx = {T(0), T(0)};
      if (certA) {
        hx = hth_at(Xs + (size_t)s * n1, i, n1);  // P = I
      } else {
        for (int u = 0; u < r; ++u) cfma(hx, hth_at(Xs + (size_t)u * n1, i, n1), P[u * r + s]);
      }
      acc = acc - hx * rho1;
    }
    Ts[e] = acc;
  }
  __syncthreads();
  // ---- d_X = H_rho1^{-1} B: one column per thread, one FMA per step ---------------------
  if (rho1 != T(0) && n1 > 1) {
    constexpr int CH = 16;  // values staged in registers per chunk
    for (int s = tid; s < r; s += blockDim.x) {
      cx<T>* col = Ts + (size_t)s * n1;
      cx<T> y = {T(0), T(0)};
      for (int i0 = 0; i0 < n1; i0 += CH) {
        cx<T> v[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) v[q] = (i0 + q < n1) ? col[i0 + q] : cx<T>{T(0), T(0)};
#pragma unroll
        for (int q = 0; q < CH; ++q) {
          const int i = i0 + q;
          if (i < n1) {
            const T a = ha[i], b = hinv[i];
            y = cx<T>{fma(a, y.re, v[q].re * b), fma(a, y.im, v[q].im * b)};
            v[q] = y;
          }
        }
#pragma unroll
        for (int q = 0; q < CH; ++q)
          if (i0 + q < n1) col[i0 + q] = v[q];
      }
      cx<T> x = col[n1 - 1];
      for (int i1 = n1 - 2; i1 >= 0; i1 -= CH) {
        cx<T> v[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) v[q] = (i1 - q >= 0) ? col[i1 - q] : cx<T>{T(0), T(0)};
#pragma unroll
        for (int q = 0; q < CH; ++q) {
          const int i = i1 - q;
          if (i >= 0) {
            const T a = ha[i];
            x = cx<T>{fma(a, x.re, v[q].re), fma(a, x.im, v[q].im)};
            v[q] = x;
          }
        }
#pragma unroll
        for (int q = 0; q < CH; ++q)
          if (i1 - q >= 0) col[i1 - q] = v[q];
      }
    }
    __syncthreads();
  }
  // ---- X~' = X~ + d_X (Ts; Xs keeps the old factor) ---------------------------------------
  for (int e = tid; e < r * n1; e += blockDim.x) {
    cx<T> v = Xs[e] + Ts[e];
    if (realslice) v.im = T(0);
    Ts[e] = v;
  }
  __syncthreads();

  // ---- G = X~'^H H_rho1 X~' (Hermitian) and Dg = E - G ----------------------------------
  // (H X~')^H (H X~') = sum_i conj(x_i - x_{i+1}) (x_i - x_{i+1}) row by row
  for (int task = wid; task < rr; task += nw) {
    const int s = task / r, u = task - s * r;
    const cx<T>* xs = Ts + (size_t)s * n1;
    const cx<T>* xu = Ts + (size_t)u * n1;
    const cx<T>* ou = Xs + (size_t)u * n1;
    cx<T> a0 = {T(0), T(0)}, hh = {T(0), T(0)}, dd = {T(0), T(0)};
    for (int i = lane; i < n1; i += 32) {
      const cx<T> a = xs[i], b = xu[i];
      cfmaconj(a0, a, b);
      cfmaconj(dd, a, b - ou[i]);
      if (i + 1 < n1) cfmaconj(hh, a - xs[i + 1], b - xu[i + 1]);
    }
    T f[8] = {a0.re, a0.im, hh.re, hh.im, dd.re, dd.im, T(0), T(0)};
    const T tot = warp_reduce_scatter<T, 8>(f);  // lane l: value index l >> 2
    const T h_re = __shfl_sync(0xffffffffu, tot, 8), h_im = __shfl_sync(0xffffffffu, tot, 12);
    const T a_re = __shfl_sync(0xffffffffu, tot, 0), a_im = __shfl_sync(0xffffffffu, tot, 4);
    const T d_re = __shfl_sync(0xffffffffu, tot, 16), d_im = __shfl_sync(0xffffffffu, tot, 20);
    if (lane == 0) {
      cx<T> dg = {-(d_re + rho1 * h_re), -(d_im + rho1 * h_im)};
      if (realslice) dg.im = T(0);
      Dgm[s * r + u] = dg;
      if (s <= u) {
        cx<T> g = {a_re + rho1 * h_re, a_im + rho1 * h_im};
        if (s == u || realslice) g.im = T(0);
        Gm[s * r + u] = g;
        Gm[u * r + s] = cx<T>{g.re, -g.im};
      }
    }
  }
  __syncthreads();
  block_pinv_herm<T>(Gm, Ap, P, V, Wk, pivbuf, sred, r, rtol);
  // ---- Dg and G^+ for k_ystep; X~ <- X~' ---------------------------------------------------
  for (int e = tid; e < rr; e += blockDim.x) {
    cx<T> gp = Ap[e];
    if (realslice) gp.im = T(0);
    d.Dg[(size_t)k * rr + e] = Dgm[e];
    d.Gp[(size_t)k * rr + e] = gp;
  }
  for (int e = tid; e < r * n1; e += blockDim.x) Xg[e] = Ts[e];
}

// ---------------------------------------------------------------------------
// Y-step of slice k on a tile of 32 columns (step 2):
//   D   = X~'^H R~_k(:, tile)       (contraction over n1; reads R~ once)
//   Y~' = Y~ + G^+ (Dg Y~ + D)      (= Y~ - G^+ grad_Y, see k_xstep)
// then the tile Gram of Y~' (A of the next X-step) and Z~ = X~'Y~' on the tile
// (step 3, read by the slab kernel).
// Grid (S, ceil(n2/32)); warp w accumulates rows i = w, w + 8, ...
// ---------------------------------------------------------------------------
constexpr int kYThreads = 256;

template <typename T, int RP>
__global__ void __launch_bounds__(kYThreads) k_ystep(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * 32;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* red = reinterpret_cast<cx<T>*>(smem);  // [nw][RP][32]
  cx<T>* Ds = red + nw * RP * 32;               // [RP][32]
  cx<T>* Yo = Ds + RP * 32;                     // [RP][32]
  cx<T>* Dgs = Yo + RP * 32;                    // [rr]
  cx<T>* Gh = Dgs + rr;                         // [rr]
  cx<T>* Yn = Gh + rr;                          // [RP][32] the new Y~' of the tile
  cx<T>* Xs = Yn + RP * 32;                     // [r][n1]
  const cx<T>* Xg = d.Xt + (size_t)k * r * n1;
  for (int e = tid; e < r * n1; e += blockDim.x) Xs[e] = Xg[e];
  for (int e = tid; e < rr; e += blockDim.x) {
    Dgs[e] = d.Dg[(size_t)k * rr + e];
    Gh[e] = d.Gp[(size_t)k * rr + e];
  }
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    Yo[s * 32 + c] = (j0 + c < n2) ? d.Yt[((size_t)k * r + s) * n2 + j0 + c] : cx<T>{T(0), T(0)};
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
  // V = Dg Y~ + D (= -grad_Y on the tile)
  for (int e = tid; e < r * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    cx<T> v = {T(0), T(0)};
    for (int w = 0; w < nw; ++w) v = v + red[(w * RP + s) * 32 + c];
    for (int u = 0; u < r; ++u) cfma(v, Dgs[s * r + u], Yo[u * 32 + c]);
    Ds[s * 32 + c] = v;
  }
  __syncthreads();
  const bool realslice = (k == 0) || (2 * k == d.n3);
  for (int e = tid; e < RP * 32; e += blockDim.x) {
    const int s = e >> 5, c = e & 31;
    if (s >= r || j0 + c >= n2) {
      Yn[e] = cx<T>{T(0), T(0)};
      continue;
    }
    cx<T> y = Yo[e];
    for (int u = 0; u < r; ++u) cfma(y, Gh[s * r + u], Ds[u * 32 + c]);
    if (realslice) y.im = T(0);
    d.Yt[((size_t)k * r + s) * n2 + j0 + c] = y;
    Yn[e] = y;
  }
  __syncthreads();

  // ---- Gram of the new Y~' over this tile (A of the next X-step) ----------------------
  const int ntask = r * (r + 1) / 2;
  for (int task = wid; task < ntask; task += nw) {
    int s, u;
    tri_index(task, r, s, u);
    cx<T> g = {T(0), T(0)};
    cfmac(g, Yn[s * 32 + lane], Yn[u * 32 + lane]);
    g.re = warp_sum(g.re);
    g.im = warp_sum(g.im);
    if (lane == 0) d.Ag[((size_t)k * d.ytiles + blockIdx.y) * ntask + task] = cx<double>{(double)g.re, (double)g.im};
  }

  // ---- Z~(:, tile, k) = X~' Y~'  (step 3, written for the slab kernel) ----------------
  cx<T> yv[RP];
#pragma unroll
  for (int s = 0; s < RP; ++s) yv[s] = Yn[s * 32 + lane];
  if (j < n2) {
    cx<T>* zc = d.Zt + (size_t)k * n2 + j;
    for (int i = wid; i < n1; i += nw) {
      cx<T> z = {T(0), T(0)};
#pragma unroll
      for (int s = 0; s < RP; ++s)
        if (s < r) cfma(z, Xs[(size_t)s * n1 + i], yv[s]);
      zc[(size_t)i * S * n2] = z;
    }
  }
}

template <typename T>
__host__ inline size_t ystep_smem_bytes(int n1, int r, int rp) {
  return ((size_t)(kYThreads / 32 + 3) * rp * 32 + 2 * (size_t)r * r + (size_t)r * n1) * sizeof(cx<T>);
}

template <typename T>
__host__ inline size_t qcon_smem_bytes(int n2, int r, int) {
  return (size_t)r * n2 * sizeof(cx<T>);
}

}  // namespace tc
