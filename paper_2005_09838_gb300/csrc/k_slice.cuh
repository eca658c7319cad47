// Per-slice solvers of the TCTF2R iteration (Sec. 4.1, Eq. (updataXYW1)):
// the X-step contraction, the FP64 pseudo-inverses, the X-step and the Y-step.
#pragma once

namespace tc {

// ---------------------------------------------------------------------------
// Pseudo-inverse of a Hermitian PSD r x r matrix in the working precision T
// (Lemma "SVPMPI": A^+ = V diag(1/lambda) V^* over the eigenvalues above the
// cutoff rtol * lambda_max).
//
// Fast path: Gauss-Jordan inverse without pivoting (stable for Hermitian
// positive definite A), accepted only when a bound on lambda_max/lambda_min
// stays below a fraction of 1/rtol, which certifies lambda_min > rtol *
// lambda_max: no eigenvalue is cut, A^+ = A^-1 and the projector A A^+ is
// exactly I.  r <= 16: one warp with the matrix in registers, bound
// ||A||_F ||A^-1||_F < 1/(2 rtol) (lambda_max <= ||A||_F, 1/lambda_min =
// ||A^-1||_2 <= ||A^-1||_F; at that size the computed inverse is within a
// few percent of the true one).  Larger r: the block, same bound.
// Otherwise warp 0 runs a parallel cyclic Jacobi eigendecomposition
// (round-robin pairs, r/2 rotations at a time) that applies the cutoff rule
// literally.
//
// A, Ap, P, V: r*r row-major complex values in shared memory; W: 2*r*r work;
// piv: 3*r complex values; sred: 4 values.  Every thread of the block must
// call it.  Returns (block-uniform) 1 if the inverse path was taken.
// ---------------------------------------------------------------------------
template <typename TS, bool DF>
__device__ __noinline__ void jacobi_fallback(const cx<TS>* A, cx<TS>* Ap, cx<TS>* P, cx<TS>* V, cx<TS>* W, cx<TS>* piv,
                                       int r, TS rtol, TS* lmax_out);

// Frobenius norm of the r x r block at column col0 of a row-major matrix with
// leading dimension ld, by one warp.
template <typename T>
__device__ inline T warp_frob(const cx<T>* M, int ld, int col0, int r) {
  const int lane = threadIdx.x & 31;
  T s = T(0);
  for (int e = lane; e < r * r; e += 32) {
    const cx<T> v = M[(e / r) * ld + col0 + e % r];
    s += v.re * v.re + v.im * v.im;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return sqrt(s);
}

// Frobenius norms in FP32 without overflow, underflow, divisions or branches:
// a pair (e, sq) stands for 2^e sqrt(sq), the entries scaled by 2^-e staying
// below 2 (e the largest binary exponent seen, clamped to the normal range).
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((min(max(k, -126), 127) + 127) << 23); }
__device__ __forceinline__ void nrm_add(int& e, float& sq, float x) {
  const int ex = min(((__float_as_int(x) >> 23) & 0xff) - 126, 126);  // |x| < 2^ex
  const int en = max(e, ex);
  const float t = fabsf(x) * pow2f(-en);
  sq = fmaf(t, t, sq * pow2f(2 * (e - en)));
  e = en;
}
__device__ __forceinline__ void nrm_merge(int& e, float& sq, int e2, float sq2) {
  const int en = max(e, e2);
  sq = sq * pow2f(2 * (e - en)) + sq2 * pow2f(2 * (e2 - en));
  e = en;
}
__device__ __forceinline__ void warp_nrm(int& e, float& sq) {
  for (int o = 16; o > 0; o >>= 1) {
    const int e2 = __shfl_xor_sync(0xffffffffu, e, o);
    const float q2 = __shfl_xor_sync(0xffffffffu, sq, o);
    nrm_merge(e, sq, e2, q2);
  }
}
constexpr int kNrmE0 = -126;  // the empty pair: (kNrmE0, 0)

// The same in FP32 arithmetic (a certificate needs only a few digits; the
// FP64 pipe of this part is slow), as a scaled sum of squares.
template <typename T>
__device__ inline float warp_frob_lowp(const cx<T>* M, int r) {
  const int lane = threadIdx.x & 31;
  int ex = kNrmE0;
  float sq = 0.f;
  for (int e = lane; e < r * r; e += 32) {
    nrm_add(ex, sq, (float)M[e].re);
    nrm_add(ex, sq, (float)M[e].im);
  }
  warp_nrm(ex, sq);
  return sqrtf(sq) * pow2f(ex);  // infinite beyond the FP32 range
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

// Gauss-Jordan inverse of the r x r matrix W (row-major) without pivoting:
// at pivot p, a_pp <- 1/a_pp, a_pj <- a_pj / a_pp, a_ij <- a_ij - a_ip a_pj /
// a_pp and a_ip <- -a_ip / a_pp (r^3 complex multiply-adds).  W holds 2 r^2
// values: its halves alternate as source and destination, so one barrier per
// pivot suffices; piv[0], piv[1] carry the next pivot's reciprocal (re) and a
// validity flag (im), set by the thread that forms that pivot.  The inverse
// ends in the first half.  Threads [t, t + nt) of the caller; sync() orders
// the steps among them.  Returns 0 when a pivot is not positive.
template <typename T, typename Sync>
__device__ __forceinline__ int gauss_jordan_inplace(cx<T>* W, cx<T>* piv, int r, int t, int nt, Sync sync) {
  const int rr = r * r;
  auto pivot_info = [](T pv) {
    const bool ok = (pv > tiny_pivot<T>()) && isfinite(pv);
    return cx<T>{ok ? rcp_refined(pv) : T(0), ok ? T(1) : T(0)};
  };
  if (t == 0) piv[0] = pivot_info(W[0].re);
  const bool one = rr <= nt;  // each thread owns at most one element: its (i, j) once
  const int ti = t / r, tj = t - ti * r;
  sync();
  for (int p = 0; p < r; ++p) {
    const cx<T>* src = W + (p & 1) * rr;
    cx<T>* dst = W + ((p + 1) & 1) * rr;
    const cx<T> pinfo = piv[p & 1];
    if (pinfo.im == T(0)) return 0;
    const T ip = pinfo.re;
    auto step = [&](int e, int i, int j) {
      cx<T> v;
      if (i == p) v = (j == p) ? cx<T>{ip, T(0)} : src[p * r + j] * ip;
      else if (j == p) v = src[i * r + p] * (-ip);
      else v = src[e] - cmul(src[i * r + p], src[p * r + j] * ip);
      dst[e] = v;
      if (i == p + 1 && j == p + 1) piv[(p + 1) & 1] = pivot_info(v.re);
    };
    if (one) {
      if (t < rr) step(t, ti, tj);
    } else {
      for (int e = t; e < rr; e += nt) step(e, e / r, e % r);
    }
    sync();
  }
  if (r & 1) {
    for (int e = t; e < rr; e += nt) W[e] = W[rr + e];
    sync();
  }
  return 1;
}

// Double-FP32 ("df64") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits on the FP32 pipes (Dekker's and Knuth's
// error-free sum and product; the product's error term from an FMA).  Used
// for the r x r inverses of FP32 engines, where FP64 units are too slow.
struct df {
  float hi, lo;
};
struct alignas(16) dfc {
  df re, im;
};
__device__ __forceinline__ df df_from(double x) {
  const float h = (float)x;
  return df{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df df_norm(float s, float e) {
  const float h = s + e;
  return df{h, e - (h - s)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  return df_norm(s, e);
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);  // not contracted: fmaf below recovers its rounding error
  const float e = fmaf(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  return df_norm(p, e);
}
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return dfc{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return dfc{df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
__device__ __forceinline__ dfc dfc_scale(dfc a, df s) { return dfc{df_mul(a.re, s), df_mul(a.im, s)}; }
// 1/a for a > 0: FP32 reciprocal y0, then one Newton step y0 + y0 (1 - a y0)
// in df64 (the error squares: about 2^-46 relative).
__device__ __forceinline__ df df_rcp(df a) {
  const float y0 = 1.0f / a.hi;
  const df e = df_add(df{1.0f, 0.0f}, df_neg(df_mul(a, df{y0, 0.0f})));
  return df_add(df{y0, 0.0f}, df_mul(df{y0, 0.0f}, e));
}

// s + c += a b with the rounding errors of the product (FMA) and of the sum
// (Knuth's two-sum) collected in c: about twice the working precision.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <typename T>
__device__ __forceinline__ void dot2(T& s, T& c, T a, T b) {
  const T p = mul_rn(a, b);  // not contracted: the FMA below recovers its rounding error
  const T pe = fma(a, b, -p);
  const T t = s + p;
  const T z = t - s;
  c += ((s - (t - z)) + (p - z)) + pe;
  s = t;
}

// gauss_jordan_inplace on an FP64 matrix, with the arithmetic in df64 (the
// matrix is converted, eliminated and converted back; no FP64 instruction in
// the elimination itself).
template <typename Sync>
__device__ __forceinline__ int gauss_jordan_inplace_df(cx<double>* W64, cx<double>* piv, int r, int t, int nt,
                                                       Sync sync) {
  const int rr = r * r;
  dfc* W = reinterpret_cast<dfc*>(W64);
  dfc* pv2 = reinterpret_cast<dfc*>(piv);
  auto pivot_info = [](df pv) {
    const bool ok = (pv.hi > 1e-30f) && isfinite(pv.hi);
    return dfc{ok ? df_rcp(pv) : df{0.f, 0.f}, df{ok ? 1.f : 0.f, 0.f}};
  };
  if (t == 0) pv2[0] = pivot_info(df_from(W64[0].re));
  for (int e = t; e < rr; e += nt) {
    const cx<double> v = W64[e];
    W[e] = dfc{df_from(v.re), df_from(v.im)};
  }
  const bool one = rr <= nt;  // each thread owns at most one element: its (i, j) once
  const int ti = t / r, tj = t - ti * r;
  sync();
  int ok = 1;
  for (int p = 0; p < r; ++p) {
    const dfc* src = W + (p & 1) * rr;
    dfc* dst = W + ((p + 1) & 1) * rr;
    const dfc pinfo = pv2[p & 1];
    if (pinfo.im.hi == 0.f) {
      ok = 0;
      break;
    }
    const df ip = pinfo.re, nip = df_neg(ip);
    auto step = [&](int e, int i, int j) {
      dfc v;
      if (i == p) v = (j == p) ? dfc{ip, df{0.f, 0.f}} : dfc_scale(src[p * r + j], ip);
      else if (j == p) v = dfc_scale(src[i * r + p], nip);
      else v = dfc_sub(src[e], dfc_mul(src[i * r + p], dfc_scale(src[p * r + j], ip)));
      dst[e] = v;
      if (i == p + 1 && j == p + 1) pv2[(p + 1) & 1] = pivot_info(v.re);
    };
    if (one) {
      if (t < rr) step(t, ti, tj);
    } else {
      for (int e = t; e < rr; e += nt) step(e, e / r, e % r);
    }
    sync();
  }
  const dfc* res = W + (r & 1) * rr;
  for (int e = t; e < rr; e += nt) {
    const dfc v = res[e];
    W64[e] = cx<double>{df_to(v.re), df_to(v.im)};
  }
  sync();
  return ok;
}

// Gauss-Jordan inverse of the Hermitian r x r matrix A (r <= RP <= 16) by one
// warp with [A | I] in registers: lane j holds column j of the 2r augmented
// columns, and the pivot column reaches the other lanes by shuffles.  On
// success (return 1) Ainv (row-major r x r) holds A^-1 and an, in the
// Frobenius norms of A and A^-1; 0 when a pivot is not positive.
template <typename T, int RP>
__device__ int warp_gj_inverse(const cx<T>* A, cx<T>* Ainv, int r, T& an, T& in) {
  const int lane = threadIdx.x & 31;
  cx<T> c[RP];
#pragma unroll
  for (int i = 0; i < RP; ++i) {
    cx<T> v = {T(0), T(0)};
    if (i < r) {
      if (lane < r) v = A[i * r + lane];
      else if (lane == r + i) v = cx<T>{T(1), T(0)};
    }
    c[i] = v;
  }
  T cs = T(0);
#pragma unroll
  for (int i = 0; i < RP; ++i) cs += c[i].re * c[i].re + c[i].im * c[i].im;
  an = T(0);
  in = T(0);
  T a = (lane < r) ? cs : T(0);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  an = sqrt(a);
  if (!(a > T(0) && isfinite(a))) return 0;
  // a runtime pivot loop with row p picked by selects: the body (RP rows) is
  // fetched once and stays in the instruction cache for the later pivots (the
  // code runs once per launch and CTA, so an unrolled body runs cold)
#pragma unroll 1
  for (int p = 0; p < r; ++p) {
    cx<T> cpv = c[0];
#pragma unroll
    for (int i = 1; i < RP; ++i)
      if (i == p) cpv = c[i];
    const T pv = __shfl_sync(0xffffffffu, cpv.re, p);
    if (!((pv > tiny_pivot<T>()) && isfinite(pv))) return 0;
    const T ip = rcp_refined(pv);
    const cx<T> rp = cpv * ip;
#pragma unroll
    for (int i = 0; i < RP; ++i) {
      const cx<T> cp = {__shfl_sync(0xffffffffu, c[i].re, p), __shfl_sync(0xffffffffu, c[i].im, p)};
      const cx<T> u = c[i] - cmul(cp, rp);
      c[i] = cx<T>{i == p ? rp.re : u.re, i == p ? rp.im : u.im};
    }
  }
  cs = T(0);
#pragma unroll
  for (int i = 0; i < RP; ++i) cs += c[i].re * c[i].re + c[i].im * c[i].im;
  a = (lane >= r && lane < 2 * r) ? cs : T(0);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  in = sqrt(a);
  if (lane >= r && lane < 2 * r) {
#pragma unroll
    for (int i = 0; i < RP; ++i)
      if (i < r) Ainv[i * r + (lane - r)] = c[i];
  }
  __syncwarp();
  return 1;
}

// Barrier 1 among the first n threads of the block (n a multiple of 32).
__device__ __forceinline__ void bar_first(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }

// Static shared scratch of the register eliminations and of the norm
// reduction of herm_inverse_refined (used one after the other), independent
// of the callers' dynamic carve; within the kStaticSmemReserve headroom.
static __shared__ float g_solve_xch[256];

// Gauss-Jordan inverse without pivoting (the update rules of
// gauss_jordan_inplace) of an r x r matrix, r <= 32, with the matrix in
// registers: lane j holds column j, warp w rows RPL w .. RPL w + RPL - 1
// (ceil(r / RPL) warps), padded with the identity beyond r.  At pivot p the
// warp holding row p scales it by the pivot's reciprocal and passes it on
// through shared memory (two buffers, so one barrier of those warps per pivot
// suffices); each warp takes column p of its rows from lane p by shuffles.
// Every candidate value is formed by every lane and selected, so no branch
// diverges.  A warp runs this serial chain at well under one instruction per
// clock, so two rows per lane (sixteen warps at r = 32) are used where the
// block has the warps.  The other warps only meet the final __syncthreads.
// Exchange area: g_solve_xch.  Returns 1 (block-uniform) unless a pivot is
// not positive.  ld: row pitch of Ainv.  Every thread of the block calls it.
template <int RPL>
static __device__ __noinline__ int gj_regs_cf_t(const cx<float>* A, cx<float>* Ainv, int r, int ld) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float* xch = g_solve_xch;
  cx<float>* trow = reinterpret_cast<cx<float>*>(xch);  // [2][32] scaled pivot rows
  float* prc = xch + 128;                                // [2] pivot reciprocals
  int* okf = reinterpret_cast<int*>(xch + 130);
  const int nwu = (r + RPL - 1) / RPL;
  if (w < nwu) {
    cx<float> a[RPL];
#pragma unroll
    for (int m = 0; m < RPL; ++m) {
      const int i = RPL * w + m;
      a[m] = (i < r && lane < r) ? A[i * r + lane] : cx<float>{i == lane ? 1.f : 0.f, 0.f};
    }
    int ok = 1;
    for (int p = 0; p < r; ++p) {
      const int b = p & 1;
      if (w == p / RPL) {
        cx<float> rp = a[0];
#pragma unroll
        for (int m = 1; m < RPL; ++m)
          if (m == p % RPL) rp = a[m];
        const float pv = __shfl_sync(0xffffffffu, rp.re, p);
        const bool good = pv > tiny_pivot<float>() && isfinite(pv);
        const float ip = good ? __frcp_rn(pv) : 0.f;
        trow[b * 32 + lane] = rp * ip;
        if (lane == 0) prc[b] = ip;
      }
      bar_first(32 * nwu);
      const float ip = prc[b];
      if (ip == 0.f) {
        ok = 0;
        break;
      }
      const cx<float> t = trow[b * 32 + lane];
      const bool lp = lane == p;
#pragma unroll
      for (int m = 0; m < RPL; ++m) {
        const cx<float> c = {__shfl_sync(0xffffffffu, a[m].re, p), __shfl_sync(0xffffffffu, a[m].im, p)};
        const cx<float> u = a[m] - cmul(c, t);
        const bool rp = RPL * w + m == p;
        const float vr = lp ? (rp ? ip : -c.re * ip) : (rp ? t.re : u.re);
        const float vi = lp ? (rp ? 0.f : -c.im * ip) : (rp ? t.im : u.im);
        a[m] = cx<float>{vr, vi};
      }
    }
#pragma unroll
    for (int m = 0; m < RPL; ++m) {
      const int i = RPL * w + m;
      if (i < r && lane < r) Ainv[i * ld + lane] = a[m];
    }
    if (tid == 0) *okf = ok;
  }
  __syncthreads();
  return *okf;
}
static __device__ __forceinline__ int gj_regs_cf(const cx<float>* A, cx<float>* Ainv, int r, int ld) {
  return (int)blockDim.x >= 32 * ((r + 1) / 2) ? gj_regs_cf_t<2>(A, Ainv, r, ld) : gj_regs_cf_t<8>(A, Ainv, r, ld);
}

// The same for a real r x r matrix in df64 arithmetic (FP64 in and out, pitch
// r); also leaves ||A||_F and ||A^-1||_F (FP32, a certificate needs a few
// digits; infinite beyond the FP32 range) in g_solve_xch[200], [201].
template <int RPL>
static __device__ __noinline__ int gj_regs_df_t(const double* A, double* Ainv, int r) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float* xch = g_solve_xch;
  df* trow = reinterpret_cast<df*>(xch);  // [2][32]
  df* prc = trow + 64;                    // [2]
  int* okf = reinterpret_cast<int*>(xch + 132);
  int* xe = reinterpret_cast<int*>(xch + 136);  // [16][4] per-warp norm pairs
  const int nwu = (r + RPL - 1) / RPL;
  if (w < nwu) {
    df a[RPL];
    int ae = kNrmE0;
    float aq = 0.f;
#pragma unroll
    for (int m = 0; m < RPL; ++m) {
      const int i = RPL * w + m;
      a[m] = (i < r && lane < r) ? df_from(A[i * r + lane]) : df{i == lane ? 1.f : 0.f, 0.f};
      if (i < r && lane < r) nrm_add(ae, aq, a[m].hi);
    }
    int ok = 1;
    for (int p = 0; p < r; ++p) {
      const int b = p & 1;
      if (w == p / RPL) {
        df rp = a[0];
#pragma unroll
        for (int m = 1; m < RPL; ++m)
          if (m == p % RPL) rp = a[m];
        const df pv = {__shfl_sync(0xffffffffu, rp.hi, p), __shfl_sync(0xffffffffu, rp.lo, p)};
        const bool good = pv.hi > 1e-30f && isfinite(pv.hi);
        const df ip = good ? df_rcp(pv) : df{0.f, 0.f};
        trow[b * 32 + lane] = df_mul(rp, ip);
        if (lane == 0) prc[b] = ip;
      }
      bar_first(32 * nwu);
      const df ip = prc[b];
      if (!(ip.hi > 0.f)) {
        ok = 0;
        break;
      }
      const df t = trow[b * 32 + lane];
      const bool lp = lane == p;
#pragma unroll
      for (int m = 0; m < RPL; ++m) {
        const df c = {__shfl_sync(0xffffffffu, a[m].hi, p), __shfl_sync(0xffffffffu, a[m].lo, p)};
        const df u = df_add(a[m], df_neg(df_mul(c, t)));
        const df cq = df_neg(df_mul(c, ip));
        const bool rp = RPL * w + m == p;
        a[m] = df{lp ? (rp ? ip.hi : cq.hi) : (rp ? t.hi : u.hi), lp ? (rp ? ip.lo : cq.lo) : (rp ? t.lo : u.lo)};
      }
    }
    int ie = kNrmE0;
    float iq = 0.f;
#pragma unroll
    for (int m = 0; m < RPL; ++m) {
      const int i = RPL * w + m;
      if (i < r && lane < r) {
        Ainv[i * r + lane] = df_to(a[m]);
        nrm_add(ie, iq, a[m].hi);
      }
    }
    warp_nrm(ae, aq);
    warp_nrm(ie, iq);
    if (lane == 0) {
      xe[4 * w] = ae;
      xch[137 + 4 * w] = aq;
      xe[4 * w + 2] = ie;
      xch[139 + 4 * w] = iq;
    }
    bar_first(32 * nwu);
    if (w == 0) {  // lane q merges warp q's pairs
      int e1 = kNrmE0, e2 = kNrmE0;
      float q1 = 0.f, q2 = 0.f;
      if (lane < nwu) {
        e1 = xe[4 * lane];
        q1 = xch[137 + 4 * lane];
        e2 = xe[4 * lane + 2];
        q2 = xch[139 + 4 * lane];
      }
      warp_nrm(e1, q1);
      warp_nrm(e2, q2);
      if (lane == 0) {
        xch[200] = sqrtf(q1) * pow2f(e1);
        xch[201] = sqrtf(q2) * pow2f(e2);
        *okf = ok;
      }
    }
  }
  __syncthreads();
  return *okf;
}
static __device__ __forceinline__ int gj_regs_df(const double* A, double* Ainv, int r) {
  return (int)blockDim.x >= 32 * ((r + 1) / 2) ? gj_regs_df_t<2>(A, Ainv, r) : gj_regs_df_t<8>(A, Ainv, r);
}

// Inverse of a Hermitian positive definite r x r matrix A = Ah + Al (FP32 head
// and tail, row-major, shared memory) to FP64-class accuracy on the FP32
// pipes, for well-conditioned A: X0 = FP32 Gauss-Jordan inverse of Ah, then
// one refinement step X1 = X0 + X0 R with the residual R = I - A X0 formed
// from error-free products and compensated sums (Ogita-Rump-Oishi Dot2), so
// that R is exact to a few units of 2^-48 |A| |X0|.  The error of X1 is about
// ||R||^2 relative plus the FP32 rounding of the correction (2^-24 ||R||):
// the step is accepted when ||R||_F <= 2^-14, which keeps it below 2^-27,
// under the FP32 rounding every caller applies to the result, and when the
// certificate ||A||_F ||A^-1||_F < 1/(2 rtol) holds (||A^-1||_F bounded by
// ||X0||_F / (1 - ||R||_F)).  Returns 1 (block-uniform) with the Hermitian part
// of X1 in Xo; 0 when a pivot is not positive or a test fails, and the caller
// takes the df64 elimination or the eigendecomposition.  LO: Al is present
// (else A = Ah exactly).  work: 3 r^2 values, red: 4 floats, shared memory;
// every thread of the block calls it.
template <bool LO>
__device__ __noinline__ int herm_inverse_refined(const cx<float>* Ah, const cx<float>* Al, cx<float>* Xo,
                                                 cx<float>* work, float* red, int r, double rtol) {
  const int tid = threadIdx.x, nt = blockDim.x, rr = r * r;
  cx<float>* X0 = work;          // r^2
  cx<float>* C = work + rr;      // r^2: X0 R
  cx<float>* R = work + 2 * rr;  // r^2
  if (!gj_regs_cf(Ah, X0, r, r)) return 0;
  // R = I - (Ah + Al) X0: Ah X0 by Dot2 (TwoProduct by FMA, TwoSum), Al X0 in
  // FP32; the squared norms of R, X0 and Ah on the way
  float nr = 0.f, xq = 0.f, aq = 0.f;
  int xe = kNrmE0, ae = kNrmE0;
  for (int e = tid; e < rr; e += nt) {
    const int i = e / r, j = e - i * r;
    const cx<float>* ah = Ah + i * r;
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f, tr = 0.f, ti = 0.f;
    for (int l = 0; l < r; ++l) {
      const cx<float> a = ah[l], b = X0[l * r + j];
      dot2(sr, cr, a.re, b.re);
      dot2(sr, cr, -a.im, b.im);
      dot2(si, ci, a.re, b.im);
      dot2(si, ci, a.im, b.re);
      if constexpr (LO) {
        const cx<float> t = Al[i * r + l];
        tr = fmaf(t.re, b.re, fmaf(-t.im, b.im, tr));
        ti = fmaf(t.re, b.im, fmaf(t.im, b.re, ti));
      }
    }
    // the diagonal: 1 - s is exact (s within a factor 2 of 1 once ||R|| is small)
    const cx<float> v = {((i == j ? 1.f : 0.f) - sr) - (cr + tr), -si - (ci + ti)};
    R[e] = v;
    const cx<float> x = X0[e], a = Ah[e];
    nr = fmaf(v.re, v.re, fmaf(v.im, v.im, nr));  // R is small: a plain sum
    nrm_add(xe, xq, x.re);
    nrm_add(xe, xq, x.im);
    nrm_add(ae, aq, a.re);
    nrm_add(ae, aq, a.im);
  }
  {
    float* part = g_solve_xch;  // [32][5]
    int* parti = reinterpret_cast<int*>(g_solve_xch);
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_xor_sync(0xffffffffu, nr, o);
    warp_nrm(xe, xq);
    warp_nrm(ae, aq);
    if ((tid & 31) == 0) {
      const int w = tid >> 5;
      part[5 * w] = nr;
      parti[5 * w + 1] = xe;
      part[5 * w + 2] = xq;
      parti[5 * w + 3] = ae;
      part[5 * w + 4] = aq;
    }
    __syncthreads();
    if (tid < 32) {  // lane q merges warp q's partials
      float sr = 0.f, q1 = 0.f, q2 = 0.f;
      int e1 = kNrmE0, e2 = kNrmE0;
      if (tid < ((nt + 31) >> 5)) {
        sr = part[5 * tid];
        e1 = parti[5 * tid + 1];
        q1 = part[5 * tid + 2];
        e2 = parti[5 * tid + 3];
        q2 = part[5 * tid + 4];
      }
      for (int o = 16; o > 0; o >>= 1) sr += __shfl_xor_sync(0xffffffffu, sr, o);
      warp_nrm(e1, q1);
      warp_nrm(e2, q2);
      if (tid == 0) {
        const float rn = sqrtf(sr);
        // log2 of ||X0||_F ||A||_F against log2 of (1 - ||R||_F) / (2 rtol)
        const float lhs = (float)(e1 + e2) + 0.5f * __log2f(q1 * q2);
        const float rhs = __log2f((1.f - rn) * 0.5f) - __log2f((float)rtol);
        red[0] = rn;
        red[3] = (rn <= 0x1p-14f && q2 > 0.f && isfinite(lhs) && lhs < rhs) ? 1.f : 0.f;
      }
    }
    __syncthreads();
  }
  if (red[3] == 0.f) return 0;
  for (int e = tid; e < rr; e += nt) {
    const int i = e / r, j = e - i * r;
    cx<float> c = {0.f, 0.f};
    for (int l = 0; l < r; ++l) cfma(c, X0[i * r + l], R[l * r + j]);
    C[e] = c;
  }
  __syncthreads();
  // Hermitian part of X1 = X0 + C; thread t takes (i, j) = (L, (L + c) mod r),
  // L = t mod r, c = t / r, so that both the (i, j) and the (j, i) reads of a
  // warp fall in distinct banks
  for (int t = tid; t < rr; t += nt) {
    const int c0 = t / r, i = t - c0 * r, j = (i + c0) % r;
    const cx<float> a = X0[i * r + j], b = X0[j * r + i], c = C[i * r + j], g = C[j * r + i];
    Xo[i * r + j] = cx<float>{0.5f * ((a.re + b.re) + (c.re + g.re)), 0.5f * ((a.im - b.im) + (c.im - g.im))};
  }
  __syncthreads();
  return 1;
}

// DF: the block inverse (r > 16) of an FP64 matrix runs in df64 arithmetic,
// after herm_inverse_refined on the FP32 split of A.
template <typename T, int RP, bool DF = false>
__device__ __noinline__ int block_pinv_herm(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, cx<T>* piv, T* sred,
                                      int r, T rtol, bool force_eig = false, bool refine = true) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int ok;
  if (force_eig) {
    // the eigendecomposition is wanted for lambda_max (scaled steps): sred[2]
    jacobi_fallback<T, DF>(A, Ap, P, V, W, piv, r, rtol, sred + 2);
    __syncthreads();
    return 0;
  }
  if constexpr (RP <= 16 && !DF) {
    // W receives A^-1 (row-major r x r)
    if (tid < 32) {
      T an, in;
      const int g = warp_gj_inverse<T, RP>(A, W, r, an, in);
      if (tid == 0) sred[1] = (g && isfinite(in) && an * in < T(0.5) / rtol) ? T(1) : T(0);
    }
    __syncthreads();
    ok = sred[1] != T(0);
    if (ok) {
      for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e - i * r;
        // symmetrise: A^-1 of a Hermitian matrix is Hermitian
        const cx<T> a = W[i * r + j];
        const cx<T> b = W[j * r + i];
        Ap[e] = cx<T>{T(0.5) * (a.re + b.re), T(0.5) * (a.im - b.im)};
        P[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
      }
      __syncthreads();
      return 1;
    }
  } else {
    if constexpr (DF && sizeof(T) == 8) {
      if (refine) {
        // A = Ah + Al in V (2 r^2 complex floats); the work of the refined inverse
        // and its result in W (4 r^2 complex floats).  refine = false: the caller
        // has tried it already.
        const int rr = r * r;
        cx<float>* ahf = reinterpret_cast<cx<float>*>(V);
        cx<float>* alf = ahf + rr;
        cx<float>* wf = reinterpret_cast<cx<float>*>(W);
        cx<float>* xo = wf + 3 * rr;
        for (int e = tid; e < rr; e += nt) {
          const cx<T> a = A[e];
          const cx<float> h = {(float)a.re, (float)a.im};
          ahf[e] = h;
          alf[e] = cx<float>{(float)(a.re - (T)h.re), (float)(a.im - (T)h.im)};
        }
        __syncthreads();
        if (herm_inverse_refined<true>(ahf, alf, xo, wf, reinterpret_cast<float*>(sred), r, (double)rtol)) {
          for (int e = tid; e < rr; e += nt) {
            const int i = e / r, j = e - i * r;
            Ap[e] = cx<T>{(T)xo[e].re, (T)xo[e].im};
            P[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
          }
          __syncthreads();
          return 1;
        }
        __syncthreads();
      }
    }
    for (int e = tid; e < r * r; e += nt) W[e] = A[e];
    if (tid < 32) {
      const T an = DF ? (T)warp_frob_lowp(A, r) : warp_frob(A, r, 0, r);
      if (tid == 0) sred[0] = an;
    }
    __syncthreads();
    const T anorm = sred[0];
    ok = (anorm > T(0)) && isfinite(anorm);
    if (ok) {
      if constexpr (DF && sizeof(T) == 8) ok = gauss_jordan_inplace_df(W, piv, r, tid, nt, []() { __syncthreads(); });
      else ok = gauss_jordan_inplace<T>(W, piv, r, tid, nt, []() { __syncthreads(); });
    }
    if (tid < 32) {
      const T in = ok ? (DF ? (T)warp_frob_lowp(W, r) : warp_frob(W, r, 0, r)) : T(0);
      if (tid == 0) sred[1] = (ok && isfinite(in) && anorm * in < T(0.5) / rtol) ? T(1) : T(0);
    }
    __syncthreads();
    ok = sred[1] != T(0);
    if (ok) {
      for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e - i * r;
        const cx<T> a = W[i * r + j];
        const cx<T> b = W[j * r + i];
        Ap[e] = cx<T>{T(0.5) * (a.re + b.re), T(0.5) * (a.im - b.im)};
        P[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
      }
      __syncthreads();
      return 1;
    }
  }
  __syncthreads();
  jacobi_fallback<T, DF>(A, Ap, P, V, W, piv, r, rtol, sred + 2);
  __syncthreads();
  return 0;
}

// Parallel cyclic complex Jacobi eigendecomposition A = V diag(lambda) V^* by
// the whole block, then A^+ and P = A A^+ with the cutoff rule.  Each round
// rotates the disjoint pairs of a round-robin schedule (m - 1 rounds of m/2
// pairs, m = r rounded up to even, index r a dummy when r is odd): the pair
// threads form the rotations, then all threads apply them to the columns
// (W J, V J) and to the rows (J^H W J).  A rotation is skipped when
// |a_pq| <= 4 u max(|a_pp|, |a_qq|) (u the unit roundoff), and the sweeps stop
// after one without rotations.
template <typename T>
__device__ __noinline__ void block_jacobi_pinv(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, cx<T>* piv, int r,
                                         T rtol, T* lmax_out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const T u_round = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-8f);
  const int m = (r + 1) & ~1, np = m / 2;
  // rotation of pair k: piv[2k] = (cs, sn), piv[2k + 1] = unit phase u; rows p, q in rpq
  int* rpq = reinterpret_cast<int*>(piv + 2 * np);
  for (int e = tid; e < r * r; e += nt) {
    W[e] = A[e];
    const int i = e / r, j = e - i * r;
    V[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    bool any = false;
    for (int round = 0; round < m - 1; ++round) {
      int rot = 0;
      if (tid < np) {
        int a, b;
        if (tid == 0) {
          a = round;
          b = m - 1;
        } else {
          a = (round + tid) % (m - 1);
          b = (round - tid + m - 1) % (m - 1);
        }
        const int p = min(a, b), q = max(a, b);
        T cs = T(1), sn = T(0);
        cx<T> uu = {T(1), T(0)};
        if (q < r) {
          const cx<T> c = W[p * r + q];
          const T n2 = c.re * c.re + c.im * c.im;
          const T app = W[p * r + p].re, aqq = W[q * r + q].re;
          // below 4u max(|a_pp|, |a_qq|) the entry is at the rounding level of the
          // rotations themselves (its effect on any eigenvalue is below u^2 lambda_max)
          const T thr = T(4) * u_round * fmax(fabs(app), fabs(aqq));
          if (n2 > tiny_pivot<T>() && n2 > thr * thr) {
            const T iac = rsqrt(n2);
            uu = cx<T>{c.re * iac, c.im * iac};
            const T tau = (aqq - app) * T(0.5) * iac;
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            cs = rsqrt(T(1) + t * t);
            sn = t * cs;
            rot = 1;
          }
        }
        piv[2 * tid] = cx<T>{cs, sn};
        piv[2 * tid + 1] = uu;
        rpq[2 * tid] = p;
        rpq[2 * tid + 1] = (q < r) ? q : -1;
      }
      if (!__syncthreads_or(rot)) continue;
      any = true;
      // ---- columns: W J and V J (item = row i, pair k) ----
      for (int e = tid; e < r * np; e += nt) {
        const int k = e / r, i = e - k * r;
        const int p = rpq[2 * k], q = rpq[2 * k + 1];
        if (q < 0) continue;
        const T cs = piv[2 * k].re, sn = piv[2 * k].im;
        const cx<T> uu = piv[2 * k + 1];
        // J = [[cs, sn u], [-sn conj(u), cs]] on columns p, q
        const cx<T> aip = W[i * r + p], aiq = W[i * r + q];
        W[i * r + p] = aip * cs - cmulc(aiq, uu) * sn;
        W[i * r + q] = cmul(aip, uu) * sn + aiq * cs;
        const cx<T> vip = V[i * r + p], viq = V[i * r + q];
        V[i * r + p] = vip * cs - cmulc(viq, uu) * sn;
        V[i * r + q] = cmul(vip, uu) * sn + viq * cs;
      }
      __syncthreads();
      // ---- rows: J^H (W J) (item = pair k, column j) ----
      for (int e = tid; e < r * np; e += nt) {
        const int k = e / r, j = e - k * r;
        const int p = rpq[2 * k], q = rpq[2 * k + 1];
        if (q < 0) continue;
        const T cs = piv[2 * k].re, sn = piv[2 * k].im;
        const cx<T> uu = piv[2 * k + 1];
        const cx<T> apj = W[p * r + j], aqj = W[q * r + j];
        W[p * r + j] = apj * cs - cmul(aqj, uu) * sn;
        W[q * r + j] = cmulc(apj, uu) * sn + aqj * cs;
      }
      __syncthreads();
    }
    if (!any) break;
  }
  // eigenvalues on the diagonal; cutoff relative to lambda_max
  T lmax = T(0);
  for (int i = 0; i < r; ++i) lmax = fmax(lmax, W[i * r + i].re);
  const T cut = rtol * lmax;
  if (tid == 0) *lmax_out = lmax;
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e - i * r;
    cx<T> sa = {T(0), T(0)}, sp = {T(0), T(0)};
    for (int mm = 0; mm < r; ++mm) {
      const T lam = W[mm * r + mm].re;
      if (lmax > T(0) && lam > cut) {
        const cx<T> vv = cmulc(V[i * r + mm], V[j * r + mm]);  // V_im conj(V_jm)
        sa = sa + vv * (T(1) / lam);
        sp = sp + vv;
      }
    }
    Ap[e] = sa;
    P[e] = sp;
  }
  __syncthreads();
}

// The same eigendecomposition by one warp, for small r, where the block-wide
// barriers of block_jacobi_pinv would cost more than the rotations: then A^+
// and P = A A^+ with the cutoff rule.
template <typename T>
__device__ __noinline__ void warp_jacobi_pinv(const cx<T>* A, cx<T>* Ap, cx<T>* P, cx<T>* V, cx<T>* W, cx<T>* piv, int r,
                                        T rtol, T* lmax_out) {
  const int lane = threadIdx.x & 31;
  const T u_round = sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-8f);
  const int m = (r + 1) & ~1, np = m / 2;
  // rotation of pair k: piv[2k] = (cs, sn), piv[2k + 1] = unit phase u; rows p, q in rpq
  int* rpq = reinterpret_cast<int*>(piv + 2 * np);  // 2 ints per pair (fits in the third r values)
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    W[e] = A[e];
    const int i = e / r, j = e - i * r;
    V[e] = cx<T>{(i == j) ? T(1) : T(0), T(0)};
  }
  __syncwarp();
  for (int sweep = 0; sweep < 30; ++sweep) {
    bool any = false;
    for (int round = 0; round < m - 1; ++round) {
      // ---- rotations of this round (lane k < np) ----
      bool rot = false;
      if (lane < np) {
        int a, b;
        if (lane == 0) {
          a = round;
          b = m - 1;
        } else {
          a = (round + lane) % (m - 1);
          b = (round - lane + m - 1) % (m - 1);
        }
        const int p = min(a, b), q = max(a, b);
        T cs = T(1), sn = T(0);
        cx<T> uu = {T(1), T(0)};
        if (q < r) {
          const cx<T> c = W[p * r + q];
          const T n2 = c.re * c.re + c.im * c.im;
          const T app = W[p * r + p].re, aqq = W[q * r + q].re;
          // below 4u max(|a_pp|, |a_qq|) the entry is at the rounding level of the
          // rotations themselves (its effect on any eigenvalue is below u^2 lambda_max)
          const T thr = T(4) * u_round * fmax(fabs(app), fabs(aqq));
          if (n2 > tiny_pivot<T>() && n2 > thr * thr) {
            const T iac = rsqrt(n2);
            uu = cx<T>{c.re * iac, c.im * iac};
            const T tau = (aqq - app) * T(0.5) * iac;
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            cs = rsqrt(T(1) + t * t);
            sn = t * cs;
            rot = true;
          }
        }
        piv[2 * lane] = cx<T>{cs, sn};
        piv[2 * lane + 1] = uu;
        rpq[2 * lane] = p;
        rpq[2 * lane + 1] = (q < r) ? q : -1;
      }
      rot = __any_sync(0xffffffffu, rot);
      __syncwarp();
      if (!rot) continue;
      any = true;
      // ---- columns: W J and V J (item = row i, pair k) ----
      for (int e = lane; e < r * np; e += 32) {
        const int k = e / r, i = e - k * r;
        const int p = rpq[2 * k], q = rpq[2 * k + 1];
        if (q < 0) continue;
        const T cs = piv[2 * k].re, sn = piv[2 * k].im;
        const cx<T> uu = piv[2 * k + 1];
        // J = [[cs, sn u], [-sn conj(u), cs]] on columns p, q
        const cx<T> aip = W[i * r + p], aiq = W[i * r + q];
        W[i * r + p] = aip * cs - cmulc(aiq, uu) * sn;
        W[i * r + q] = cmul(aip, uu) * sn + aiq * cs;
        const cx<T> vip = V[i * r + p], viq = V[i * r + q];
        V[i * r + p] = vip * cs - cmulc(viq, uu) * sn;
        V[i * r + q] = cmul(vip, uu) * sn + viq * cs;
      }
      __syncwarp();
      // ---- rows: J^H (W J) (item = pair k, column j) ----
      for (int e = lane; e < r * np; e += 32) {
        const int k = e / r, j = e - k * r;
        const int p = rpq[2 * k], q = rpq[2 * k + 1];
        if (q < 0) continue;
        const T cs = piv[2 * k].re, sn = piv[2 * k].im;
        const cx<T> uu = piv[2 * k + 1];
        const cx<T> apj = W[p * r + j], aqj = W[q * r + j];
        W[p * r + j] = apj * cs - cmul(aqj, uu) * sn;
        W[q * r + j] = cmulc(apj, uu) * sn + aqj * cs;
      }
      __syncwarp();
    }
    if (!any) break;
  }
  // eigenvalues on the diagonal; cutoff relative to lambda_max
  T lmax = T(0);
  for (int i = 0; i < r; ++i) lmax = fmax(lmax, W[i * r + i].re);
  const T cut = rtol * lmax;
  if (lane == 0) *lmax_out = lmax;
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int i = e / r, j = e - i * r;
    cx<T> sa = {T(0), T(0)}, sp = {T(0), T(0)};
    for (int mm = 0; mm < r; ++mm) {
      const T lam = W[mm * r + mm].re;
      if (lmax > T(0) && lam > cut) {
        const cx<T> vv = cmulc(V[i * r + mm], V[j * r + mm]);  // V_im conj(V_jm)
        sa = sa + vv * (T(1) / lam);
        sp = sp + vv;
      }
    }
    Ap[e] = sa;
    P[e] = sp;
  }
  __syncwarp();
}

// The eigendecomposition fallback of block_pinv_herm.  For the FP64-storage
// solves of an FP32 engine (DF) it runs in FP32 on the FP32 pipes (the FP64
// pipe of this part is 1/64 of it), with the cutoff raised to at least
// r 2^-23 lambda_max: the Gram was accumulated in FP32 and cannot resolve
// smaller eigenvalues.
template <typename TS, bool DF>
__device__ __noinline__ void jacobi_fallback(const cx<TS>* A, cx<TS>* Ap, cx<TS>* P, cx<TS>* V, cx<TS>* W, cx<TS>* piv,
                                       int r, TS rtol, TS* lmax_out) {
  const bool small = r <= 16;  // one warp; the other threads wait at the caller's barrier
  if constexpr (DF && sizeof(TS) == 8) {
    const int tid = threadIdx.x, nt = blockDim.x, rr = r * r;
    cx<float>* Af = reinterpret_cast<cx<float>*>(W);  // W holds 4 r^2 float pairs
    cx<float>* Wf = Af + rr;
    cx<float>* Vf = Wf + rr;
    cx<float>* Pf = Vf + rr;
    cx<float>* Apf = reinterpret_cast<cx<float>*>(V);  // V holds 2 r^2 float pairs
    float* lmf = reinterpret_cast<float*>(Apf + rr);
    cx<float>* pivf = reinterpret_cast<cx<float>*>(piv);
    for (int e = tid; e < rr; e += nt) Af[e] = cx<float>{(float)A[e].re, (float)A[e].im};
    __syncthreads();
    const float rt = fmaxf((float)rtol, (float)r * 1.1920929e-7f);
    if (small) {
      if (tid < 32) warp_jacobi_pinv<float>(Af, Apf, Pf, Vf, Wf, pivf, r, rt, lmf);
      __syncthreads();
    } else {
      block_jacobi_pinv<float>(Af, Apf, Pf, Vf, Wf, pivf, r, rt, lmf);
    }
    for (int e = tid; e < rr; e += nt) {
      Ap[e] = cx<TS>{(TS)Apf[e].re, (TS)Apf[e].im};
      P[e] = cx<TS>{(TS)Pf[e].re, (TS)Pf[e].im};
    }
    if (tid == 0) *lmax_out = (TS)*lmf;
    __syncthreads();
  } else if (small) {
    if (threadIdx.x < 32) warp_jacobi_pinv<TS>(A, Ap, P, V, W, piv, r, rtol, lmax_out);
    __syncthreads();
  } else {
    block_jacobi_pinv<TS>(A, Ap, P, V, W, piv, r, rtol, lmax_out);
  }
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
// Eq. (hkXYDer) that involves the residual.  Grid (S, ceil(n1/32)); a warp
// takes one or two rows at a time with coalesced loads along the rows, four
// 32-column loads per row in flight, Y~_k staged in shared memory.  Reads R~
// once.
// ---------------------------------------------------------------------------
template <typename T, int RP>
__global__ void __launch_bounds__(kSliceThreads) k_qcon(Dev<T> d, cx<T>* __restrict__ Qout) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* Ys = reinterpret_cast<cx<T>*>(smem);  // [r][n2]
  const cx<T>* Y = d.Yt + (size_t)k * r * n2;
  for (int e = tid; e < r * n2; e += blockDim.x) Ys[e] = Y[e];
  __syncthreads();
  constexpr int HALF = (RP > 16) ? 16 : RP;  // complex values per reduction pass
  constexpr int RR = (RP <= 8) ? 2 : 1;       // rows per pass of a warp
  constexpr int U = 4;                        // 32-column loads in flight per row
  for (int ii = wid * RR; ii < 32; ii += nw * RR) {
    const cx<T>* rowp[RR];
    bool live[RR];
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      const int i = blockIdx.y * 32 + ii + q;
      live[q] = i < n1;
      rowp[q] = d.Rt + ((size_t)(live[q] ? i : 0) * S + k) * n2;
    }
    if (!live[0]) break;
    cx<T> acc[RR][RP];
#pragma unroll
    for (int q = 0; q < RR; ++q)
#pragma unroll
      for (int s = 0; s < RP; ++s) acc[q][s] = cx<T>{T(0), T(0)};
    for (int j0 = 0; j0 < n2; j0 += 32 * U) {
      cx<T> v[RR][U];
#pragma unroll
      for (int q = 0; q < RR; ++q)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j = j0 + 32 * u + lane;
          v[q][u] = (live[q] && j < n2) ? ldg_cx(rowp[q] + j) : cx<T>{T(0), T(0)};
        }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = j0 + 32 * u + lane;
        if (j < n2) {
#pragma unroll
          for (int s = 0; s < RP; ++s)
            if (s < r) {
              const cx<T> y = Ys[(size_t)s * n2 + j];
#pragma unroll
              for (int q = 0; q < RR; ++q) cfmac(acc[q][s], v[q][u], y);
            }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RR; ++q) {
      if (!live[q]) continue;
      const int i = blockIdx.y * 32 + ii + q;
#pragma unroll
      for (int h = 0; h < RP; h += HALF) {
        T f[2 * HALF];
#pragma unroll
        for (int s = 0; s < HALF; ++s) {
          f[2 * s] = acc[q][h + s].re;
          f[2 * s + 1] = acc[q][h + s].im;
        }
        const T tot = warp_reduce_scatter<T, 2 * HALF>(f);
        const int idx = lane >> (5 - Log2<2 * HALF>::value);
        const int s = h + idx / 2;
        const bool first = (lane & ((32 >> Log2<2 * HALF>::value) - 1)) == 0;
        if (first && s < r) reinterpret_cast<T*>(Qout + ((size_t)k * r + s) * n1 + i)[idx & 1] = tot;
      }
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
// Block-wide maximum of a non-negative value, folded into *dst (stopping test).
__device__ __forceinline__ void block_max_to(double v, unsigned long long* dst) {
  __shared__ double smax[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) smax[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, smax[w]);
    atomic_max_nonneg(dst, m);
  }
}

struct XLayout {
  size_t mats, ht, gs, xs, qs, ts, total;
};

// Rows of X~' and X~ staged per step of the X-step Grams; rows are padded to
// kGramLd complex values (odd, so the threads of a warp that read different
// columns hit different banks).
constexpr int kGramRows = 32;
constexpr int kGramLd = kGramRows + 1;

// TS: the type of the r x r solves (the pseudo-inverses); T: everything else.
template <typename T, typename TS = T>
__host__ __device__ inline XLayout xstep_layout(int n1, int n2, int r, bool arrays_in_smem) {
  XLayout L{};
  const size_t rr = (size_t)r * r;
  size_t off = 0;
  L.mats = off;  // A, A^+, P, V, work (2), G, Dg, pivots, reductions (complex doubles:
                 // the FP64 real-slice solve of an FP32 engine uses the same region)
  off = align_up(off + (rr * 8 + 3 * (size_t)r + 2) * sizeof(cx<double>), 16);
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
  // Gram staging rows, used only when the arrays are not resident
  if (arrays_in_smem) {
    L.gs = L.qs;
  } else {
    L.gs = off;
    off = align_up(off + sizeof(cx<T>) * 2 * (size_t)r * kGramLd, 16);
  }
  L.total = off;
  return L;
}

// col <- H_rho1^{-1} col for H_rho1 = I + rho1 H^T H (tridiagonal, Eq. (KKTcondition)),
// by one warp.  The LU sweeps are the first-order recurrences
//   forward   y_i = a_i y_{i-1} + hinv_i b_i,   backward  x_i = a_i x_{i+1} + y_i,
// a_i = rho1 hinv_i (hinv: inverse LU pivots), each evaluated as a parallel
// prefix scan of affine maps over 32 segments of the column: every lane
// composes its segment, a 5-step shuffle scan gives the value entering it,
// and the lane then runs its segment.
template <typename T>
__device__ void warp_tridiag_solve(cx<T>* col, int n1, const T* __restrict__ hinv, const T* __restrict__ ha) {
  const int lane = threadIdx.x & 31;
  const int seg = (n1 + 31) >> 5;
  const int i0 = min(lane * seg, n1), i1 = min(i0 + seg, n1);
  // ---- forward ----
  T A = T(1);
  cx<T> B = {T(0), T(0)};
  for (int i = i0; i < i1; ++i) {
    const T a = ha[i], b = hinv[i];
    const cx<T> v = col[i];
    B = cx<T>{fma(a, B.re, v.re * b), fma(a, B.im, v.im * b)};
    A *= a;
  }
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const T Ap = __shfl_up_sync(0xffffffffu, A, dd);
    const T Br = __shfl_up_sync(0xffffffffu, B.re, dd), Bi = __shfl_up_sync(0xffffffffu, B.im, dd);
    if (lane >= dd) {
      B = cx<T>{fma(A, Br, B.re), fma(A, Bi, B.im)};
      A *= Ap;
    }
  }
  cx<T> y = {__shfl_up_sync(0xffffffffu, B.re, 1), __shfl_up_sync(0xffffffffu, B.im, 1)};
  if (lane == 0) y = cx<T>{T(0), T(0)};
  for (int i = i0; i < i1; ++i) {
    const T a = ha[i], b = hinv[i];
    const cx<T> v = col[i];
    y = cx<T>{fma(a, y.re, v.re * b), fma(a, y.im, v.im * b)};
    col[i] = y;
  }
  __syncwarp();
  // ---- backward (x_{n1} = 0) ----
  A = T(1);
  B = cx<T>{T(0), T(0)};
  for (int i = i1 - 1; i >= i0; --i) {
    const T a = ha[i];
    const cx<T> v = col[i];
    B = cx<T>{fma(a, B.re, v.re), fma(a, B.im, v.im)};
    A *= a;
  }
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const T Ap = __shfl_down_sync(0xffffffffu, A, dd);
    const T Br = __shfl_down_sync(0xffffffffu, B.re, dd), Bi = __shfl_down_sync(0xffffffffu, B.im, dd);
    if (lane + dd < 32) {
      B = cx<T>{fma(A, Br, B.re), fma(A, Bi, B.im)};
      A *= Ap;
    }
  }
  cx<T> x = {__shfl_down_sync(0xffffffffu, B.re, 1), __shfl_down_sync(0xffffffffu, B.im, 1)};
  if (lane == 31) x = cx<T>{T(0), T(0)};
  for (int i = i1 - 1; i >= i0; --i) {
    const T a = ha[i];
    const cx<T> v = col[i];
    x = cx<T>{fma(a, x.re, v.re), fma(a, x.im, v.im)};
    col[i] = x;
  }
  __syncwarp();
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

template <typename T, typename S>
__device__ __forceinline__ cx<T> cvt(cx<S> v) {
  return cx<T>{(T)v.re, (T)v.im};
}

// ---------------------------------------------------------------------------
// Y-step Gram of a real slice (k = 0, and k = n3/2 for even n3) in an FP32
// engine, in FP64 accuracy.  X~' of a real slice is real, and for traffic data
// the DC slice is badly conditioned: it carries the mean traffic, the columns
// of X~'_0 lie close together, and G = X~'^H H_rho1 X~' reaches a condition
// number near 2e6 along a completion of the 144 x 288 x 168 tensor at 40-60%
// observed, while every other slice stays below 1e2.  An FP32 G^+ has entries
// of size 1/lambda_min; their rounding reaches the new Y~ amplified by that
// condition number.  So on these slices G and Dg are accumulated with
// error-free products and sums (the callers), the pseudo-inverse is taken in
// df64 arithmetic (FP64-class, on the FP32 pipes) with the FP64 path's cutoff (d.rtol64), and t G^+ is kept in
// FP64 (d.Gp64, slot 0 for k = 0, slot 1 for the Nyquist slice) so that
// k_ystep applies it in FP64.
//
// M: 7 r^2 + 3 r + 2 complex doubles of shared memory holding G (first r^2,
// row-major) and Dg (at 6 r^2, after the 2 r^2 work area) on entry.  Every thread of the block calls it.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t real_gram_doubles(int r) { return 7 * (size_t)r * r + 3 * (size_t)r + 2; }
// Where the callers leave G and Dg in M (the layout below).
__device__ __forceinline__ cx<double>* real_gram_G(cx<double>* M, int) { return M; }
__device__ __forceinline__ cx<double>* real_gram_Dg(cx<double>* M, int rr) { return M + 6 * rr; }

template <typename T, int RP>
__device__ __noinline__ void real_gram_solve_store(const Dev<T>& d, int k, cx<double>* M) {
  const int r = d.r, rr = r * r, tid = threadIdx.x, nt = blockDim.x;
  cx<double>* G64 = real_gram_G(M, rr);
  cx<double>* Ap64 = G64 + rr;
  cx<double>* P64 = Ap64 + rr;
  cx<double>* V64 = P64 + rr;
  cx<double>* W64 = V64 + rr;  // 2 r^2
  cx<double>* Dg64 = real_gram_Dg(M, rr);
  cx<double>* piv64 = Dg64 + rr;  // 3 r
  double* sred = reinterpret_cast<double*>(piv64 + 3 * r);  // 4
  const double rtol = d.rtol64;
  if (d.scaled) {
    // lambda_max of G for the step beta / L2 (the eigendecomposition in FP32;
    // the inverse below is the df64 one whenever it is certified)
    jacobi_fallback<double, true>(G64, Ap64, P64, V64, W64, piv64, r, rtol, sred + 2);
    __syncthreads();
  }
  // Gauss-Jordan on the real Gram (df64), accepted when ||G||_F ||G^-1||_F < 1/(2 rtol)
  // (then lambda_min > rtol lambda_max: nothing is cut, G^+ = G^-1); otherwise the
  // eigendecomposition fallback applies the cutoff
  // With the rank rule on (step 5), only the leading ra x ra block is active: the
  // other rows and columns of G are zero, and so are those of G^+.
  const int ra = d.rk ? d.rk[k] : r, ra2 = ra * ra;
  double* g = reinterpret_cast<double*>(Ap64);      // ra^2 real values of G (compact)
  double* wk = reinterpret_cast<double*>(W64);      // 2 ra^2
  for (int e = tid; e < ra2; e += nt) g[e] = G64[(e / ra) * r + e % ra].re;
  __syncthreads();
  {
    // df64 elimination in registers (FP64-pipe operations here wait some 250
    // cycles each, and the elimination is a chain of them); the norms come with it
    const int ok = gj_regs_df(g, wk, ra);
    if (tid == 0) {  // ||G||_F ||G^-1||_F < 1/(2 rtol)
      const double an = g_solve_xch[200], in = g_solve_xch[201];
      sred[1] = (ok && isfinite(in) && isfinite(an) && an * in < 0.5 / rtol) ? 1.0 : 0.0;
    }
  }
  __syncthreads();
  if (sred[1] != 0.0) {
    for (int e = tid; e < rr; e += nt) {  // g (aliasing Ap64) is no longer read
      const int i = e / r, j = e - i * r;
      Ap64[e] = cx<double>{(i < ra && j < ra) ? 0.5 * (wk[i * ra + j] + wk[j * ra + i]) : 0.0, 0.0};
    }
  } else {
    jacobi_fallback<double, true>(G64, Ap64, P64, V64, W64, piv64, r, rtol, sred + 2);
  }
  __syncthreads();
  const double t2 = d.scaled ? ((sred[2] > 0.0) ? (double)d.beta / sred[2] : 0.0) : 1.0;
  const int slot = (k == 0) ? 0 : 1;
  for (int e = tid; e < rr; e += nt) {
    const double g = Ap64[e].re * t2;
    d.Gp64[(size_t)slot * rr + e] = cx<double>{g, 0.0};
    d.Gp[(size_t)k * rr + e] = cx<T>{(T)g, T(0)};
    d.Dg[(size_t)k * rr + e] = cx<T>{(T)Dg64[e].re, T(0)};
  }
}

// G = X~'^H H_rho1 X~' and Dg = -(X~'^H (X~' - X~) + rho1 (H X~')^H (H X~')) of
// a real slice from the real parts of X~' (Xn) and X~ (Xo), [r][n1] each, with
// dot2 accumulation; tp adjacent threads per entry split the rows and their
// (sum + compensation) values are added in FP64.  Writes G and Dg in the
// layout of real_gram_solve_store.
template <typename T>
__device__ __noinline__ void real_gram_accumulate(const Dev<T>& d, const cx<T>* Xn, const cx<T>* Xo, cx<double>* M) {
  const int n1 = d.n1, r = d.r, rr = r * r, tid = threadIdx.x, nt = blockDim.x;
  const double rho1 = (double)d.rho1;
  int tp = 1;
  while (tp < 32 && tp * 2 * rr <= nt) tp *= 2;
  const int q = tid & (tp - 1);
  for (int base = 0; base < rr * tp; base += nt) {  // every thread runs the same passes
    const int task = (base + tid) / tp;
    double a0 = 0.0, hh = 0.0, dd = 0.0;
    if (task < rr) {
      const int s = task / r, u = task - s * r;
      const cx<T>* xs = Xn + (size_t)s * n1;
      const cx<T>* xu = Xn + (size_t)u * n1;
      const cx<T>* ou = Xo + (size_t)u * n1;
      T s0 = T(0), c0 = T(0), s1 = T(0), c1 = T(0), s2 = T(0), c2 = T(0);
      // this thread's rows q, q + tp, ... from a task-dependent start, so that the
      // tasks of a warp read different banks (rows of the r columns often sit a
      // multiple of 128 bytes apart)
      const int K = (n1 - q + tp - 1) / tp;
      const int off = K > 0 ? ((base + tid) / tp & 7) % K : 0;
      for (int kk = 0; kk < K; ++kk) {
        const int i = q + tp * (kk + off < K ? kk + off : kk + off - K);
        const T a = xs[i].re, b = xu[i].re;
        dot2(s0, c0, a, b);
        dot2(s2, c2, a, b - ou[i].re);
        if (i + 1 < n1) dot2(s1, c1, a - xs[i + 1].re, b - xu[i + 1].re);
      }
      a0 = (double)s0 + (double)c0;
      hh = (double)s1 + (double)c1;
      dd = (double)s2 + (double)c2;
    }
    for (int o = tp >> 1; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      hh += __shfl_xor_sync(0xffffffffu, hh, o);
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
    }
    if (task < rr && q == 0) {
      real_gram_G(M, rr)[task] = cx<double>{a0 + rho1 * hh, 0.0};
      real_gram_Dg(M, rr)[task] = cx<double>{-(dd + rho1 * hh), 0.0};
    }
  }
  __syncthreads();
}

// TS is the type of the two r x r pseudo-inverses (double in the precision
// form, where the Grams go to FP64 for the solve); the contractions run in T.
// Threads of the X-step CTA: 1024 for r > 16, where one CTA per slice does
// r^3 solve steps and r^2 n1 Gram products (more warps hide the latencies and
// the Gauss-Jordan steps take one element per thread).
__host__ __device__ constexpr int xstep_threads(int rp) { return rp > 16 ? 1024 : kSliceThreads; }

template <typename T, int RP, typename TS = T>
__global__ void __launch_bounds__(xstep_threads(RP), 1) k_xstep(Dev<T> d, const cx<T>* __restrict__ Qin, int arrays_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  const int k = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, r = d.r, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const XLayout lay = xstep_layout<T, TS>(n1, n2, r, arrays_in_smem != 0);
  cx<TS>* A = reinterpret_cast<cx<TS>*>(smem + lay.mats);
  cx<TS>* Ap = A + rr;
  cx<TS>* P = Ap + rr;
  cx<TS>* V = P + rr;
  cx<TS>* Wk = V + rr;
  cx<TS>* Gm = Wk + 2 * rr;
  cx<TS>* Dgm = Gm + rr;
  cx<TS>* pivbuf = Dgm + rr;  // 3 r
  TS* sred = reinterpret_cast<TS*>(pivbuf + 3 * r);
  T* hinv = reinterpret_cast<T*>(smem + lay.ht);
  T* ha = hinv + n1;
  cx<T>* Xs;
  cx<T>* Qs;
  cx<T>* Ts;
  cx<T>* Xg = d.Xt + (size_t)k * r * n1;
  const cx<T>* Qg = Qin + (size_t)k * r * n1;
  // the slice's X~, Q and the H_rho1 pivots go to shared memory by asynchronous
  // copies, all in flight while A is summed below
  if (arrays_in_smem) {
    Xs = reinterpret_cast<cx<T>*>(smem + lay.xs);
    Qs = reinterpret_cast<cx<T>*>(smem + lay.qs);
    Ts = reinterpret_cast<cx<T>*>(smem + lay.ts);
    for (int e = tid; e < r * n1; e += blockDim.x) {
      cp_async_elem(Xs + e, Xg + e);
      cp_async_elem(Qs + e, Qg + e);
    }
  } else {
    Xs = Xg;
    Qs = const_cast<cx<T>*>(Qg);
    Ts = d.Tb + (size_t)k * r * n1;
  }
  for (int i = tid; i < 2 * n1; i += blockDim.x) cp_async_elem(hinv + i, d.hinv + i);
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const T rho1 = d.rho1;
  const TS rtol = (TS)d.rtol;

  constexpr bool kDF = sizeof(T) == 4 && sizeof(TS) == 8;  // FP64 solves of an FP32 engine: df64
  bool certA;
  T t1;
  if (d.apre) {
    // A^+, P, the certificate and the step along d_X were formed by k_xa from the
    // tile Grams of the last Y-step
    for (int e = tid; e < rr; e += blockDim.x) {
      Ap[e] = cvt<TS>(d.Apg[(size_t)k * rr + e]);
      P[e] = cvt<TS>(d.Pg[(size_t)k * rr + e]);
    }
    certA = d.certA[k] != 0;
    t1 = d.tstep[k];
    cp_async_wait_all();
    __syncthreads();
  } else {
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
      A[s * r + u] = cx<TS>{(TS)v.re, (TS)v.im};
      A[u * r + s] = cx<TS>{(TS)v.re, (TS)(-v.im)};
    }
  }
  cp_async_wait_all();
  __syncthreads();
  certA = block_pinv_herm<TS, RP, kDF>(A, Ap, P, V, Wk, pivbuf, sred, r, rtol, d.scaled != 0) != 0;
  // step along d_X: 1, or alpha / L1 with L1 = ||H_rho1||_2 lambda_max(A)
  t1 = d.scaled ? ((sred[2] > TS(0)) ? d.alpha / (d.hnorm * (T)sred[2]) : T(0)) : T(1);
  }

  // ---- B = Q A^+ - rho1 (H^T H X~) P ------------------------------------------------------
  // A^+ and P in T (the work area of the solve is free again); a thread forms
  // SB columns of one row, so each Q value it loads feeds SB products.
  cx<T>* ApT = reinterpret_cast<cx<T>*>(Wk);
  cx<T>* PT = ApT + rr;
  for (int e = tid; e < rr; e += blockDim.x) {
    ApT[e] = cvt<T>(Ap[e]);
    PT[e] = cvt<T>(P[e]);
  }
  __syncthreads();
  {
    constexpr int SB = RP < 8 ? RP : (RP == 8 ? 2 : 8);  // enough items to fill the CTA at small n1
    const int nsb = (r + SB - 1) / SB;
    for (int e = tid; e < nsb * n1; e += blockDim.x) {
      const int sb = e / n1, i = e - sb * n1, s0 = sb * SB;
      cx<T> acc[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) acc[c] = cx<T>{T(0), T(0)};
      for (int u = 0; u < r; ++u) {
        const cx<T> q = Qs[(size_t)u * n1 + i];
#pragma unroll
        for (int c = 0; c < SB; ++c)
          if (s0 + c < r) cfma(acc[c], q, ApT[u * r + s0 + c]);
      }
#pragma unroll
      for (int c = 0; c < SB; ++c) {
        const int s = s0 + c;
        if (s >= r) break;
        if (rho1 != T(0)) {
          cx<T> hx = {T(0), T(0)};
          if (certA) {
            hx = hth_at(Xs + (size_t)s * n1, i, n1);  // P = I
          } else {
            for (int u = 0; u < r; ++u) cfma(hx, hth_at(Xs + (size_t)u * n1, i, n1), PT[u * r + s]);
          }
          acc[c] = acc[c] - hx * rho1;
        }
        Ts[(size_t)s * n1 + i] = acc[c];
      }
    }
  }
  __syncthreads();
  // ---- d_X = H_rho1^{-1} B: one warp per column --------------------------------------------
  if (rho1 != T(0) && n1 > 1) {
    for (int s = wid; s < r; s += nw) warp_tridiag_solve<T>(Ts + (size_t)s * n1, n1, hinv, ha);
    __syncthreads();
  }
  // ---- X~' = X~ + t d_X (Ts; Xs keeps the old factor) -------------------------------------
  double dmax = 0.0;
  for (int e = tid; e < r * n1; e += blockDim.x) {
    const cx<T> x0 = Xs[e];
    cx<T> v = (d.scaled ? x0 + Ts[e] * t1 : x0 + Ts[e]);
    if (realslice) v.im = T(0);
    Ts[e] = v;
    if (d.conv) dmax = fmax(dmax, (double)cabs(v - x0));
  }
  if (d.conv) block_max_to(dmax, d.conv + 0);
  __syncthreads();

  if (sizeof(T) == 4 && realslice) {
    // FP64-accurate Gram, df64 pseudo-inverse, FP64 G^+ (see real_gram_solve_store)
    cx<double>* M64 = reinterpret_cast<cx<double>*>(smem + lay.mats);
    real_gram_accumulate<T>(d, Ts, Xs, M64);
    real_gram_solve_store<T, RP>(d, k, M64);
    for (int e = tid; e < r * n1; e += blockDim.x) Xg[e] = Ts[e];
    return;
  }
  // ---- G = X~'^H H_rho1 X~' (Hermitian) and Dg = E - G ----------------------------------
  // (H X~')^H (H X~') = sum_i conj(x_i - x_{i+1}) (x_i - x_{i+1}) row by row.
  // tp adjacent threads share one (s, u) pair and split the rows; their partial
  // sums are combined by shuffles in a fixed order.  The rows go through
  // shared memory kGramRows at a time (X~' with one row of halo).
  {
    int tp = 1;
    while (tp < 32 && tp * 2 * rr <= (int)blockDim.x) tp *= 2;
    const int per_pass = blockDim.x / tp;
    const int q = tid & (tp - 1);
    constexpr int MT = (RP * RP + xstep_threads(RP) - 1) / xstep_threads(RP);  // passes (tp = 1 when r r >= threads)
    cx<T> a0[MT], hh[MT], dd[MT];
#pragma unroll
    for (int t = 0; t < MT; ++t) a0[t] = hh[t] = dd[t] = cx<T>{T(0), T(0)};
    cx<T>* gx = reinterpret_cast<cx<T>*>(smem + lay.gs);  // [r][kGramLd] rows i0 .. i0 + kGramRows of X~'
    cx<T>* go = gx + (size_t)r * kGramLd;                 // [r][kGramLd] rows i0 .. of X~
    if (arrays_in_smem) {
      // X~' and X~ are resident: read them in place
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const int task = t * per_pass + tid / tp;
        if (task < rr) {
          const int s = task / r, u = task - s * r;
          const cx<T>* xs = Ts + (size_t)s * n1;
          const cx<T>* xu = Ts + (size_t)u * n1;
          const cx<T>* ou = Xs + (size_t)u * n1;
          // rows from a task-dependent start: the tasks of a warp read different banks
          const int K = (n1 - q + tp - 1) / tp;
          const int off = K > 0 ? ((tid / tp) & 7) % K : 0;
          for (int kk = 0; kk < K; ++kk) {
            const int i = q + tp * (kk + off < K ? kk + off : kk + off - K);
            const cx<T> a = xs[i], b = xu[i];
            cfmaconj(a0[t], a, b);
            cfmaconj(dd[t], a, b - ou[i]);
            if (i + 1 < n1) cfmaconj(hh[t], a - xs[i + 1], b - xu[i + 1]);
          }
        }
      }
    }
    for (int i0 = 0; !arrays_in_smem && i0 < n1; i0 += kGramRows) {
      const int nrow = min(kGramRows + 1, n1 - i0);
      for (int e = tid; e < r * kGramLd; e += blockDim.x) {
        const int s = e / kGramLd, ii = e - s * kGramLd;
        if (ii < nrow) {
          gx[e] = Ts[(size_t)s * n1 + i0 + ii];
          if (ii < kGramRows) go[e] = Xs[(size_t)s * n1 + i0 + ii];
        }
      }
      __syncthreads();
      const int iend = min(kGramRows, n1 - i0);
#pragma unroll
      for (int t = 0; t < MT; ++t) {
        const int task = t * per_pass + tid / tp;
        if (task < rr) {
          const int s = task / r, u = task - s * r;
          const cx<T>* xs = gx + s * kGramLd;
          const cx<T>* xu = gx + u * kGramLd;
          const cx<T>* ou = go + u * kGramLd;
          for (int ii = q; ii < iend; ii += tp) {
            const cx<T> a = xs[ii], b = xu[ii];
            cfmaconj(a0[t], a, b);
            cfmaconj(dd[t], a, b - ou[ii]);
            if (i0 + ii + 1 < n1) cfmaconj(hh[t], a - xs[ii + 1], b - xu[ii + 1]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int t = 0; t < MT; ++t) {
      for (int o = tp >> 1; o > 0; o >>= 1) {
        a0[t].re += __shfl_xor_sync(0xffffffffu, a0[t].re, o);
        a0[t].im += __shfl_xor_sync(0xffffffffu, a0[t].im, o);
        hh[t].re += __shfl_xor_sync(0xffffffffu, hh[t].re, o);
        hh[t].im += __shfl_xor_sync(0xffffffffu, hh[t].im, o);
        dd[t].re += __shfl_xor_sync(0xffffffffu, dd[t].re, o);
        dd[t].im += __shfl_xor_sync(0xffffffffu, dd[t].im, o);
      }
      const int task = t * per_pass + tid / tp;
      if (task < rr && q == 0) {
        const int s = task / r, u = task - s * r;
        cx<T> dg = {-(dd[t].re + rho1 * hh[t].re), -(dd[t].im + rho1 * hh[t].im)};
        if (realslice) dg.im = T(0);
        Dgm[s * r + u] = cvt<TS>(dg);
        if (s <= u) {
          cx<T> g = {a0[t].re + rho1 * hh[t].re, a0[t].im + rho1 * hh[t].im};
          if (s == u || realslice) g.im = T(0);
          Gm[s * r + u] = cvt<TS>(g);
          Gm[u * r + s] = cx<TS>{(TS)g.re, -(TS)g.im};
        }
      }
    }
  }
  __syncthreads();
  block_pinv_herm<TS, RP, kDF>(Gm, Ap, P, V, Wk, pivbuf, sred, r, rtol, d.scaled != 0);
  // step along d_Y: 1, or beta / L2 with L2 = lambda_max(G), folded into G^+
  const TS t2 = d.scaled ? ((sred[2] > TS(0)) ? (TS)d.beta / sred[2] : TS(0)) : TS(1);
  // ---- Dg and t G^+ for k_ystep; X~ <- X~' -------------------------------------------------
  for (int e = tid; e < rr; e += blockDim.x) {
    cx<T> gp = cvt<T>(Ap[e] * t2);
    if (realslice) gp.im = T(0);
    d.Dg[(size_t)k * rr + e] = cvt<T>(Dgm[e]);
    d.Gp[(size_t)k * rr + e] = gp;
  }
  for (int e = tid; e < r * n1; e += blockDim.x) Xg[e] = Ts[e];
}

// ---------------------------------------------------------------------------
// Y-step of slice k on a tile of TW = 32 CPL columns (step 2):
//   D   = X~'^H R~_k(:, tile)       (contraction over n1; reads R~ once)
//   Y~' = Y~ + G^+ (Dg Y~ + D)      (= Y~ - G^+ grad_Y, see k_xstep)
// then the Grams of Y~' over each 32 columns (A of the next X-step) and
// Z~ = X~'Y~' on the tile (step 3, read by the slab kernel).
// Grid (S, ceil(n2/TW)); warp w accumulates rows i = w, w + 8, ...; a lane
// holds CPL columns (two for r <= 16, so each X~' value read from shared
// memory feeds two columns).
// ---------------------------------------------------------------------------
constexpr int kYThreads = 256;

__host__ __device__ constexpr int ystep_cpl(int rp) { return rp <= 16 ? 2 : 1; }

// Shared memory of k_ystep: partial sums, D, old and new Y~ of the tile, Dg,
// G^+, X~' of the slice (XSH), then r^2 doubles for the FP64 G^+ of a real slice.
template <typename T>
__host__ __device__ inline size_t ystep_gh64_offset(int n1, int r, int rp, bool x_in_smem, bool tcy) {
  const size_t tw = 32 * (size_t)ystep_cpl(rp);
  return align_up(((size_t)((tcy ? 0 : kYThreads / 32) + 3) * rp * tw + 2 * (size_t)r * r +
                   (x_in_smem && !tcy ? (size_t)r * n1 : 0)) *
                      sizeof(cx<T>),
                  16);
}
// TCY (precision form, r > 16): D comes as ksplit partial sums over ranges of
// n1 from k_dcon_tc (d.Dpart) and Z~ is formed by k_zsyn_tc afterwards.
// XSH: X~' of the slice staged in shared memory (the compiler then sees
// shared-memory loads in the contraction loops), else read through L1.
template <typename T, int RP, bool TCY, bool XSH>
__device__ __forceinline__ void ystep_impl(const Dev<T>& d, unsigned char* smem) {
  constexpr int CPL = ystep_cpl(RP), TW = 32 * CPL;
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * TW;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S, rr = r * r;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  cx<T>* red = reinterpret_cast<cx<T>*>(smem);  // [nw][RP][TW]
  cx<T>* Ds = red + (TCY ? 0 : nw * RP * TW);   // [RP][TW]
  cx<T>* Yo = Ds + RP * TW;                     // [RP][TW]
  cx<T>* Dgs = Yo + RP * TW;                    // [rr]
  cx<T>* Gh = Dgs + rr;                         // [rr]
  cx<T>* Yn = Gh + rr;                          // [RP][TW] the new Y~' of the tile
  const cx<T>* Xg = d.Xt + (size_t)k * r * n1;
  const cx<T>* Xs = Xg;                         // [r][n1]
  if constexpr (XSH) {
    cx<T>* xs = Yn + RP * TW;
    for (int e = tid; e < r * n1; e += blockDim.x) xs[e] = Xg[e];
    Xs = xs;
  }
  // real slices of an FP32 engine: t G^+ in FP64 (k_xstep / k_xc), applied in FP64
  const bool realslice = (k == 0) || (2 * k == d.n3);
  const bool g64 = sizeof(T) == 4 && realslice && d.Gp64 != nullptr;
  double* gh64 = reinterpret_cast<double*>(smem + ystep_gh64_offset<T>(n1, r, RP, XSH, TCY));
  for (int e = tid; e < rr; e += blockDim.x) {
    Dgs[e] = d.Dg[(size_t)k * rr + e];
    Gh[e] = d.Gp[(size_t)k * rr + e];
    if (g64) gh64[e] = d.Gp64[(size_t)(k == 0 ? 0 : 1) * rr + e].re;
  }
  for (int e = tid; e < r * TW; e += blockDim.x) {
    const int s = e / TW, c = e - s * TW;
    Yo[s * TW + c] = (j0 + c < n2) ? d.Yt[((size_t)k * r + s) * n2 + j0 + c] : cx<T>{T(0), T(0)};
  }
  __syncthreads();
  cx<T> acc[CPL][RP];
#pragma unroll
  for (int h = 0; h < CPL; ++h)
#pragma unroll
    for (int s = 0; s < RP; ++s) acc[h][s] = cx<T>{T(0), T(0)};
  bool live[CPL];
#pragma unroll
  for (int h = 0; h < CPL; ++h) live[h] = j0 + 32 * h + lane < n2;
  const cx<T>* rbase = d.Rt + (size_t)k * n2 + j0 + lane;  // + i * S * n2 + 32 h
  const size_t rstride = (size_t)S * n2;
  if constexpr (!TCY) {
    int i = wid;
    for (; i + nw < n1; i += 2 * nw) {
      cx<T> v[2][CPL];
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int h = 0; h < CPL; ++h)
          v[q][h] = live[h] ? ldg_cx(rbase + (size_t)(i + q * nw) * rstride + 32 * h) : cx<T>{T(0), T(0)};
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int s = 0; s < RP; ++s)
          if (s < r) {
            const cx<T> x = Xs[(size_t)s * n1 + i + q * nw];
#pragma unroll
            for (int h = 0; h < CPL; ++h) cfmaconj(acc[h][s], x, v[q][h]);
          }
    }
    for (; i < n1; i += nw) {
      cx<T> v[CPL];
#pragma unroll
      for (int h = 0; h < CPL; ++h)
        v[h] = live[h] ? ldg_cx(rbase + (size_t)i * rstride + 32 * h) : cx<T>{T(0), T(0)};
#pragma unroll
      for (int s = 0; s < RP; ++s)
        if (s < r) {
          const cx<T> x = Xs[(size_t)s * n1 + i];
#pragma unroll
          for (int h = 0; h < CPL; ++h) cfmaconj(acc[h][s], x, v[h]);
        }
    }
  }
  if constexpr (!TCY) {
#pragma unroll
    for (int s = 0; s < RP; ++s)
#pragma unroll
      for (int h = 0; h < CPL; ++h) red[(wid * RP + s) * TW + 32 * h + lane] = acc[h][s];
  }
  __syncthreads();
  // V = Dg Y~ + D (= -grad_Y on the tile)
  for (int e = tid; e < r * TW; e += blockDim.x) {
    const int s = e / TW, c = e - s * TW;
    cx<T> v = {T(0), T(0)};
    if constexpr (TCY) {
      if (j0 + c < n2) {
        const cx<T>* dp = d.Dpart + ((size_t)k * d.ksplit * r + s) * n2 + j0 + c;  // + z r n2
        const size_t zs = (size_t)r * n2;
        int z = 0;
        for (; z + 4 <= d.ksplit; z += 4) {  // four loads in flight, summed in order
          cx<T> q[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) q[w] = dp[(z + w) * zs];
#pragma unroll
          for (int w = 0; w < 4; ++w) v = v + q[w];
        }
        for (; z < d.ksplit; ++z) v = v + dp[z * zs];
      }
    } else {
      for (int w = 0; w < nw; ++w) v = v + red[(w * RP + s) * TW + c];
    }
    for (int u = 0; u < r; ++u) cfma(v, Dgs[s * r + u], Yo[u * TW + c]);
    Ds[s * TW + c] = v;
  }
  __syncthreads();
  double dmax = 0.0;
  for (int e = tid; e < RP * TW; e += blockDim.x) {
    const int s = e / TW, c = e - s * TW;
    if (s >= r || j0 + c >= n2) {
      Yn[e] = cx<T>{T(0), T(0)};
      continue;
    }
    cx<T> y = Yo[e];
    if (g64) {
      double yd = (double)y.re;
      for (int u = 0; u < r; ++u) yd = fma(gh64[s * r + u], (double)Ds[u * TW + c].re, yd);
      y.re = (T)yd;
    } else {
      for (int u = 0; u < r; ++u) cfma(y, Gh[s * r + u], Ds[u * TW + c]);
    }
    if (realslice) y.im = T(0);
    d.Yt[((size_t)k * r + s) * n2 + j0 + c] = y;
    Yn[e] = y;
    if (d.conv) dmax = fmax(dmax, (double)cabs(y - Yo[e]));
  }
  if (d.conv) block_max_to(dmax, d.conv + 1);
  __syncthreads();

  // ---- Grams of the new Y~' over each 32 columns (A of the next X-step) ----------------
  // a thread per (s, u) pair of a tile; the columns are visited from (u mod 32)
  // on, so the threads of a half-warp (consecutive u) read different banks
  const int ntask = r * (r + 1) / 2;
  for (int t = tid; t < CPL * ntask; t += blockDim.x) {
    const int h = t / ntask, task = t - h * ntask;
    const int tile = blockIdx.y * CPL + h;
    if (tile >= d.ytiles) continue;
    int s, u;
    tri_index(task, r, s, u);
    const cx<T>* ys = Yn + s * TW + 32 * h;
    const cx<T>* yu = Yn + u * TW + 32 * h;
    cx<T> g = {T(0), T(0)};
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      const int cc = (c + u) & 31;
      cfmac(g, ys[cc], yu[cc]);
    }
    d.Ag[((size_t)k * d.ytiles + tile) * ntask + task] = cx<double>{(double)g.re, (double)g.im};
  }

  // ---- Z~(:, tile, k) = X~' Y~'  (step 3, written for the slab kernel) ----------------
  if constexpr (TCY) return;
  cx<T> yv[CPL][RP];
#pragma unroll
  for (int h = 0; h < CPL; ++h)
#pragma unroll
    for (int s = 0; s < RP; ++s) yv[h][s] = Yn[s * TW + 32 * h + lane];
  cx<T>* zc = d.Zt + (size_t)k * n2 + j0 + lane;
  for (int i = wid; i < n1; i += nw) {
    cx<T> z[CPL];
#pragma unroll
    for (int h = 0; h < CPL; ++h) z[h] = cx<T>{T(0), T(0)};
#pragma unroll
    for (int s = 0; s < RP; ++s)
      if (s < r) {
        const cx<T> x = Xs[(size_t)s * n1 + i];
#pragma unroll
        for (int h = 0; h < CPL; ++h) cfma(z[h], x, yv[h][s]);
      }
#pragma unroll
    for (int h = 0; h < CPL; ++h)
      if (live[h]) {
        const size_t o = (size_t)i * rstride + 32 * h;
        if (d.dZt) d.dZt[zc - d.Zt + o] = z[h] - zc[o];  // Z~^{l+1} - Z~^l for the stopping test
        zc[o] = z[h];
      }
  }
}

// XSH is chosen at launch (d.yx_global == 0 for XSH, TCY never stages).
template <typename T, int RP, bool TCY = false, bool XSH = !TCY>
__global__ void __launch_bounds__(kYThreads) k_ystep(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (converged(d)) return;
  ystep_impl<T, RP, TCY, XSH && !TCY>(d, smem);
}

template <typename T>
__host__ inline size_t ystep_smem_bytes(int n1, int r, int rp, bool x_in_smem = true, bool tcy = false) {
  return ystep_gh64_offset<T>(n1, r, rp, x_in_smem, tcy) + (size_t)r * r * sizeof(double);
}

template <typename T>
__host__ inline size_t qcon_smem_bytes(int n2, int r, int) {
  return (size_t)r * n2 * sizeof(cx<T>);
}

}  // namespace tc
