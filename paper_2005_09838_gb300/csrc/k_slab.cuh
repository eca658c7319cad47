// Slab kernel of the TCTF2R iteration: one CTA per mode-1 index i1 (one OD
// pair), holding the spatial slab (i1, :, :) in shared memory.
//
//   phase A  Z~(i1, j, k) = sum_s X~(i1, s, k) Y~(s, j, k) for the solved
//            slices k (step 3), inverse mode-3 DFT of every tube (Eq. (barAAk))
//   phase B  W-step of every row (i1, :, i3) (step 4, Eq. (subquKKT)), written
//            as the residual R = W - Z
//   phase C  forward mode-3 DFT of every tube of R (step 7, Eq. (bar BA-k)),
//            stored as R~
#pragma once

namespace tc {

enum SlabMode : int { MODE_ITER = 0, MODE_W = 1, MODE_R = 2 };

constexpr int kSlabMaxThreads = 288;

struct SlabLayout {
  size_t xrow, wtab, red, spec, spat, total;  // byte offsets and total shared bytes
  size_t slab_bytes;                          // bytes of the slab buffers per CTA
};

// Shared-memory layout.  With a register FFT (specialised) only the spatial
// slab n3 x n2 is kept; the generic transform also stages the half spectrum.
template <typename T>
__host__ __device__ inline SlabLayout slab_layout(int n2, int n3, int r, bool specialised, bool slabs_in_smem) {
  SlabLayout L{};
  const int S = n3 / 2 + 1;
  size_t off = 0;
  L.xrow = off;
  off = align_up(off + sizeof(cx<T>) * S * r, 16);
  L.wtab = off;
  off = align_up(off + sizeof(T) * 4 * n2, 16);
  L.red = off;
  off = align_up(off + sizeof(double) * 4 * 32, 16);
  const size_t spec_bytes = specialised ? 0 : align_up(sizeof(cx<T>) * (size_t)S * n2, 16);
  const size_t spat_bytes = align_up(sizeof(T) * (size_t)n3 * n2, 16);
  L.slab_bytes = spec_bytes + spat_bytes;
  if (slabs_in_smem) {
    L.spec = off;
    L.spat = off + spec_bytes;
    off += spec_bytes + spat_bytes;
  } else {
    L.spec = 0;
    L.spat = spec_bytes;
  }
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// W-step of one spatial row (i1, :, i3) in residual form.
//
// Eq. (subquKKT): for a missing (i, j), (W K_{mu rho2})_ij = Z_ij with
// K_{mu rho2} = (1+mu) I + rho2 K^T K (tridiagonal); W_ij = G_ij on the mask.
// With W = Z + R the unknown R solves the same tridiagonal system with
// right-hand side -(mu + rho2 deg_j) z_j + rho2 (z_{j-1} + z_{j+1}) at missing
// entries and g_j - z_j at observed ones (identity rows).  Observed entries
// split the row into runs; the LU pivots of a run depend only on the position
// in the run and on whether it starts at j = 0, so their inverses come from a
// table and each sweep is a single fused multiply-add chain:
//   forward   d_j = a_j d_{j-1} + b_j,   backward  r_j = c_j r_{j+1} + d_j.
// The last entry of the row (one neighbour) gets its pivot computed here.
// On return row[j] holds r_j = w_j - z_j.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void wstep_row(T* __restrict__ row, const T* __restrict__ g, const uint32_t* __restrict__ m, int n2,
                          int words, T mu, T rho2, const T* __restrict__ wtab) {
  const T* inv1 = wtab;           // runs starting at j = 0
  const T* inv0 = wtab + n2;      // runs starting at j > 0
  const T* c1 = wtab + 2 * n2;    // rho2 * inv1
  const T* c0 = wtab + 3 * n2;    // rho2 * inv0
  const T rho2sq = rho2 * rho2;
  // ---- forward sweep -------------------------------------------------------
  T dprev = T(0), zprev = T(0);
  T z = row[0];
  int p = -1;
  bool st0 = false;
  T invprev = T(0);
  for (int w = 0; w < words; ++w) {
    const uint32_t mw = __ldg(m + w);
    T gv[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int j = 32 * w + q;
      gv[q] = (j < n2) ? __ldg(g + j) : T(0);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int j = 32 * w + q;
      if (j < n2) {
        const T znext = (j + 1 < n2) ? row[j + 1] : T(0);
        T a, b;
        if ((mw >> q) & 1u) {
          a = T(0);
          b = gv[q] - z;
          p = -1;
        } else {
          if (p < 0) st0 = (j == 0);
          ++p;
          T inv;
          if (j == n2 - 1 && n2 > 1) {
            inv = T(1) / (T(1) + mu + rho2 - ((p > 0) ? rho2sq * invprev : T(0)));
          } else {
            inv = st0 ? inv1[p] : inv0[p];
          }
          invprev = inv;
          const T deg = T((j > 0) + (j + 1 < n2));
          const T e = -(mu + rho2 * deg) * z + rho2 * (zprev + znext);
          a = rho2 * inv;
          b = e * inv;
        }
        const T d = fma(a, dprev, b);
        row[j] = d;
        dprev = d;
        zprev = z;
        z = znext;
      }
    }
  }
  // ---- backward sweep ------------------------------------------------------
  T rnext = T(0);
  int pb = -1, rs = 0;
  for (int w = words - 1; w >= 0; --w) {
    const uint32_t mw = __ldg(m + w);
#pragma unroll
    for (int q = 31; q >= 0; --q) {
      const int j = 32 * w + q;
      if (j < n2) {
        const T d = row[j];
        T c = T(0);
        if (!((mw >> q) & 1u)) {
          if (pb < 0) {  // right end of a run: locate its start
            const uint32_t below = q ? (mw & ((1u << q) - 1u)) : 0u;
            const int po = below ? (32 * w + 31 - __clz(below)) : prev_observed(m, 32 * w);
            rs = po + 1;
            pb = j - rs;
          }
          if (j < n2 - 1) c = (rs == 0) ? c1[pb] : c0[pb];
          --pb;
        } else {
          pb = -1;
        }
        const T rv = fma(c, rnext, d);
        row[j] = rv;
        rnext = rv;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Generic (any n3) direct transforms of one tube, used when no register FFT
// is specialised for n3: the sums of Eq. (bar BA-k) and Eq. (barAAk).
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
      acc += T(2) * (v.re * w.re + v.im * w.im);  // 2 Re(v conj(w))
    }
    if (even) acc += ((l & 1) ? -spec[(S - 1) * sstride].re : spec[(S - 1) * sstride].re);
    spat[l * pstride] = acc * inv;
  }
}

template <typename T>
__device__ void generic_rdft(const T* spat, int pstride, cx<T>* out, size_t ostride, int n3,
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
    out[k * ostride] = acc;
  }
}

// ---------------------------------------------------------------------------
// MODE_ITER: phases A, B, C (init != 0: W = P_Omega(G), the initial point, in
//            place of the W-step).
// MODE_W   : W = iDFT(X~Y~ + R~); optional copy to Wout (column-major), partial
//            sums ||W||^2 and ||K unfold(W,2)||^2.
// MODE_R   : R = iDFT(R~); partial sums ||R||^2 and ||P_Omega R||^2.
// ---------------------------------------------------------------------------
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kSlabMaxThreads, 1)
    k_slab(Dev<T> d, T* __restrict__ Wout, int slabs_in_smem, int init) {
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
  unsigned char* slab_base =
      slabs_in_smem ? smem : reinterpret_cast<unsigned char*>(d.scratch) + (size_t)i1 * lay.slab_bytes;
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
    for (int j = tid; j < 4 * n2; j += nt) wtab[j] = d.winv[j];
  }
  __syncthreads();

  // ---- phase A: spectrum of each tube, inverse transform ---------------------
  if constexpr (L > 0) {
    constexpr int SL = L / 2 + 1;
    const int t = tid;
    if (t < n2) {
      cx<T> X[SL];
#pragma unroll
      for (int k = 0; k < SL; ++k) {
        X[k] = (MODE == MODE_ITER) ? cx<T>{T(0), T(0)} : d.Rt[((size_t)i1 * SL + k) * n2 + t];
      }
      if (synth) {
        // s-chunks outside, slices inside: all loads of a chunk are independent
        for (int s0 = 0; s0 < r; s0 += 4) {
#pragma unroll
          for (int k = 0; k < SL; ++k) {
            const cx<T>* yk = d.Yt + ((size_t)k * r + s0) * n2 + t;
            const cx<T>* xk = xrow + k * r + s0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (s0 + q < r) cfma(X[k], xk[q], ldg_cx(yk + (size_t)q * n2));
          }
        }
      }
      T x[L];
      fft::irfft<T, L>(X, x);
#pragma unroll
      for (int l = 0; l < L; ++l) spat[l * n2 + t] = x[l];
    }
  } else {
    for (int t = tid; t < n2; t += nt) {
      for (int k = 0; k < S; ++k) {
        cx<T> acc = (MODE == MODE_ITER) ? cx<T>{T(0), T(0)} : d.Rt[((size_t)i1 * S + k) * n2 + t];
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
      a += (double)v * (double)v;
      if (MODE == MODE_W) {
        if (j + 1 < n2) {
          const double dv = (double)v - (double)spat[e + 1];
          b += dv * dv;
        }
        if (Wout) Wout[(size_t)i1 + (size_t)n1 * ((size_t)j + (size_t)n2 * l)] = v;
      } else {
        if (bit_at(d.mask + ((size_t)i1 * n3 + l) * d.words, j)) b += (double)v * (double)v;
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

  if (init || d.rho2 == T(0)) {
    // W = P_Omega(G) (initial point) or the entry-wise form of Eq. (Wkiom)
    // with rho2 = 0: W = Z / (1 + mu) off the mask.
    const T shrink = init ? T(-1) : -d.mu / (T(1) + d.mu);
    for (int e = tid; e < n3 * n2; e += nt) {
      const int l = e / n2, j = e - l * n2;
      const size_t rowi = (size_t)i1 * n3 + l;
      const T z = spat[e];
      spat[e] = bit_at(d.mask + rowi * d.words, j) ? __ldg(d.G + rowi * n2 + j) - z : shrink * z;
    }
  } else {
    for (int l = tid; l < n3; l += nt) {
      const size_t rowi = (size_t)i1 * n3 + l;
      wstep_row<T>(spat + (size_t)l * n2, d.G + rowi * n2, d.mask + rowi * d.words, n2, d.words, d.mu, d.rho2,
                   wtab);
    }
  }
  __syncthreads();

  // ---- phase C: forward transform, store R~ --------------------------------
  if constexpr (L > 0) {
    constexpr int SL = L / 2 + 1;
    const int t = tid;
    if (t < n2) {
      T x[L];
#pragma unroll
      for (int l = 0; l < L; ++l) x[l] = spat[l * n2 + t];
      cx<T> X[SL];
      fft::rfft<T, L>(x, X);
      cx<T>* rt = d.Rt + (size_t)i1 * SL * n2 + t;
#pragma unroll
      for (int k = 0; k < SL; ++k) rt[(size_t)k * n2] = X[k];
    }
  } else {
    for (int t = tid; t < n2; t += nt) {
      generic_rdft<T>(spat + t, n2, d.Rt + (size_t)i1 * S * n2 + t, (size_t)n2, n3, d.twg);
    }
  }
}

}  // namespace tc
