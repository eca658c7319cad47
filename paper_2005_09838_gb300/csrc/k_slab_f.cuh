// Slab kernel with the mode-3 transforms in shared memory: one CTA per mode-1
// index i1 (one OD pair), n3 = 2 M with M = N1 N2, and many threads per tube.
//
// The real transform of length n3 runs as a complex transform of length M on
// the packed even/odd samples z_m = x_{2m} + i x_{2m+1} (Eq. (bar BA-k),
// Eq. (barAAk); the half spectrum of Eq. (rcm_3-k+2) is all that is stored).
// The length-M transform is split into two passes of small DFTs held in
// registers (Cooley-Tukey with M = N1 N2):
//   inverse: DFT_N1 over the stride-N2 slots, twiddle, DFT_N2 over contiguous
//            groups; the spatial value z_m, m = k1 + N1 k2, lands in slot
//            N2 k1 + k2 (a fixed permutation of each tube);
//   forward: the same two passes in reverse order take that permuted order
//            back to the natural order of the spectrum.
// The W-step acts on the rows (i1, :, i3) one by one, so it works in the
// permuted order unchanged: row i3 sits at offset slab_f_off(i3) of every tube.
// Every pass is a loop over independent (group, tube) items with the tube
// index fastest, so a warp reads one slot of 32 tubes (odd tube stride: no
// bank conflicts) and shares its twiddle index; the code of each pass is one
// small DFT, which keeps the instruction footprint small.
//
//   MODE_ITER  A1 split of the half spectrum of Z~ (written by k_ystep);
//              A2/A3 inverse passes; v = G on the mask, Z elsewhere;
//              W-step sweeps (Eq. (subquKKT)); C1/C2 forward passes;
//              C3 split and R~ = W~ - Z~ stored.
//   MODE_W     W = iDFT(Z~ + R~): optional copy to Wout (column-major),
//              partial sums ||W||^2 and ||K unfold(W,2)||^2.
//   MODE_R     R = iDFT(R~): partial sums ||R||^2 and ||P_Omega R||^2.
//   MODE_GRAD  differentiation form: E = P_Omega(iDFT(Z~) - G) and R~ = DFT(E)
//              stored, partial sum ||E||^2 (the masked loss).
#pragma once

namespace tc {

constexpr int kSlabFThreads = 512;
// Items per thread whose global loads are issued together in the first split phase.
constexpr int kSlabFBatch = 4;

// Floats between consecutive tubes: room for the M + 1 complex values of the
// half spectrum, even (complex slots are 8-byte aligned) with an odd number of
// complex values (a warp's slot accesses across 32 tubes hit distinct banks).
__host__ __device__ constexpr int slab_f_stride(int L) { return (((L + 2) / 2) % 2 == 1) ? L + 2 : L + 4; }

struct SlabFLayout {
  size_t msk, stw, wtab, red, buf, total;  // byte offsets and total shared bytes
};

template <typename T>
__host__ __device__ inline SlabFLayout slab_f_layout(int n2, int L) {
  SlabFLayout Lo{};
  const size_t mw = (size_t)(n2 + 31) / 32;
  size_t off = 0;
  Lo.msk = off;  // row mask words [L][mw]
  off = align_up(off + 4 * (size_t)L * mw, 16);
  Lo.stw = off;  // W-step run starts per row and word
  off = align_up(off + 4 * (size_t)L * mw, 16);
  Lo.wtab = off;
  off = align_up(off + sizeof(T) * 6 * (size_t)n2, 16);
  Lo.red = off;
  off = align_up(off + sizeof(double) * 2 * (kSlabFThreads / 32), 16);
  Lo.buf = off;  // [n2][slab_f_stride(L)]
  off = align_up(off + sizeof(T) * (size_t)n2 * slab_f_stride(L), 16);
  Lo.total = off;
  return Lo;
}

// Float offset of spatial index l (0 <= l < 2 N1 N2) inside a tube after the
// inverse passes.
template <int N1, int N2>
__device__ __forceinline__ int slab_f_off(int l) {
  const int m = l >> 1;
  return 2 * (N2 * (m % N1) + m / N1) + (l & 1);
}

template <typename T>
__device__ __forceinline__ cx<T> ld_slot(const T* tb, int slot) {
  return reinterpret_cast<const cx<T>*>(tb)[slot];
}
template <typename T>
__device__ __forceinline__ void st_slot(T* tb, int slot, cx<T> v) {
  reinterpret_cast<cx<T>*>(tb)[slot] = v;
}

// (group, tube) items of a pass, tube index fastest, strided by the block size
// (replaces a division per item).
struct ItemIter {
  int g, t;
  __device__ __forceinline__ ItemIter(int e, int n2) : g(e / n2), t(e - (e / n2) * n2) {}
  __device__ __forceinline__ void advance(int nt, int n2) {
    t += nt;
    while (t >= n2) {
      t -= n2;
      ++g;
    }
  }
};

// One entry of the packed sequence for the inverse real transform:
// z_k = E + i O, E = (a + conj b)/2, O = (a - conj b)/2 * w_L^{-k}, with
// a = X[k], b = X[M - k].
template <typename T, int L>
__device__ __forceinline__ cx<T> inv_split(cx<T> a, cx<T> b, int k) {
  const cx<T> bc = conj(b);
  const cx<T> E = (a + bc) * T(0.5);
  const cx<T> D = (a - bc) * T(0.5);
  const cx<T> O = (k == 0) ? D : cmul(D, fft::tw<T, L, true>(k));
  return cx<T>{E.re - O.im, E.im + O.re};
}

// X[k] of the forward real transform from Z[k] and Z[M - k] of the packed
// transform (0 < k < M): E + O w_L^k, E = (Z_k + conj Z_{M-k})/2,
// O = (Z_k - conj Z_{M-k}) / (2i).
template <typename T, int L>
__device__ __forceinline__ cx<T> fwd_split(cx<T> zk, cx<T> zm, int k) {
  const cx<T> zc = conj(zm);
  const cx<T> E = (zk + zc) * T(0.5);
  const cx<T> D = (zk - zc) * T(0.5);
  const cx<T> O = {D.im, -D.re};
  return E + cmul(O, fft::tw<T, L, false>(k));
}

template <typename T, int L, int N1, int N2, int MODE>
__global__ void __launch_bounds__(kSlabFThreads, 1) k_slab_f(Dev<T> d, T* __restrict__ Wout, int, int init) {
  constexpr int M = L / 2;
  static_assert(L % 2 == 0 && M == N1 * N2, "n3 = 2 N1 N2");
  constexpr int LP = slab_f_stride(L);
  extern __shared__ __align__(16) unsigned char smem[];
  const int i1 = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2, mw = d.mw;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (MODE == MODE_ITER && !init && converged(d)) return;
  if (d.n3 != L) {
    if (tid == 0) set_err(d.err, DEV_BAD_LAUNCH);
    return;
  }
  const SlabFLayout lay = slab_f_layout<T>(n2, L);
  uint32_t* msk = reinterpret_cast<uint32_t*>(smem + lay.msk);
  int* stw = reinterpret_cast<int*>(smem + lay.stw);
  T* wtab = reinterpret_cast<T*>(smem + lay.wtab);
  double* red = reinterpret_cast<double*>(smem + lay.red);
  T* buf = reinterpret_cast<T*>(smem + lay.buf);
  const cx<T>* zrow = d.Zt + (size_t)i1 * (M + 1) * n2;
  const cx<T>* rrow = d.Rt + (size_t)i1 * (M + 1) * n2;
  const T* Gi = d.G + (size_t)i1 * L * n2;
  const bool wsolve = (MODE == MODE_ITER) && !init && d.rho2 != T(0);
  const T zfac = init ? T(0) : ((d.rho2 == T(0)) ? T(1) / (T(1) + d.mu) : T(1));

  if (MODE != MODE_W)
    for (int j = tid; j < L * mw; j += nt) msk[j] = __ldg(d.mask + (size_t)i1 * L * mw + j);
  if (wsolve)
    for (int j = tid; j < 6 * n2; j += nt) wtab[j] = d.winv[j];

  // ---- A1: half spectrum -> packed sequence z (pairs k, M - k) -----------------------
  // Each item reads the pair (k, M - k) of one tube straight from the stored
  // half spectrum (coalesced along the tubes), kSlabFBatch items per thread with all
  // their loads in flight, and writes the split values to the tube's slots.
  {
    constexpr int U = kSlabFBatch;
    const int nitem = (M / 2 + 1) * n2;
    const cx<T>* src = (MODE == MODE_R) ? rrow : zrow;
    for (int e0 = tid; e0 < nitem; e0 += U * nt) {
      cx<T> a[U], b[U];
      int kk[U], tt[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nt;
        kk[u] = e / n2;
        tt[u] = e - kk[u] * n2;
        if (e < nitem) {
          const size_t ok = (size_t)kk[u] * n2 + tt[u], oc = (size_t)(M - kk[u]) * n2 + tt[u];
          if (MODE == MODE_W) {
            a[u] = ldg_cx(zrow + ok) + ldg_cx(rrow + ok);
            b[u] = ldg_cx(zrow + oc) + ldg_cx(rrow + oc);
          } else {
            a[u] = ldg_cx(src + ok);
            b[u] = ldg_cx(src + oc);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (e0 + u * nt >= nitem) break;
        const int k = kk[u], kc = M - k;
        T* tb = buf + (size_t)tt[u] * LP;
        cx<T> av = a[u], bv = b[u];
        if (k == 0) {  // DC and Nyquist slices are real
          av.im = T(0);
          bv.im = T(0);
        }
        st_slot(tb, k, inv_split<T, L>(av, bv, k));
        if (k != 0 && k != kc) st_slot(tb, kc, inv_split<T, L>(bv, av, kc));
      }
    }
  }
  __syncthreads();

  // ---- A2: inverse DFT_N1 over slots N2 n1 + q, twiddle w_M^{-q k1} ------------------------
  {
    ItemIter it(tid, n2);
    for (int e = tid; e < N2 * n2; e += nt, it.advance(nt, n2)) {
      const int q = it.g;
      T* tb = buf + (size_t)it.t * LP;
      cx<T> v[N1], o[N1];
#pragma unroll
      for (int j = 0; j < N1; ++j) v[j] = ld_slot(tb, N2 * j + q);
      fft::CFFT<T, N1, L, true>::run(v, 1, o);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const cx<T> x = (k1 == 0) ? o[0] : cmul(o[k1], fft::tw<T, L, true>(2 * q * k1));
        st_slot(tb, N2 * k1 + q, x);
      }
    }
  }
  __syncthreads();

  // ---- A3: inverse DFT_N2 over slots N2 k1 + j -> spatial values; v = G on the mask -------
  // (the G values of the next item are loaded while the current one is computed)
  const T scale = T(1) / T(M);
  double gsum = 0.0;  // MODE_GRAD: ||E||^2 partial
  {
    T gn[2 * N2];
    auto load_g = [&](int k1, int t) {
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int l = 2 * (k1 + N1 * k2);
        gn[2 * k2] = __ldg(Gi + (size_t)l * n2 + t);
        gn[2 * k2 + 1] = __ldg(Gi + (size_t)(l + 1) * n2 + t);
      }
    };
    ItemIter it(tid, n2);
    constexpr bool NEED_G = (MODE == MODE_ITER || MODE == MODE_GRAD);
    if (NEED_G && tid < N1 * n2) load_g(it.g, it.t);
    for (int e = tid; e < N1 * n2; e += nt) {
      const int k1 = it.g, t = it.t;
      it.advance(nt, n2);
      T* tb = buf + (size_t)t * LP + 2 * N2 * k1;
      T g[2 * N2];
      if (NEED_G) {
#pragma unroll
        for (int q = 0; q < 2 * N2; ++q) g[q] = gn[q];
        if (e + nt < N1 * n2) load_g(it.g, it.t);
      }
      cx<T> v[N2], o[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = ld_slot(tb, j);
      fft::CFFT<T, N2, L, true>::run(v, 1, o);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        T x0 = o[k2].re * scale, x1 = o[k2].im * scale;
        if (MODE == MODE_ITER) {
          const int l = 2 * (k1 + N1 * k2);
          const uint32_t w0 = msk[l * mw + (t >> 5)], w1 = msk[(l + 1) * mw + (t >> 5)];
          x0 = ((w0 >> (t & 31)) & 1u) ? g[2 * k2] : x0 * zfac;
          x1 = ((w1 >> (t & 31)) & 1u) ? g[2 * k2 + 1] : x1 * zfac;
        } else if (MODE == MODE_GRAD) {
          const int l = 2 * (k1 + N1 * k2);
          const uint32_t w0 = msk[l * mw + (t >> 5)], w1 = msk[(l + 1) * mw + (t >> 5)];
          x0 = ((w0 >> (t & 31)) & 1u) ? x0 - g[2 * k2] : T(0);
          x1 = ((w1 >> (t & 31)) & 1u) ? x1 - g[2 * k2 + 1] : T(0);
          gsum += (double)x0 * (double)x0 + (double)x1 * (double)x1;
        }
        st_slot(tb, k2, cx<T>{x0, x1});
      }
    }
  }
  __syncthreads();

  // ---- partial sums of the read-back modes ----------------------------------------------
  if (MODE == MODE_W || MODE == MODE_R) {
    double a = 0.0, b = 0.0;
    for (int e = tid; e < L * n2; e += nt) {
      const int l = e / n2, t = e - l * n2;
      const int off = slab_f_off<N1, N2>(l);
      const T v = buf[(size_t)t * LP + off];
      a += (double)v * (double)v;
      if (MODE == MODE_W) {
        if (t + 1 < n2) {
          const double dv = (double)v - (double)buf[(size_t)(t + 1) * LP + off];
          b += dv * dv;
        }
        if (Wout) Wout[(size_t)i1 + (size_t)n1 * ((size_t)t + (size_t)n2 * l)] = v;
      } else {
        if ((msk[l * mw + (t >> 5)] >> (t & 31)) & 1u) b += (double)v * (double)v;
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

  // ---- W-step (rows split into segments of mask words) ---------------------------------------
  if (wsolve) {
    // rows split into nseg segments so that every thread has one (row, segment)
    const int nseg = max(1, nt / L);
    auto col_of = [&](int l) { return buf + slab_f_off<N1, N2>(l); };
    wstep_sweeps_seg<T>(col_of, LP, msk, stw, L, nseg, tid, n2, d.rho2, wtab);
  }

  // ---- C1: forward DFT_N2 over slots N2 k1 + j, twiddle w_M^{k1 q} -----------------------
  {
    ItemIter it(tid, n2);
    for (int e = tid; e < N1 * n2; e += nt, it.advance(nt, n2)) {
      const int k1 = it.g;
      T* tb = buf + (size_t)it.t * LP + 2 * N2 * k1;
      cx<T> v[N2], o[N2];
#pragma unroll
      for (int j = 0; j < N2; ++j) v[j] = ld_slot(tb, j);
      fft::CFFT<T, N2, L, false>::run(v, 1, o);
#pragma unroll
      for (int q = 0; q < N2; ++q) {
        const cx<T> x = (q == 0) ? o[0] : cmul(o[q], fft::tw<T, L, false>(2 * k1 * q));
        st_slot(tb, q, x);
      }
    }
  }
  __syncthreads();

  // ---- C2: forward DFT_N1 over slots N2 k1 + q -> natural order -----------------------------
  {
    ItemIter it(tid, n2);
    for (int e = tid; e < N2 * n2; e += nt, it.advance(nt, n2)) {
      const int q = it.g;
      T* tb = buf + (size_t)it.t * LP;
      cx<T> v[N1], o[N1];
#pragma unroll
      for (int j = 0; j < N1; ++j) v[j] = ld_slot(tb, N2 * j + q);
      fft::CFFT<T, N1, L, false>::run(v, 1, o);
#pragma unroll
      for (int j = 0; j < N1; ++j) st_slot(tb, N2 * j + q, o[j]);
    }
  }
  __syncthreads();

  // ---- C3: split to the half spectrum; R~ = W~ - Z~ ------------------------------------------
  cx<T>* rt = d.Rt + (size_t)i1 * (M + 1) * n2;
  const bool track = (MODE == MODE_ITER) && !init && d.dZt != nullptr;
  const cx<T>* dz = track ? d.dZt + (size_t)i1 * (M + 1) * n2 : nullptr;
  double dw2 = 0.0;
  {
    ItemIter it(tid, n2);
    for (int e = tid; e < (M / 2 + 1) * n2; e += nt, it.advance(nt, n2)) {
      const int k = it.g, t = it.t;
      const int kc = M - k;
      const T* tb = buf + (size_t)t * LP;
      const size_t ok = (size_t)k * n2 + t, oc = (size_t)kc * n2 + t;
      const cx<T> zk0 = (MODE == MODE_GRAD) ? cx<T>{T(0), T(0)} : ldg_cx(zrow + ok);
      const cx<T> zc0 = (MODE == MODE_GRAD) ? cx<T>{T(0), T(0)} : ldg_cx(zrow + oc);
      cx<T> rk, rc;
      if (k == 0) {
        const cx<T> z0 = ld_slot(tb, 0);
        rk = cx<T>{z0.re + z0.im - zk0.re, T(0)};
        rc = cx<T>{z0.re - z0.im - zc0.re, T(0)};
      } else {
        const cx<T> zk = ld_slot(tb, k), zm = ld_slot(tb, kc);
        rk = fwd_split<T, L>(zk, zm, k) - zk0;
        rc = fwd_split<T, L>(zm, zk, kc) - zc0;
      }
      if (track) {
        dw2 += dw_term(rk, rt[ok], dz[ok], k, L);
        if (k != kc) dw2 += dw_term(rc, rt[oc], dz[oc], kc, L);
      }
      rt[ok] = rk;
      if (k != kc) rt[oc] = rc;
    }
  }
  if (track) {
    double unused = 0.0;
    block_sum2(dw2, unused, red);
    if (tid == 0) d.part_dw[i1] = dw2;
  }
  if (MODE == MODE_GRAD) {
    double unused = 0.0;
    block_sum2(gsum, unused, red);
    if (tid == 0) d.part[(size_t)i1 * 4] = gsum;
  }
}

}  // namespace tc
