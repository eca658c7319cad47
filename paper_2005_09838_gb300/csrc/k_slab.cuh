// Slab kernel of the TCTF2R iteration: one CTA per mode-1 index i1 (one OD
// pair).  The spatial slab (i1, :, :) lives in shared memory, tube-major with
// an odd stride (conflict-free for tube-per-thread and row-per-thread access).
//
//   phase A  inverse mode-3 DFT (Eq. (barAAk)) of every tube of Z~ = X~Y~
//            (step 3; the half spectrum is written by the Y-step kernel);
//            the slab receives v = G on the mask and Z elsewhere
//   phase B  W-step of every row (i1, :, i3) (step 4, Eq. (subquKKT))
//   phase C  forward mode-3 DFT of every tube of W (step 7, Eq. (bar BA-k));
//            the residual spectrum R~ = W~ - Z~ is stored
#pragma once

namespace tc {

enum SlabMode : int { MODE_ITER = 0, MODE_W = 1, MODE_R = 2, MODE_GRAD = 3 };

// Threads per CTA: the register transforms and the W-step sweeps need the
// 255-register budget of two warps per scheduler (nine warps would put three
// on one scheduler and cap a thread at 168 registers); tubes beyond the thread
// count loop.
__host__ __device__ constexpr int slab_max_threads(int) { return 256; }
// Rows (inverse) or slices (forward) per item of the generic transform, by
// default; the engine picks among 2, 4 and 8 by timing (slab_tile_candidates).
constexpr int kTL = 4;

// Odd stride between tubes in the slab (n3 values per tube).
__host__ __device__ inline int slab_stride(int n3) { return n3 | 1; }

struct SlabLayout {
  size_t wtab, red, msk, stw, tw, spec, spat, total;  // byte offsets and total shared bytes
  size_t slab_bytes;                         // bytes of the slab buffers per CTA
};

template <typename T>
__host__ __device__ inline SlabLayout slab_layout(int n2, int n3, bool specialised, bool slabs_in_smem) {
  SlabLayout L{};
  const int S = n3 / 2 + 1;
  size_t off = 0;
  L.wtab = off;
  off = align_up(off + sizeof(T) * 6 * n2, 16);
  L.red = off;
  off = align_up(off + sizeof(double) * 4 * 32, 16);
  L.msk = off;  // row-major mask bits: [n3][ceil(n2/32)]
  off = align_up(off + sizeof(uint32_t) * (size_t)n3 * ((n2 + 31) / 32), 16);
  L.stw = off;  // per row and mask word: start of the run of missing entries entering the word
  off = align_up(off + sizeof(int) * (size_t)n3 * ((n2 + 31) / 32), 16);
  L.tw = off;  // generic transform: the n3 twiddles exp(-2 pi i m / n3)
  if (!specialised) off = align_up(off + sizeof(cx<T>) * (size_t)n3, 16);
  const size_t spec_bytes = specialised ? 0 : align_up(sizeof(cx<T>) * (size_t)S * n2, 16);
  const size_t spat_bytes = align_up(sizeof(T) * (size_t)n2 * slab_stride(n3), 16);
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
// W-step of one row (i1, :, i3) (Eq. (subquKKT), Eq. (Wkiom)).
//
// For a missing j, (W K_{mu rho2})_j = Z_j with K_{mu rho2} = (1+mu) I +
// rho2 K^T K (tridiagonal); W_j = G_j on the mask (identity rows).  On entry
// the row holds v_j = G_j on the mask and Z_j elsewhere; the observed
// neighbours of a missing entry enter through the elimination itself.  The
// LU pivots of a run of missing entries depend only on the position p in the
// run, on whether the run starts at j = 0 and on whether j is the last entry
// of the row (the first and last entries have one neighbour), so their
// inverses come from a table and each sweep is a single fused multiply-add
// chain:
//   forward   d_j = a_j d_{j-1} + b_j,   a_j = rho2 inv_j,  b_j = v_j inv_j
//   backward  w_j = c_j w_{j+1} + d_j,   c_j = rho2 inv_j (0 at j = n2-1)
// with a_j = c_j = 0, b_j = v_j at observed entries.  On return the row
// holds W.  row[j] is at col[j * LP].  The row is processed one mask word
// (32 entries) at a time: the entries are read into registers first and the
// table indices come from the mask bits, so only the multiply-add chain stays
// on the critical path.  The run start entering each word is saved by the
// forward sweep for the backward one.
//
// wtab: [6][n2] inv1, inv0 (runs starting at j = 0 / j > 0), c1 = rho2 inv1,
//       c0 = rho2 inv0, e1, e0 (inverse pivot when the run ends at j = n2-1)
// rowm: the row's mask bits along j (word j / 32, bit j % 32)
// rowst: per-word run starts (written here)
// ---------------------------------------------------------------------------
// Fills the [6][n2] W-step table of wstep_sweeps in FP64, rounded to T.
// Pivots of a run of missing entries by position p: the first has diagonal
// 1 + mu + rho2 (run at j = 0, one neighbour) or 1 + mu + 2 rho2; each later
// one subtracts rho2^2 times the previous inverse pivot; at j = n2 - 1 the
// diagonal loses one rho2 (one neighbour).
template <typename T>
__host__ __device__ inline void wstep_tables(T* w, int n2, double mu, double rho2) {
  const double first[2] = {1.0 + mu + rho2 * (n2 > 1 ? 1.0 : 0.0), 1.0 + mu + 2.0 * rho2};
  const double last[2] = {first[0], 1.0 + mu + rho2};
  for (int b = 0; b < 2; ++b) {  // b = 0: run starting at j = 0; b = 1: j > 0
    double prev = 0.0;
    for (int q = 0; q < n2; ++q) {
      const double sub = (q > 0) ? rho2 * rho2 * prev : 0.0;
      const double inv = 1.0 / (((q > 0) ? 1.0 + mu + 2.0 * rho2 : first[b]) - sub);
      const double inv_last = 1.0 / (last[b] - sub);
      w[(size_t)b * n2 + q] = (T)inv;
      w[(size_t)(2 + b) * n2 + q] = (T)(rho2 * inv);
      w[(size_t)(4 + b) * n2 + q] = (T)inv_last;
      prev = inv;
    }
  }
}

// One mask word (32 entries, fewer in the last word) of the forward sweep.
// The table index of entry j is inv-table + (j - rs), rs the start of the run
// holding j: from the mask bits below j (rs = 32 w + 32 - clz(below)) or,
// when there are none in this word, the run start st_w entering the word, so
// every index is known without the recurrence; the recurrence itself is one
// fused multiply-add per entry (a_j = 0, b_j = v_j at observed entries).
// LAST: the word holds j = n2 - 1 (the e-table pivot there).
template <typename T, bool FULL, bool LAST>
__device__ __forceinline__ void wstep_fwd_word(T* __restrict__ col, int LP, uint32_t mw, int w, int qn, int st_w,
                                               int n2, T rho2, const T* __restrict__ wtab, T& d) {
  const int base = 32 * w;
  const int cw = ((st_w == 0) ? 0 : n2) + base - st_w;  // index base of entries without bits below
  T v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q)
    if (FULL || q < qn) v[q] = col[(base + q) * LP];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (FULL || q < qn) {
      const bool ob = (mw >> q) & 1u;
      const uint32_t below = mw & ((1u << q) - 1u);
      int idx = below ? (n2 - 32 + q + __clz(below)) : (cw + q);
      if (LAST && base + q == n2 - 1) idx += 4 * n2;
      const T inv = wtab[idx];
      d = fma(ob ? T(0) : rho2 * inv, d, ob ? v[q] : v[q] * inv);
      v[q] = d;
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q)
    if (FULL || q < qn) col[(base + q) * LP] = v[q];
}

// One mask word of the backward sweep: c_j = rho2 inv_j at table index
// 2 n2 + (forward index), 0 at observed entries and at j = n2 - 1 (observed
// slots already hold G).
template <typename T, bool FULL, bool LAST>
__device__ __forceinline__ void wstep_bwd_word(T* __restrict__ col, int LP, uint32_t mw, int w, int qn, int st_w,
                                               int n2, const T* __restrict__ wtab, T& wn) {
  const int base = 32 * w;
  const int cw = ((st_w == 0) ? 2 * n2 : 3 * n2) + base - st_w;
  T v[32];
#pragma unroll
  for (int q = 0; q < 32; ++q)
    if (FULL || q < qn) v[q] = col[(base + q) * LP];
#pragma unroll
  for (int q = 31; q >= 0; --q) {
    if (FULL || q < qn) {
      const bool ob = (mw >> q) & 1u;
      const uint32_t below = mw & ((1u << q) - 1u);
      const int idx = below ? (3 * n2 - 32 + q + __clz(below)) : (cw + q);
      const T c = wtab[idx];
      const bool zero = ob || (LAST && base + q == n2 - 1);
      wn = fma(zero ? T(0) : c, wn, v[q]);
      v[q] = wn;
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q)
    if (FULL || q < qn) col[(base + q) * LP] = v[q];
}

template <typename T>
__device__ void wstep_sweeps(T* __restrict__ col, int LP, const uint32_t* __restrict__ rowm, int* __restrict__ rowst,
                             int n2, T rho2, const T* __restrict__ wtab) {
  const int words = (n2 + 31) >> 5;
  const int ql = n2 - 32 * (words - 1);  // entries in the last word
  // ---- forward: d_j = a_j d_{j-1} + b_j --------------------------------------
  T d = T(0);
  int st = 0;  // start of the run of missing entries entering the word
  for (int w = 0; w < words - 1; ++w) {
    const uint32_t mw = rowm[w];
    rowst[w] = st;
    wstep_fwd_word<T, true, false>(col, LP, mw, w, 32, st, n2, rho2, wtab, d);
    if (mw) st = 32 * w + 32 - __clz(mw);
  }
  {
    const int w = words - 1;
    rowst[w] = st;
    if (ql == 32) wstep_fwd_word<T, true, true>(col, LP, rowm[w], w, 32, st, n2, rho2, wtab, d);
    else wstep_fwd_word<T, false, true>(col, LP, rowm[w], w, ql, st, n2, rho2, wtab, d);
  }
  // ---- backward: w_j = c_j w_{j+1} + d_j ---------------------------------------
  T wn = T(0);
  {
    const int w = words - 1;
    if (ql == 32) wstep_bwd_word<T, true, true>(col, LP, rowm[w], w, 32, rowst[w], n2, wtab, wn);
    else wstep_bwd_word<T, false, true>(col, LP, rowm[w], w, ql, rowst[w], n2, wtab, wn);
  }
  for (int w = words - 2; w >= 0; --w)
    wstep_bwd_word<T, true, false>(col, LP, rowm[w], w, 32, rowst[w], n2, wtab, wn);
}

// ---------------------------------------------------------------------------
// The same W-step with each row split into nseg segments of whole mask words,
// one thread per (row, segment): a block-wide call that takes three barriers.
// Both recurrences restart at every observed entry (there a_j = 0 and c_j = 0:
// the value is G), and the backward one also at j = n2 - 1.  So the value
// entering a segment follows from the entries between the last restart and
// the segment boundary, and each thread recomputes it with the very operations
// the sequential sweep would apply (results are bit-identical to
// wstep_sweeps): forward, from the last observed entry before the segment (or
// j = 0); backward, from the first observed entry at or after the segment's
// end (or j = n2 - 1).  The carries are formed before the values they read
// are overwritten.
//   item: this thread's (row, segment) index, row = item % nrows, segment =
//         item / nrows; items >= nrows * nseg only join the barriers
//   col(l): the row's first entry; rows are strided by LP along j
// ---------------------------------------------------------------------------
template <typename T, typename ColFn>
__device__ void wstep_sweeps_seg(ColFn col_of, int LP, const uint32_t* __restrict__ msk, int* __restrict__ stw,
                                 int nrows, int nseg, int item, int n2, T rho2, const T* __restrict__ wtab) {
  const int words = (n2 + 31) >> 5;
  const int ql = n2 - 32 * (words - 1);  // entries in the last word
  const int wps = (words + nseg - 1) / nseg;
  const bool active = item < nrows * nseg;
  const int l = active ? item % nrows : 0, sg = active ? item / nrows : 0;
  const int w0 = min(sg * wps, words), w1 = min(w0 + wps, words);
  const bool work = active && w0 < w1;
  T* col = col_of(l);
  const uint32_t* rowm = msk + (size_t)l * ((n2 + 31) >> 5);
  int* rowst = stw + (size_t)l * ((n2 + 31) >> 5);
  auto bit = [&](int j) { return (rowm[j >> 5] >> (j & 31)) & 1u; };

  // ---- forward carry: d_{j0 - 1} and the run start entering word w0 -------------------
  T d = T(0);
  int st = 0;
  if (work && w0 > 0) {
    for (int w = w0 - 1; w >= 0; --w) {
      const uint32_t mw = rowm[w];
      if (mw) {
        st = 32 * w + 32 - __clz(mw);
        break;
      }
    }
    const int j0 = 32 * w0;
    if (st > 0) d = col[(size_t)(st - 1) * LP];  // observed: the recurrence restarts at G
    for (int j = st; j < j0; ++j) {             // the run of missing entries up to the boundary
      const T inv = wtab[((st == 0) ? 0 : n2) + (j - st)];
      d = fma(rho2 * inv, d, col[(size_t)j * LP] * inv);
    }
  }
  __syncthreads();
  // ---- forward sweep of the segment -----------------------------------------------------
  if (work) {
    for (int w = w0; w < w1; ++w) {
      const uint32_t mw = rowm[w];
      rowst[w] = st;
      if (w < words - 1) wstep_fwd_word<T, true, false>(col, LP, mw, w, 32, st, n2, rho2, wtab, d);
      else if (ql == 32) wstep_fwd_word<T, true, true>(col, LP, mw, w, 32, st, n2, rho2, wtab, d);
      else wstep_fwd_word<T, false, true>(col, LP, mw, w, ql, st, n2, rho2, wtab, d);
      if (mw) st = 32 * w + 32 - __clz(mw);
    }
  }
  __syncthreads();
  // ---- backward carry: w_{j1}, j1 = 32 w1, from the first restart at or after it --------
  T wn = T(0);
  if (work && w1 < words) {
    const int j1 = 32 * w1;
    int k = j1;
    while (k < n2 - 1 && !bit(k)) ++k;
    wn = col[(size_t)k * LP];  // w_k = d_k at a restart
    for (int j = k - 1; j >= j1; --j) {
      const int w = j >> 5, q = j & 31;
      const uint32_t below = rowm[w] & ((1u << q) - 1u);
      const int rs = below ? 32 * w + 32 - __clz(below) : rowst[w];
      const T c = wtab[2 * n2 + ((rs == 0) ? 0 : n2) + (j - rs)];
      wn = fma(c, wn, col[(size_t)j * LP]);
    }
  }
  __syncthreads();
  // ---- backward sweep of the segment ----------------------------------------------------
  if (work) {
    for (int w = w1 - 1; w >= w0; --w) {
      if (w < words - 1) wstep_bwd_word<T, true, false>(col, LP, rowm[w], w, 32, rowst[w], n2, wtab, wn);
      else if (ql == 32) wstep_bwd_word<T, true, true>(col, LP, rowm[w], w, 32, rowst[w], n2, wtab, wn);
      else wstep_bwd_word<T, false, true>(col, LP, rowm[w], w, ql, rowst[w], n2, wtab, wn);
    }
  }
  __syncthreads();
}

// Weighted |W~^{l+1} - W~^l|^2 of one half-spectrum entry: W~ = Z~ + R~, so the
// change is (R~new - R~old) + (Z~new - Z~old); weight 1 for the real slices
// (k = 0 and, for even n3, k = n3/2), 2 for the others (their mirror).
template <typename T>
__device__ __forceinline__ double dw_term(cx<T> rnew, cx<T> rold, cx<T> dz, int k, int n3) {
  const double a = (double)rnew.re - (double)rold.re + (double)dz.re;
  const double b = (double)rnew.im - (double)rold.im + (double)dz.im;
  return ((k == 0 || 2 * k == n3) ? 1.0 : 2.0) * (a * a + b * b);
}

// ---------------------------------------------------------------------------
// MODE_ITER: phases A, B, C (init != 0: W = P_Omega(G), the initial point, in
//            place of the W-step).
// MODE_W   : W = iDFT(Z~ + R~); optional copy to Wout (column-major), partial
//            sums ||W||^2 and ||K unfold(W,2)||^2.
// MODE_R   : R = iDFT(R~); partial sums ||R||^2 and ||P_Omega R||^2.
// Layouts used here: G row-major [i1][n3][n2] and mask words row-major
// [i1][n3][ceil(n2/32)] (written by k_pack), copied to shared memory.
// ---------------------------------------------------------------------------
// TL: rows (inverse) or slices (forward) per item of the generic transform
// (L = 0); every TL gives the same sums in the same order.
template <typename T, int L, int MODE, int TL = kTL>
__global__ void __launch_bounds__(slab_max_threads(L), 1)
    k_slab(Dev<T> d, T* __restrict__ Wout, int slabs_in_smem, int init) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int i1 = blockIdx.x;
  const int n1 = d.n1, n2 = d.n2;
  const int n3 = (L > 0) ? L : d.n3;
  const int S = n3 / 2 + 1;
  const int LP = slab_stride(n3);
  const int tid = threadIdx.x, nt = blockDim.x;
  if (MODE == MODE_ITER && !init && converged(d)) return;
  if (L > 0 && d.n3 != L) {
    if (tid == 0) set_err(d.err, DEV_BAD_LAUNCH);
    return;
  }
  const SlabLayout lay = slab_layout<T>(n2, n3, L > 0, slabs_in_smem != 0);
  T* wtab = reinterpret_cast<T*>(smem + lay.wtab);
  double* red = reinterpret_cast<double*>(smem + lay.red);
  uint32_t* msk = reinterpret_cast<uint32_t*>(smem + lay.msk);
  int* stw = reinterpret_cast<int*>(smem + lay.stw);
  unsigned char* slab_base =
      slabs_in_smem ? smem : reinterpret_cast<unsigned char*>(d.scratch) + (size_t)i1 * lay.slab_bytes;
  cx<T>* spec = reinterpret_cast<cx<T>*>(slab_base + lay.spec);
  T* spat = reinterpret_cast<T*>(slab_base + lay.spat);
  const cx<T>* zrow = d.Zt + (size_t)i1 * S * n2;
  const cx<T>* rrow = d.Rt + (size_t)i1 * S * n2;
  const T* Gi = d.G + (size_t)i1 * n2 * n3;
  const int mwords = d.mw;
  const uint32_t* Mi = d.mask + (size_t)i1 * n3 * mwords;
  const bool wsolve = (MODE == MODE_ITER) && !init && d.rho2 != T(0);
  const T zfac = init ? T(0) : ((d.rho2 == T(0)) ? T(1) / (T(1) + d.mu) : T(1));

  if (wsolve)
    for (int j = tid; j < 6 * n2; j += nt) wtab[j] = d.winv[j];
  if (MODE != MODE_W) {
    for (int j = tid; j < n3 * mwords; j += nt) msk[j] = __ldg(Mi + j);
    __syncthreads();
  }

  // ---- phase A: inverse transform of each tube; v = G on the mask ------------
  // (MODE_GRAD: v = Z - G on the mask, 0 elsewhere; gsum = ||v||^2)
  double gsum = 0.0;
  if constexpr (L > 0) {
    constexpr int SL = L / 2 + 1;
    if (MODE == MODE_ITER || MODE == MODE_GRAD) {
      // G (row-major, read coalesced) is staged into the slab, transposed to the
      // tube-major layout, with asynchronous copies issued ahead of the transforms;
      // each tube then picks its observed values from its own column.
      int l = tid / n2, t = tid - (tid / n2) * n2;
      if (slabs_in_smem) {
        for (int e = tid; e < n3 * n2; e += nt) {
          cp_async_elem(spat + t * LP + l, Gi + e);
          t += nt;
          while (t >= n2) {
            t -= n2;
            ++l;
          }
        }
        cp_async_wait_all();
      } else {
        for (int e = tid; e < n3 * n2; e += nt) {
          spat[(size_t)t * LP + l] = __ldg(Gi + e);
          t += nt;
          while (t >= n2) {
            t -= n2;
            ++l;
          }
        }
      }
      __syncthreads();
    }
    for (int t0 = 0; t0 < n2; t0 += nt) {
      const int t = t0 + tid;
      if (t0 + (tid & ~31) >= n2) continue;  // whole warp past the last column (warp-uniform)
      const bool act = t < n2;
      cx<T> X[SL];
#pragma unroll
      for (int k = 0; k < SL; ++k) {
        const size_t o = (size_t)k * n2 + (act ? t : 0);
        if (MODE == MODE_ITER || MODE == MODE_GRAD) X[k] = ldg_cx(zrow + o);
        else if (MODE == MODE_W) X[k] = ldg_cx(zrow + o) + ldg_cx(rrow + o);
        else X[k] = ldg_cx(rrow + o);
      }
      T x[L];
      fft::irfft<T, L>(X, x);
      if (MODE == MODE_ITER) {
        const int ta = act ? t : 0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const bool ob = act && ((msk[l * mwords + (ta >> 5)] >> (ta & 31)) & 1u);
          x[l] = ob ? spat[(size_t)ta * LP + l] : x[l] * zfac;
        }
      } else if (MODE == MODE_GRAD) {
        const int ta = act ? t : 0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const bool ob = act && ((msk[l * mwords + (ta >> 5)] >> (ta & 31)) & 1u);
          x[l] = ob ? x[l] - spat[(size_t)ta * LP + l] : T(0);
          gsum += (double)x[l] * (double)x[l];
        }
      }
      if (act) {
#pragma unroll
        for (int l = 0; l < L; ++l) spat[t * LP + l] = x[l];
      }
    }
  } else {
    // the half spectrum of the slab ([k][n2], as stored) and the twiddles
    cx<T>* tw = reinterpret_cast<cx<T>*>(smem + lay.tw);
    for (int m = tid; m < n3; m += nt) tw[m] = d.twg[m];
    for (int e = tid; e < S * n2; e += nt) {
      cx<T> v;
      if (MODE == MODE_ITER || MODE == MODE_GRAD) v = zrow[e];
      else if (MODE == MODE_W) v = zrow[e] + rrow[e];
      else v = rrow[e];
      spec[e] = v;
    }
    __syncthreads();
    // Eq. (barAAk) for any n3, as a product of the spectrum with the DFT matrix:
    // x_l = (1/n3) (X_0 + 2 sum_{k=1}^{kmax} Re(X_k conj(w_{kl})) [+ (-1)^l X_{n3/2}]),
    // w_m = exp(-2 pi i m / n3), for items of one tube and TL consecutive rows l,
    // tube index fastest (a warp reads one slice of 32 tubes and shares the
    // twiddles)
    const bool even = (n3 % 2) == 0;
    const int kmax = even ? S - 2 : S - 1;
    const T inv = T(1) / T(n3);
    const int nlb = (n3 + TL - 1) / TL;
    for (int e = tid; e < nlb * n2; e += nt) {
      const int lb = e / n2, t = e - lb * n2, l0 = lb * TL;
      T acc[TL];
      const T s0 = spec[t].re;
#pragma unroll
      for (int j = 0; j < TL; ++j) acc[j] = s0;
      int base = 0;  // k l0 mod n3
      for (int k = 1; k <= kmax; ++k) {
        base += l0;
        if (base >= n3) base -= n3;
        const cx<T> v = spec[(size_t)k * n2 + t];
        int idx = base;  // k (l0 + j) mod n3
#pragma unroll
        for (int j = 0; j < TL; ++j) {
          const cx<T> w = tw[idx];
          acc[j] += T(2) * (v.re * w.re + v.im * w.im);
          idx += k;
          if (idx >= n3) idx -= n3;
        }
      }
      const T sn = even ? spec[(size_t)(S - 1) * n2 + t].re : T(0);
      T* col = spat + (size_t)t * LP;
#pragma unroll
      for (int j = 0; j < TL; ++j) {
        const int l = l0 + j;
        if (l >= n3) break;
        T a = acc[j];
        if (even) a += (l & 1) ? -sn : sn;
        T x = a * inv;
        if (MODE == MODE_ITER) {
          const bool ob = (msk[l * mwords + (t >> 5)] >> (t & 31)) & 1u;
          x = ob ? __ldg(Gi + (size_t)l * n2 + t) : x * zfac;
        } else if (MODE == MODE_GRAD) {
          const bool ob = (msk[l * mwords + (t >> 5)] >> (t & 31)) & 1u;
          x = ob ? x - __ldg(Gi + (size_t)l * n2 + t) : T(0);
          gsum += (double)x * (double)x;
        }
        col[l] = x;
      }
    }
  }
  __syncthreads();

  // ---- phase B: rows ------------------------------------------------------
  if (MODE == MODE_W || MODE == MODE_R) {
    double a = 0.0, b = 0.0;
    for (int e = tid; e < n2 * n3; e += nt) {
      const int j = e / n3, l = e - j * n3;
      const T v = spat[j * LP + l];
      a += (double)v * (double)v;
      if (MODE == MODE_W) {
        if (j + 1 < n2) {
          const double dv = (double)v - (double)spat[(j + 1) * LP + l];
          b += dv * dv;
        }
        if (Wout) Wout[(size_t)i1 + (size_t)n1 * ((size_t)j + (size_t)n2 * l)] = v;
      } else {
        if ((msk[l * mwords + (j >> 5)] >> (j & 31)) & 1u) b += (double)v * (double)v;
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
  if (wsolve) {
    for (int l = tid; l < n3; l += nt)
      wstep_sweeps<T>(spat + l, LP, msk + l * mwords, stw + l * mwords, n2, d.rho2, wtab);
    __syncthreads();
  }

  // ---- phase C: forward transform, R~ = W~ - Z~ ------------------------------
  const bool track = (MODE == MODE_ITER) && !init && d.dZt != nullptr;
  double dw2 = 0.0;
  if constexpr (L > 0) {
    constexpr int SL = L / 2 + 1;
    for (int t = tid; t < n2; t += nt) {
      T x[L];
#pragma unroll
      for (int l = 0; l < L; ++l) x[l] = spat[t * LP + l];
      cx<T> X[SL];
      fft::rfft<T, L>(x, X);
      cx<T>* rt = d.Rt + (size_t)i1 * SL * n2 + t;
      const cx<T>* zt = zrow + t;
#pragma unroll
      for (int k = 0; k < SL; ++k) {
        const cx<T> rn = (MODE == MODE_GRAD) ? X[k] : X[k] - ldg_cx(zt + (size_t)k * n2);
        if (track) dw2 += dw_term(rn, rt[(size_t)k * n2], d.dZt[(size_t)i1 * SL * n2 + (size_t)k * n2 + t], k, L);
        rt[(size_t)k * n2] = rn;
      }
    }
  } else {
    // Eq. (bar BA-k) for any n3, as a product of the slab with the DFT matrix:
    // X_k = sum_l x_l w_{kl} for k < S, for items of one tube and TL consecutive
    // slices k, tube index fastest
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(smem + lay.tw);
    const int nkb = (S + TL - 1) / TL;
    for (int e = tid; e < nkb * n2; e += nt) {
      const int kb = e / n2, t = e - kb * n2, k0 = kb * TL;
      cx<T> acc[TL];
#pragma unroll
      for (int j = 0; j < TL; ++j) acc[j] = cx<T>{T(0), T(0)};
      int idx[TL], inc[TL];  // (k0 + j) l mod n3, advanced by (k0 + j) mod n3 (< n3)
#pragma unroll
      for (int j = 0; j < TL; ++j) {
        idx[j] = 0;
        inc[j] = (k0 + j) % n3;
      }
      const T* col = spat + (size_t)t * LP;
      for (int l = 0; l < n3; ++l) {
        const T x = col[l];
#pragma unroll
        for (int j = 0; j < TL; ++j) {
          const cx<T> w = tw[idx[j]];
          acc[j].re += x * w.re;
          acc[j].im += x * w.im;
          idx[j] += inc[j];
          if (idx[j] >= n3) idx[j] -= n3;
        }
      }
      const size_t o = (size_t)i1 * S * n2 + t;
#pragma unroll
      for (int j = 0; j < TL; ++j) {
        const int k = k0 + j;
        if (k >= S) break;
        cx<T> a = acc[j];
        if (k == 0 || (2 * k == n3)) a.im = T(0);
        const size_t ok = o + (size_t)k * n2;
        const cx<T> rn = (MODE == MODE_GRAD) ? a : a - zrow[(size_t)k * n2 + t];
        if (track) dw2 += dw_term(rn, d.Rt[ok], d.dZt[ok], k, n3);
        d.Rt[ok] = rn;
      }
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
