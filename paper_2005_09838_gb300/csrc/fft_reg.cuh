// Register-resident mode-3 DFTs of one tube per thread.
//
// The t-product algebra of Sec. 2.2 needs, for every tube (i1, i2, :), the
// forward transform of Eq. (bar BA-k) restricted to the floor(n3/2)+1 slices
// that are solved, and the inverse of Eq. (barAAk) from that half spectrum
// (conjugate symmetry, Eq. (rcm_3-k+2)).  Here the transform is computed by a
// mixed-radix decimation-in-time FFT whose length is a compile-time constant,
// fully unrolled so that the tube lives in registers.
//
// Sign convention: the forward transform uses w = exp(-2 pi i / n3).  The paper
// writes omega = exp(+2 pi i / n3); every slice of one convention is the
// complex conjugate of the other, the slice updates commute with conjugation
// (all operators H, K are real), so every real quantity is unchanged.
//
// Real-input trick for even n3 = 2M: the even/odd samples are packed into one
// complex sequence of length M, transformed, and split with the twiddles
// w_n3^k.  Odd n3 runs a complex transform of length n3.
#pragma once

#include "tc_common.cuh"

namespace tc {
namespace fft {

// Tube lengths with a specialised register kernel, and the offsets of their
// twiddle tables in the concatenated table.
constexpr int kLengths[] = {7, 112, 168};
constexpr int kNumLengths = sizeof(kLengths) / sizeof(int);

__host__ __device__ constexpr int table_offset(int L) {
  return L == 7 ? 0 : L == 112 ? 7 : L == 168 ? 7 + 112 : -1;
}
constexpr int kTableSize = 7 + 112 + 168;

__host__ __device__ constexpr bool supported(int L) { return table_offset(L) >= 0; }

constexpr int pick_radix(int N) {
  return (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2 : (N % 3 == 0) ? 3 : (N % 5 == 0) ? 5 : (N % 7 == 0) ? 7 : N;
}

// Twiddle tables w_L^m = exp(-2 pi i m / L), m < L, for every specialised L,
// concatenated.  Filled from the host (FP64 cos/sin) by upload_twiddles().
static __constant__ cx<float> c_tw_f32[kTableSize];
static __constant__ cx<double> c_tw_f64[kTableSize];

template <typename T>
__device__ __forceinline__ cx<T> tw_entry(int i);
template <>
__device__ __forceinline__ cx<float> tw_entry<float>(int i) { return c_tw_f32[i]; }
template <>
__device__ __forceinline__ cx<double> tw_entry<double>(int i) { return c_tw_f64[i]; }

// w_L^m (forward); conjugated for the inverse.
template <typename T, int L, bool INV>
__device__ __forceinline__ cx<T> tw(int m) {
  constexpr int off = table_offset(L);
  static_assert(off >= 0, "no twiddle table for this length");
  const cx<T> v = tw_entry<T>(off + (m % L));
  return INV ? cx<T>{v.re, -v.im} : v;
}

// Radix-P DFT of P values x[q*xs], q < P, written to o[k*os].
// TOP is the length of the twiddle table in use (P divides TOP).
template <typename T, int P, int TOP, bool INV>
__device__ __forceinline__ void small_dft(const cx<T>* x, int xs, cx<T>* o, int os) {
  if constexpr (P == 1) {
    o[0] = x[0];
  } else if constexpr (P == 2) {
    const cx<T> a = x[0], b = x[xs];
    o[0] = a + b;
    o[os] = a - b;
  } else if constexpr (P == 4) {
    const cx<T> a = x[0], b = x[xs], c = x[2 * xs], d = x[3 * xs];
    const cx<T> s0 = a + c, d0 = a - c, s1 = b + d, d1 = b - d;
    // forward: multiply d1 by -i; inverse: by +i
    const cx<T> jd1 = INV ? cx<T>{-d1.im, d1.re} : cx<T>{d1.im, -d1.re};
    o[0] = s0 + s1;
    o[os] = d0 + jd1;
    o[2 * os] = s0 - s1;
    o[3 * os] = d0 - jd1;
  } else {
    static_assert(P % 2 == 1, "odd radix expected");
    constexpr int H = (P - 1) / 2;
    cx<T> sp[H], dm[H];
    cx<T> x0 = x[0];
    cx<T> total = x0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      sp[q - 1] = x[q * xs] + x[(P - q) * xs];
      dm[q - 1] = x[q * xs] - x[(P - q) * xs];
      total = total + sp[q - 1];
    }
    o[0] = total;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      cx<T> a = x0;     // symmetric part
      cx<T> b = {0, 0};  // antisymmetric part before multiplication by i
#pragma unroll
      for (int q = 1; q <= H; ++q) {
        const cx<T> w = tw<T, TOP, INV>(((q * k) % P) * (TOP / P));
        a.re = fma(sp[q - 1].re, w.re, a.re);
        a.im = fma(sp[q - 1].im, w.re, a.im);
        b.re = fma(dm[q - 1].re, w.im, b.re);
        b.im = fma(dm[q - 1].im, w.im, b.im);
      }
      // term: i * b  -> (-b.im, b.re)
      o[k * os] = cx<T>{a.re - b.im, a.im + b.re};
      o[(P - k) * os] = cx<T>{a.re + b.im, a.im - b.re};
    }
  }
}

// out[k] = sum_{j<N} in[j*IS] * w_N^{jk} (k < N), complex, unnormalised.
// TOP: length of the twiddle table (N divides TOP).
template <typename T, int N, int TOP, bool INV>
struct CFFT {
  static constexpr int P = pick_radix(N);
  static constexpr int M = N / P;
  __device__ __forceinline__ static void run(const cx<T>* in, int is, cx<T>* out) {
    if constexpr (N == 1) {
      out[0] = in[0];
    } else if constexpr (M == 1) {
      small_dft<T, P, TOP, INV>(in, is, out, 1);
    } else {
      cx<T> sub[P * M];
#pragma unroll
      for (int q = 0; q < P; ++q) CFFT<T, M, TOP, INV>::run(in + q * is, is * P, sub + q * M);
#pragma unroll
      for (int k1 = 0; k1 < M; ++k1) {
        cx<T> t[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const cx<T> v = sub[q * M + k1];
          t[q] = (q * k1 == 0) ? v : cmul(v, tw<T, TOP, INV>((q * k1) * (TOP / N)));
        }
        small_dft<T, P, TOP, INV>(t, 1, out + k1, M);
      }
    }
  }
};

// Forward real transform of x[0..L) -> X[0..L/2] (half spectrum, L/2+1 values).
template <typename T, int L>
__device__ __forceinline__ void rfft(const T* x, cx<T>* X) {
  if constexpr (L % 2 == 0) {
    constexpr int M = L / 2;
    cx<T> z[M];
#pragma unroll
    for (int m = 0; m < M; ++m) z[m] = cx<T>{x[2 * m], x[2 * m + 1]};
    cx<T> Z[M];
    CFFT<T, M, L, false>::run(z, 1, Z);
#pragma unroll
    for (int k = 0; k <= M; ++k) {
      const cx<T> zk = Z[k % M];
      const cx<T> zc = conj(Z[(M - k) % M]);
      const cx<T> E = (zk + zc) * T(0.5);
      const cx<T> D = (zk - zc) * T(0.5);  // O = D / i = (D.im, -D.re)
      const cx<T> O = {D.im, -D.re};
      if (k == 0) {
        X[k] = cx<T>{E.re + O.re, T(0)};
      } else if (k == M) {
        X[k] = cx<T>{E.re - O.re, T(0)};
      } else {
        X[k] = E + cmul(O, tw<T, L, false>(k));
      }
    }
  } else {
    cx<T> z[L];
#pragma unroll
    for (int m = 0; m < L; ++m) z[m] = cx<T>{x[m], T(0)};
    cx<T> Z[L];
    CFFT<T, L, L, false>::run(z, 1, Z);
#pragma unroll
    for (int k = 0; k <= L / 2; ++k) X[k] = Z[k];
    X[0].im = T(0);
  }
}

// Inverse real transform: half spectrum X[0..L/2] -> x[0..L), including the
// 1/L of Eq. (barAAk).  The imaginary parts of the DC (and, for even L, the
// Nyquist) slice are ignored, as for any Hermitian-extended spectrum.
template <typename T, int L>
__device__ __forceinline__ void irfft(const cx<T>* X, T* x) {
  if constexpr (L % 2 == 0) {
    constexpr int M = L / 2;
    cx<T> z[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      cx<T> a = X[k];
      cx<T> b = X[M - k];
      if (k == 0) {
        a.im = T(0);
        b.im = T(0);
      }
      const cx<T> bc = conj(b);
      const cx<T> E = (a + bc) * T(0.5);
      const cx<T> D = (a - bc) * T(0.5);
      const cx<T> O = (k == 0) ? D : cmul(D, tw<T, L, true>(k));
      z[k] = cx<T>{E.re - O.im, E.im + O.re};  // E + i O
    }
    cx<T> Z[M];
    CFFT<T, M, L, true>::run(z, 1, Z);
    const T s = T(1) / T(M);
#pragma unroll
    for (int m = 0; m < M; ++m) {
      x[2 * m] = Z[m].re * s;
      x[2 * m + 1] = Z[m].im * s;
    }
  } else {
    cx<T> z[L];
    z[0] = cx<T>{X[0].re, T(0)};
#pragma unroll
    for (int k = 1; k <= L / 2; ++k) {
      z[k] = X[k];
      z[L - k] = conj(X[k]);
    }
    cx<T> Z[L];
    CFFT<T, L, L, true>::run(z, 1, Z);
    const T s = T(1) / T(L);
#pragma unroll
    for (int m = 0; m < L; ++m) x[m] = Z[m].re * s;
  }
}

}  // namespace fft
}  // namespace tc

namespace tc {
namespace fft {

// Fill this translation unit's twiddle tables on the current device (FP64
// cos/sin rounded to the table type).  Each translation unit that launches a
// register-FFT kernel owns its own copy of the constant tables.
template <typename T>
static void upload_tables() {
  cx<T> tab[kTableSize];
  for (int i = 0; i < kNumLengths; ++i) {
    const int L = kLengths[i];
    const int off = table_offset(L);
    for (int m = 0; m < L; ++m) {
      const double a = 2.0 * 3.14159265358979323846 * (double)m / (double)L;
      tab[off + m] = cx<T>{(T)cos(a), (T)(-sin(a))};
    }
  }
  if constexpr (sizeof(T) == 4) {
    cudaMemcpyToSymbol(c_tw_f32, tab, sizeof(tab));
  } else {
    cudaMemcpyToSymbol(c_tw_f64, tab, sizeof(tab));
  }
}

}  // namespace fft
}  // namespace tc
