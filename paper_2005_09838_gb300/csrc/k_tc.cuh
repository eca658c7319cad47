// Slice contractions of the precision form on the fifth-generation tensor
// cores (tcgen05, sm_103a): operands rounded to TF32 or BF16 in shared memory,
// FP32 accumulation in tensor memory (TMEM).
//
// A complex product C = A B^H (or A B) is one real GEMM on the real embedding:
// row i of A~ holds (re, im) of its K complex entries as 2K reals, and the
// rows n = 2s (real part) and n = 2s + 1 (imaginary part) of the B operand hold
//   for C = A conj(B):  ( b_re,  b_im) and (-b_im, b_re)
// per complex column, so that sum_k A~[i, k] B~[n, k] gives re and im of
// C[i, s].  With `split`, each operand is carried as hi + lo (hi the rounded
// value, lo the rounded remainder) and the product takes hi*hi + hi*lo +
// lo*hi (three MMAs per step), which brings the error of a TF32 (BF16)
// contraction down from 2^-11 (2^-8) to about 2^-21 (2^-16) of its terms.
//
// Shared-memory operands use the K-major layout without swizzle: core
// matrices of 8 rows x 16 bytes, K-adjacent core matrices kLbo bytes apart,
// 8-row groups `sbo` bytes apart.  kLbo = 128 + 16: the staging stores of a
// half-warp (consecutive complex columns of one row) then hit distinct banks.
#pragma once

#include <cuda_bf16.h>

namespace tc {
namespace umma {

constexpr uint32_t kLbo = 144;
constexpr int kM = 128;        // rows of one MMA = TMEM lanes of the accumulator
constexpr int kTcThreads = 256;
constexpr int kChunk = 32;     // complex K values staged per step

enum Kind { kTF32 = 0, kBF16 = 1 };

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (sm_100 family): start address, leading
// (K-direction) and stride (8-row group) byte offsets in 16-byte units, the
// fixed version bits 46-48 = 0b001, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B types in
// bits 7-9 and 10-12 (TF32 = 2 for kind::tf32, BF16 = 1 for kind::f16), both
// K-major (bits 15, 16 clear), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int KIND>
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  const uint32_t ab = KIND == kTF32 ? 2u : 1u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
  if constexpr (KIND == kTF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(id), "r"(acc));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(id), "r"(acc));
  }
}

// Completion of this thread's earlier MMAs arrives once on the mbarrier.
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

// Bounded wait for the phase with the given parity; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity));
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM columns (a power of two >= 32): allocated and freed by one whole warp.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of the warp's TMEM lane (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(u[j]);
}

// ---- operand staging ------------------------------------------------------------------
template <int KIND>
__host__ __device__ constexpr int elem_bytes() { return KIND == kTF32 ? 4 : 2; }
// complex values per core-matrix row
template <int KIND>
__host__ __device__ constexpr int cx_per_row() { return 8 / elem_bytes<KIND>(); }
// bytes between 8-row groups for a chunk of kChunk complex K values
template <int KIND>
__host__ __device__ constexpr uint32_t chunk_sbo() { return (uint32_t)(kChunk / cx_per_row<KIND>()) * kLbo; }
template <int KIND>
__host__ __device__ constexpr uint32_t tile_bytes(int rows) { return (uint32_t)(rows / 8) * chunk_sbo<KIND>(); }

// Byte offset of complex column jj of row `row` in a staged tile.
template <int KIND>
__device__ __forceinline__ uint32_t cx_off(int row, int jj) {
  constexpr int per = cx_per_row<KIND>();
  return (uint32_t)(row >> 3) * chunk_sbo<KIND>() + (uint32_t)(jj / per) * kLbo + (uint32_t)(row & 7) * 16u +
         (uint32_t)(jj % per) * (2u * elem_bytes<KIND>());
}

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return __uint_as_float(u);
}

// Store the complex pair (a, b) at byte offset o of the hi tile (and the
// remainder at o of the lo tile when split).
template <int KIND, bool SPLIT>
__device__ __forceinline__ void put(unsigned char* hi, unsigned char* lo, uint32_t o, float a, float b) {
  if constexpr (KIND == kTF32) {
    const float ah = round_tf32(a), bh = round_tf32(b);
    *reinterpret_cast<float2*>(hi + o) = make_float2(ah, bh);
    if constexpr (SPLIT) *reinterpret_cast<float2*>(lo + o) = make_float2(round_tf32(a - ah), round_tf32(b - bh));
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    *reinterpret_cast<__nv_bfloat162*>(hi + o) = h;
    if constexpr (SPLIT) {
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(lo + o) = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    }
  }
}

// The MMAs of one staged chunk: A tile (kM rows) times B tile (N rows), all K
// steps of 32 bytes (two core matrices), accumulating into tmem.
template <int KIND, bool SPLIT>
__device__ __forceinline__ void mma_chunk(uint32_t tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                          uint32_t b_lo, int N, bool first) {
  constexpr uint32_t sbo = chunk_sbo<KIND>();
  constexpr int ksteps = kChunk / (2 * cx_per_row<KIND>());
  const uint32_t id = idesc<KIND>(kM, N);
#pragma unroll
  for (int ks = 0; ks < ksteps; ++ks) {
    const uint32_t o = (uint32_t)ks * 2u * kLbo;
    const uint64_t ah = sdesc(a_hi + o, kLbo, sbo), bh = sdesc(b_hi + o, kLbo, sbo);
    mma<KIND>(tmem, ah, bh, id, (first && ks == 0) ? 0u : 1u);
    if constexpr (SPLIT) {
      mma<KIND>(tmem, ah, sdesc(b_lo + o, kLbo, sbo), id, 1u);
      mma<KIND>(tmem, sdesc(a_lo + o, kLbo, sbo), bh, id, 1u);
    }
  }
}

constexpr int kWaitPolls = 1 << 24;

}  // namespace umma

// ---------------------------------------------------------------------------
// Q_k = R~_k Y~_k^H on the tensor cores (the contraction of k_qcon), for
// r <= 32: grid (S, ceil(n1 / 128)), 256 threads; rows i of the tile are the
// TMEM lanes, N = 64 columns (re, im) x 32.  R~ rows are read once, in chunks
// of 32 complex columns; the next chunk is loaded into registers while the
// tensor core works on the current one.
// ---------------------------------------------------------------------------
template <int KIND, bool SPLIT>
__host__ inline size_t qcon_tc_smem() {
  return (size_t)(SPLIT ? 2 : 1) * (umma::tile_bytes<KIND>(umma::kM) + umma::tile_bytes<KIND>(64)) + 64;
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(umma::kTcThreads) k_qcon_tc(Dev<float> d, cx<float>* __restrict__ Qout) {
  using namespace umma;
  extern __shared__ __align__(1024) unsigned char smem[];
  if (converged(d)) return;
  constexpr uint32_t TA = tile_bytes<KIND>(kM), TB = tile_bytes<KIND>(64);
  unsigned char* Ahi = smem;
  unsigned char* Alo = Ahi + TA;
  unsigned char* Bhi = Ahi + (SPLIT ? 2 : 1) * TA;
  unsigned char* Blo = Bhi + TB;
  unsigned char* misc = Bhi + (SPLIT ? 2 : 1) * TB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 8);
  int* bad = reinterpret_cast<int*>(misc + 16);

  const int k = blockIdx.x, i0 = blockIdx.y * kM;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nch = (n2 + kChunk - 1) / kChunk;

  if (tid == 0) {
    mbar_init(saddr(mbar));
    *bad = 0;
  }
  if (wid == 0) tmem_alloc(saddr(tslot), 64);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  // chunk loads: A 128 rows x 32 columns (16 per thread, a warp per row),
  // B 32 rows s x 32 columns (4 per thread)
  constexpr int AP = kM * kChunk / kTcThreads, BP = 32 * kChunk / kTcThreads;
  cx<float> va[AP], vb[BP];
  auto load = [&](int c) {
    const int j = c * kChunk + lane;
#pragma unroll
    for (int t = 0; t < AP; ++t) {
      const int row = (tid >> 5) + t * (kTcThreads / 32), i = i0 + row;
      va[t] = (i < n1 && j < n2) ? ldg_cx(d.Rt + ((size_t)i * S + k) * n2 + j) : cx<float>{0.f, 0.f};
    }
#pragma unroll
    for (int t = 0; t < BP; ++t) {
      const int s = (tid >> 5) + t * (kTcThreads / 32);
      vb[t] = (s < r && j < n2) ? ldg_cx(d.Yt + ((size_t)k * r + s) * n2 + j) : cx<float>{0.f, 0.f};
    }
  };
  load(0);
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    if (c > 0) {
      if (tid == 0 && !mbar_wait(saddr(mbar), (uint32_t)((c - 1) & 1), kWaitPolls)) *bad = 1;
      __syncthreads();
      if (*bad) {
        ok = false;
        break;
      }
    }
#pragma unroll
    for (int t = 0; t < AP; ++t) {
      const int row = (tid >> 5) + t * (kTcThreads / 32);
      put<KIND, SPLIT>(Ahi, Alo, cx_off<KIND>(row, lane), va[t].re, va[t].im);
    }
#pragma unroll
    for (int t = 0; t < BP; ++t) {
      const int s = (tid >> 5) + t * (kTcThreads / 32);
      // conj(Y): row 2s gives the real part, row 2s + 1 the imaginary part
      put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * s, lane), vb[t].re, vb[t].im);
      put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * s + 1, lane), -vb[t].im, vb[t].re);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      mma_chunk<KIND, SPLIT>(tmem, saddr(Ahi), saddr(Alo), saddr(Bhi), saddr(Blo), 64, c == 0);
      commit(saddr(mbar));
    }
    if (c + 1 < nch) load(c + 1);
  }
  if (ok) {
    if (tid == 0 && !mbar_wait(saddr(mbar), (uint32_t)((nch - 1) & 1), kWaitPolls)) *bad = 1;
    __syncthreads();
    ok = *bad == 0;
  }
  fence_after();
  if (ok) {
    // warp w: TMEM lanes 32 (w % 4) .., columns 32 (w / 4) .. (s = 16 (w / 4) ..)
    const int q = wid & 3, h = wid >> 2;
    const int i = i0 + q * 32 + lane;
    float v[32];
    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 32);
    tmem_ld16(ta, v);
    tmem_ld16(ta + 16, v + 16);
    if (i < n1) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int s = h * 16 + c;
        if (s < r) Qout[((size_t)k * r + s) * n1 + i] = cx<float>{v[2 * c], v[2 * c + 1]};
      }
    }
  } else if (tid == 0) {
    set_err(d.err, DEV_TIMEOUT);
    mbar_wait(saddr(mbar), (uint32_t)((nch - 1) & 1), kWaitPolls);  // let issued MMAs drain
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (wid == 0) tmem_free(tmem, 64);
}


// ---------------------------------------------------------------------------
// Partial D^T = R~_k(:, tile)^T conj(X~'_k) over one range of n1 on the tensor
// cores (the contraction of the Y-step, D = X~'^H R~): grid (S, ceil(n2 / 128),
// ksplit); rows j of the tile are the TMEM lanes, N = 64 columns (re, im) x 32,
// K = the i of the range in chunks of 32.  Partial sums go to
// Dpart[k][z][s][j], summed in a fixed order by the Y-step.
// ---------------------------------------------------------------------------
template <int KIND, bool SPLIT>
__host__ inline size_t dcon_tc_smem() {
  return qcon_tc_smem<KIND, SPLIT>();
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(umma::kTcThreads) k_dcon_tc(Dev<float> d) {
  using namespace umma;
  extern __shared__ __align__(1024) unsigned char smem[];
  if (converged(d)) return;
  constexpr uint32_t TA = tile_bytes<KIND>(kM), TB = tile_bytes<KIND>(64);
  unsigned char* Ahi = smem;
  unsigned char* Alo = Ahi + TA;
  unsigned char* Bhi = Ahi + (SPLIT ? 2 : 1) * TA;
  unsigned char* Blo = Bhi + TB;
  unsigned char* misc = Bhi + (SPLIT ? 2 : 1) * TB;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 8);
  int* bad = reinterpret_cast<int*>(misc + 16);

  const int k = blockIdx.x, j0 = blockIdx.y * kM, z = blockIdx.z;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S, ks = d.ksplit;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int ilen = ((n1 + ks - 1) / ks + kChunk - 1) / kChunk * kChunk;
  const int ib = z * ilen, ie = min(n1, ib + ilen);
  const int nch = ie > ib ? (ie - ib + kChunk - 1) / kChunk : 0;

  if (tid == 0) {
    mbar_init(saddr(mbar));
    *bad = 0;
  }
  if (wid == 0) tmem_alloc(saddr(tslot), 64);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  // A: element (i, j) of R~ at row j - j0, column i - ic (a warp reads 32
  // consecutive j of one i); B: conj(X~') rows 2s, 2s + 1, column i - ic
  constexpr int AP = kM * kChunk / kTcThreads, BP = 32 * kChunk / kTcThreads;
  cx<float> va[AP], vb[BP];
  auto load = [&](int c) {
    const int ic = ib + c * kChunk;
#pragma unroll
    for (int t = 0; t < AP; ++t) {
      const int e = tid + t * kTcThreads, jl = e & (kM - 1), il = e >> 7;
      const int i = ic + il, j = j0 + jl;
      va[t] = (i < ie && j < n2) ? ldg_cx(d.Rt + ((size_t)i * S + k) * n2 + j) : cx<float>{0.f, 0.f};
    }
#pragma unroll
    for (int t = 0; t < BP; ++t) {
      const int s = wid + t * (kTcThreads / 32), i = ic + lane;
      vb[t] = (s < r && i < ie) ? ldg_cx(d.Xt + ((size_t)k * r + s) * n1 + i) : cx<float>{0.f, 0.f};
    }
  };
  if (nch > 0) load(0);
  bool ok = true;
  for (int c = 0; c < nch; ++c) {
    if (c > 0) {
      if (tid == 0 && !mbar_wait(saddr(mbar), (uint32_t)((c - 1) & 1), kWaitPolls)) *bad = 1;
      __syncthreads();
      if (*bad) {
        ok = false;
        break;
      }
    }
#pragma unroll
    for (int t = 0; t < AP; ++t) {
      const int e = tid + t * kTcThreads, jl = e & (kM - 1), il = e >> 7;
      put<KIND, SPLIT>(Ahi, Alo, cx_off<KIND>(jl, il), va[t].re, va[t].im);
    }
#pragma unroll
    for (int t = 0; t < BP; ++t) {
      const int s = wid + t * (kTcThreads / 32);
      put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * s, lane), vb[t].re, vb[t].im);
      put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * s + 1, lane), -vb[t].im, vb[t].re);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      mma_chunk<KIND, SPLIT>(tmem, saddr(Ahi), saddr(Alo), saddr(Bhi), saddr(Blo), 64, c == 0);
      commit(saddr(mbar));
    }
    if (c + 1 < nch) load(c + 1);
  }
  if (ok && nch > 0) {
    if (tid == 0 && !mbar_wait(saddr(mbar), (uint32_t)((nch - 1) & 1), kWaitPolls)) *bad = 1;
    __syncthreads();
    ok = *bad == 0;
  }
  fence_after();
  if (ok) {
    const int q = wid & 3, h = wid >> 2;
    const int jl = q * 32 + lane, j = j0 + jl;
    float v[32];
    if (nch > 0) {
      const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 32);
      tmem_ld16(ta, v);
      tmem_ld16(ta + 16, v + 16);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = 0.f;
    }
    if (j < n2) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int s = h * 16 + c;
        if (s < r) d.Dpart[(((size_t)k * ks + z) * r + s) * n2 + j] = cx<float>{v[2 * c], v[2 * c + 1]};
      }
    }
  } else if (tid == 0) {
    set_err(d.err, DEV_TIMEOUT);
    mbar_wait(saddr(mbar), (uint32_t)((nch - 1) & 1), kWaitPolls);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (wid == 0) tmem_free(tmem, 64);
}

// ---------------------------------------------------------------------------
// Z~_k(tile) = X~'_k Y~'_k on the tensor cores (step 3 for the slab kernel):
// grid (S, ceil(n1 / 128), ceil(n2 / 64)); rows i are the TMEM lanes, N = 128
// columns (re, im) x 64, K = the r <= 32 columns of X~' (one chunk).  The
// tile goes through shared memory (rows padded to 65 complex values) so the
// stores to Z~ (and to dZ~ for the stopping test) are coalesced.
// ---------------------------------------------------------------------------
constexpr int kZCols = 64;
constexpr int kZLd = kZCols + 1;

template <int KIND, bool SPLIT>
__host__ inline size_t zsyn_tc_smem() {
  const size_t ops = (size_t)(SPLIT ? 2 : 1) * (umma::tile_bytes<KIND>(umma::kM) + umma::tile_bytes<KIND>(2 * kZCols));
  const size_t stage = (size_t)umma::kM * kZLd * sizeof(cx<float>);
  return (ops > stage ? ops : stage) + 64;
}

template <int KIND, bool SPLIT>
__global__ void __launch_bounds__(umma::kTcThreads) k_zsyn_tc(Dev<float> d) {
  using namespace umma;
  extern __shared__ __align__(1024) unsigned char smem[];
  if (converged(d)) return;
  constexpr uint32_t TA = tile_bytes<KIND>(kM), TB = tile_bytes<KIND>(2 * kZCols);
  constexpr size_t OPS = (size_t)(SPLIT ? 2 : 1) * (TA + TB);
  constexpr size_t STAGE = (size_t)kM * kZLd * sizeof(cx<float>);
  unsigned char* Ahi = smem;
  unsigned char* Alo = Ahi + TA;
  unsigned char* Bhi = Ahi + (SPLIT ? 2 : 1) * TA;
  unsigned char* Blo = Bhi + TB;
  unsigned char* misc = smem + (OPS > STAGE ? OPS : STAGE);
  cx<float>* Zs = reinterpret_cast<cx<float>*>(smem);  // [kM][kZLd] after the MMAs
  uint64_t* mbar = reinterpret_cast<uint64_t*>(misc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(misc + 8);
  int* bad = reinterpret_cast<int*>(misc + 16);

  const int k = blockIdx.x, i0 = blockIdx.y * kM, j0 = blockIdx.z * kZCols;
  const int n1 = d.n1, n2 = d.n2, r = d.r, S = d.S;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(saddr(mbar));
    *bad = 0;
  }
  if (wid == 0) tmem_alloc(saddr(tslot), 2 * kZCols);
  // A: X~'(i, s) at row i - i0, column s (a warp reads 32 consecutive i of one s)
#pragma unroll 4
  for (int t = 0; t < kM * kChunk / kTcThreads; ++t) {
    const int e = tid + t * kTcThreads, il = e & (kM - 1), s = e >> 7, i = i0 + il;
    const cx<float> x = (s < r && i < n1) ? ldg_cx(d.Xt + ((size_t)k * r + s) * n1 + i) : cx<float>{0.f, 0.f};
    put<KIND, SPLIT>(Ahi, Alo, cx_off<KIND>(il, s), x.re, x.im);
  }
  // B: rows 2 jl (real part: (y_re, -y_im)) and 2 jl + 1 (imaginary part: (y_im, y_re))
#pragma unroll 4
  for (int t = 0; t < kZCols * kChunk / kTcThreads; ++t) {
    const int e = tid + t * kTcThreads, jl = e & (kZCols - 1), s = e >> 6, j = j0 + jl;
    const cx<float> y = (s < r && j < n2) ? ldg_cx(d.Yt + ((size_t)k * r + s) * n2 + j) : cx<float>{0.f, 0.f};
    put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * jl, s), y.re, -y.im);
    put<KIND, SPLIT>(Bhi, Blo, cx_off<KIND>(2 * jl + 1, s), y.im, y.re);
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    mma_chunk<KIND, SPLIT>(tmem, saddr(Ahi), saddr(Alo), saddr(Bhi), saddr(Blo), 2 * kZCols, true);
    commit(saddr(mbar));
    if (!mbar_wait(saddr(mbar), 0u, kWaitPolls)) *bad = 1;
  }
  __syncthreads();
  fence_after();
  const bool ok = *bad == 0;
  if (ok) {
    // warp w: TMEM lanes 32 (w % 4) .., columns 64 (w / 4) .. (jl = 32 (w / 4) ..)
    const int q = wid & 3, h = wid >> 2, row = q * 32 + lane;
#pragma unroll
    for (int part = 0; part < 4; ++part) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 64 + part * 16), v);
#pragma unroll
      for (int c = 0; c < 8; ++c) Zs[row * kZLd + h * 32 + part * 8 + c] = cx<float>{v[2 * c], v[2 * c + 1]};
    }
  } else if (tid == 0) {
    set_err(d.err, DEV_TIMEOUT);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (wid == 0) tmem_free(tmem, 2 * kZCols);
  if (!ok) return;
  // coalesced stores: a warp writes 32 consecutive j of one row
  for (int e = tid; e < kM * kZCols; e += kTcThreads) {
    const int row = e / kZCols, jl = e - row * kZCols, i = i0 + row, j = j0 + jl;
    if (i < n1 && j < n2) {
      const size_t o = ((size_t)i * S + k) * n2 + j;
      const cx<float> zv = Zs[row * kZLd + jl];
      if (d.dZt) d.dZt[o] = zv - d.Zt[o];  // Z~^{l+1} - Z~^l for the stopping test
      d.Zt[o] = zv;
    }
  }
}

}  // namespace tc
