// Allocation-free completion entry point (tc_complete_static).
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework
// whose allocator owns all of the device memory (and forbids raw allocations
// behind its back), and latency-critical loops where cudaMalloc/cudaFree may
// synchronise the whole device and stall unrelated streams.  For them this file
// runs a complete TCTF2R completion of a small tensor with every intermediate
// array (packed observations, residual spectrum, factor spectra, work arrays,
// tables) carved from one file-scope device array of fixed size.
//
// The kernels are the library's own, instantiated here with the generic mode-3
// transform; only the memory they work in differs.
#include <cuda_runtime.h>

#include <cmath>
#include <limits>
#include <mutex>
#include <string>

#include "tc_engine.cuh"
#include "tctf2r.h"

namespace tc {
void set_last_error(const std::string& msg);  // tc_api.cu: the message tc_last_error() returns
}

namespace {

using namespace tc;

// Fixed scratch: 16 MiB on every device that loads this library, held until
// the process exits.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

tc_status sfail(tc_status st, const std::string& msg) {
  tc::set_last_error(msg);
  return st;
}

// Device address of g_static_scratch on the current device, looked up once per
// device (the name itself is only a host-side stand-in for the symbol).
tc_status scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return sfail(TC_ERR_ARG, "device ordinal beyond the supported range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr)
      return sfail(TC_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") +
                                    cudaGetErrorString(e));
    g_scratch_addr[dev] = ptr;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return TC_OK;
}

// Bump allocator over the static array (offsets only, nothing is allocated).
struct Carve {
  unsigned char* base;
  size_t off = 0;
  template <typename U>
  U* take(size_t elems) {
    off = align_up(off, 256);
    U* p = reinterpret_cast<U*>(base + off);
    off += elems * sizeof(U);
    return p;
  }
};

// Device-side construction of the FP64 tables (no host buffers): inverse LU
// pivots of the W-step runs and of H_rho1, and the generic DFT twiddles.
template <typename T>
__global__ void k_static_tables(T* winv, T* hinv, cx<T>* twg, int n1, int n2, int n3, double mu, double rho1,
                                double rho2) {
  if (blockIdx.x == 0 && threadIdx.x == 0) wstep_tables<T>(winv, n2, mu, rho2);
  if (blockIdx.x == 1 && threadIdx.x == 0) {
    double hi = 0.0;
    for (int i = 0; i < n1; ++i) {
      const int deg = (i > 0) + (i + 1 < n1);
      hi = 1.0 / (1.0 + rho1 * deg - (i > 0 ? rho1 * rho1 * hi : 0.0));
      hinv[i] = (T)hi;
      hinv[n1 + i] = (T)(rho1 * hi);
    }
  }
  if (blockIdx.x == 2) {
    for (int m = threadIdx.x; m < n3; m += blockDim.x) {
      double s, c;
      sincospi(2.0 * (double)m / (double)n3, &s, &c);
      twg[m] = cx<T>{(T)c, (T)(-s)};
    }
  }
}

// f0 of Eq. (TETP-optim) from the slab-kernel partial sums and the per-slice
// rho1 terms, reduced in a fixed order by one thread.
__global__ void k_static_objective(const double* part, const double* part_k, int n1, int S, int n3, double mu,
                                   double rho1, double rho2, double* out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double sr = 0, sw = 0, sk = 0, sh = 0;
  for (int i = 0; i < n1; ++i) {
    sr += part[(size_t)i * 4 + 0];
    sw += part[(size_t)i * 4 + 2];
    sk += part[(size_t)i * 4 + 3];
  }
  for (int k = 0; k < S; ++k) {
    double pk = 0.0;
    for (int c = 0; c < kRhoChunks; ++c) pk += part_k[(size_t)k * kRhoChunks + c];
    sh += ((k == 0 || 2 * k == n3) ? 1.0 : 2.0) * pk;
  }
  out[0] = 0.5 * sr + 0.5 * mu * sw + 0.5 * rho2 * sk + 0.5 * rho1 * sh / (double)n3;
}

template <typename T>
tc_status run_static(const tc_params& p, const void* G, const uint8_t* mask, const void* Y0, const void* X0,
                     int n_iters, void* W, double* f0, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return sfail(TC_ERR_CUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  tc_status s0 = scratch_address(dev, &base);
  if (s0 != TC_OK) return s0;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return sfail(TC_ERR_CUDA, "cudaDeviceGetAttribute (shared memory opt-in limit) failed");
  optin -= kStaticSmemReserve;  // room for the kernels' static shared memory

  const int n1 = (int)p.n1, n2 = (int)p.n2, n3 = (int)p.n3, r = p.r, S = n3 / 2 + 1, mw = (n2 + 31) / 32;
  const int rp = pad_rank<T>(r);
  const size_t N = (size_t)n1 * n2 * n3;
  const size_t nx = (size_t)S * r * n1, ny = (size_t)S * r * n2, nrr = (size_t)S * r * r;

  SlabLayout lay = slab_layout<T>(n2, n3, false, true);
  const bool slabs_in_smem = lay.total <= (size_t)optin;
  if (!slabs_in_smem) lay = slab_layout<T>(n2, n3, false, false);
  XLayout xl = xstep_layout_for<T>(n1, n2, r, rp, false, true);
  const bool xsmem = xl.total <= (size_t)optin;
  if (!xsmem) xl = xstep_layout_for<T>(n1, n2, r, rp, false, false);
  const bool yxg = ystep_smem_bytes<T>(n1, r, rp) > (size_t)optin;
  const size_t ysm = ystep_smem_bytes<T>(n1, r, rp, !yxg), qsm = qcon_smem_bytes<T>(n2, r, rp);
  if (xl.total > (size_t)optin || ysm > (size_t)optin || qsm > (size_t)optin)
    return sfail(TC_ERR_UNSUPPORTED, "shared memory of the slice kernels exceeds the device limit for these sizes");

  // ---- carve the state from the static array ----------------------------------------
  Carve cv{base};
  Dev<T> d{};
  T* Gint = cv.take<T>(N);
  uint32_t* maskbits = cv.take<uint32_t>((size_t)n1 * n3 * mw);
  d.Rt = cv.take<cx<T>>((size_t)n1 * S * n2);
  d.Zt = cv.take<cx<T>>((size_t)n1 * S * n2);
  d.ytiles = (n2 + 31) / 32;
  d.Ag = cv.take<cx<double>>((size_t)S * d.ytiles * (r * (r + 1) / 2));
  d.Xt = cv.take<cx<T>>(nx);
  cx<T>* Q = cv.take<cx<T>>(nx);
  d.Tb = cv.take<cx<T>>(nx);
  d.Yt = cv.take<cx<T>>(ny);
  d.Dg = cv.take<cx<T>>(nrr);
  d.Gp = cv.take<cx<T>>(nrr);
  d.Gp64 = sizeof(T) == 4 ? cv.take<cx<double>>((size_t)2 * r * r) : nullptr;
  T* winv = cv.take<T>((size_t)6 * n2);
  T* hinv = cv.take<T>((size_t)2 * n1);
  cx<T>* twg = cv.take<cx<T>>((size_t)n3);
  d.part = cv.take<double>((size_t)n1 * 4);
  d.part_k = cv.take<double>((size_t)S * kRhoChunks);
  double* fout = cv.take<double>(1);
  d.err = cv.take<int>(1);
  d.scratch = slabs_in_smem ? nullptr : cv.take<T>(lay.slab_bytes / sizeof(T) * (size_t)n1 + 16);
  if (cv.off > kStaticScratchBytes) {
    return sfail(TC_ERR_ARG, "problem needs " + std::to_string(cv.off) + " bytes of scratch; the static scratch of " +
                                 "tc_complete_static holds " + std::to_string(kStaticScratchBytes) + " bytes");
  }
  d.n1 = n1;
  d.n2 = n2;
  d.n3 = n3;
  d.S = S;
  d.r = r;
  d.mw = mw;
  d.mu = (T)p.mu;
  d.rho1 = (T)p.rho1;
  d.rho2 = (T)p.rho2;
  d.G = Gint;
  d.mask = maskbits;
  d.winv = winv;
  d.hinv = hinv;
  d.twg = twg;
  d.yx_global = yxg ? 1 : 0;
  d.rtol = (p.pinv_rtol > 0) ? p.pinv_rtol : default_rtol<T>(r, rp, false);
  d.rtol64 = (p.pinv_rtol > 0) ? p.pinv_rtol : (double)r * std::numeric_limits<double>::epsilon();

  // ---- kernels (generic mode-3 transform) ------------------------------------------------
  SlabFn<T> slab[3];
  slab_table<T, 0>(slab);
  YFn<T> ystep = pick_ystep<T>(rp, !yxg);
  QFn<T> qcon = pick_qcon<T>(rp);
  XFn<T> xstep = pick_xstep_for<T>(rp, false);
  const struct {
    const void* fn;
    size_t bytes;
    const char* name;
  } opt_in[] = {{(const void*)slab[MODE_ITER], lay.total, "slab (iteration)"},
                {(const void*)slab[MODE_W], lay.total, "slab (W read-back)"},
                {(const void*)slab[MODE_R], lay.total, "slab (objective)"},
                {(const void*)xstep, xl.total, "X-step"},
                {(const void*)ystep, ysm, "Y-step"},
                {(const void*)qcon, qsm, "Q contraction"}};
  for (const auto& o : opt_in) {
    const cudaError_t e = allow_dynamic_smem(o.fn, o.bytes);
    if (e != cudaSuccess)
      return sfail(TC_ERR_CUDA, std::string("dynamic shared memory opt-in of ") + std::to_string(o.bytes) +
                                    " bytes for the " + o.name + " kernel failed: " + cudaGetErrorString(e));
  }
  const int sis = slabs_in_smem ? 1 : 0;
  const int fgrid = 4 * 152;

  // the array keeps the previous call's contents: clear what must start at zero
  {
    const cudaError_t e = cudaMemsetAsync(d.err, 0, sizeof(int), st);
    if (e != cudaSuccess)
      return sfail(TC_ERR_CUDA, std::string("clearing the device error flag failed: ") + cudaGetErrorString(e));
  }
  k_static_tables<T><<<3, 256, 0, st>>>(winv, hinv, twg, n1, n2, n3, p.mu, p.rho1, p.rho2);
  k_pack<T><<<n1 * n3, 256, 0, st>>>(static_cast<const T*>(G), mask, Gint, maskbits, n1, n2, n3, mw);
  k_factor_dft<T><<<fgrid, 256, 0, st>>>(static_cast<const T*>(Y0), d.Yt, n2, r, n3, 1, twg);
  if (X0) {
    k_factor_dft<T><<<fgrid, 256, 0, st>>>(static_cast<const T*>(X0), d.Xt, n1, r, n3, 0, twg);
  } else {
    const cudaError_t e = cudaMemsetAsync(d.Xt, 0, nx * sizeof(cx<T>), st);
    if (e != cudaSuccess)
      return sfail(TC_ERR_CUDA, std::string("clearing X~0 failed: ") + cudaGetErrorString(e));
  }
  k_synth_init<T><<<fgrid, 256, 0, st>>>(d);
  k_gram_tiles<T><<<dim3(S, d.ytiles), 256, 0, st>>>(d);
  slab[MODE_ITER]<<<n1, 256, lay.total, st>>>(d, nullptr, sis, 1);
  for (int it = 0; it < n_iters; ++it) {
    qcon<<<dim3(S, (n1 + 31) / 32), kSliceThreads, qsm, st>>>(d, Q);
    xstep<<<S, xstep_threads(rp), xl.total, st>>>(d, Q, xsmem ? 1 : 0);
    ystep<<<dim3(S, (n2 + 32 * ystep_cpl(rp) - 1) / (32 * ystep_cpl(rp))), kYThreads, ysm, st>>>(d);
    slab[MODE_ITER]<<<n1, 256, lay.total, st>>>(d, nullptr, sis, 0);
  }
  slab[MODE_W]<<<n1, 256, lay.total, st>>>(d, static_cast<T*>(W), sis, 0);
  if (f0) {
    slab[MODE_R]<<<n1, 256, lay.total, st>>>(d, nullptr, sis, 0);
    k_rho1_term<T><<<dim3(S, kRhoChunks), 256, 0, st>>>(d);
    k_static_objective<<<1, 32, 0, st>>>(d.part, d.part_k, n1, S, n3, p.mu, p.rho1, p.rho2, fout);
  }
  cudaError_t e = cudaGetLastError();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  double hf = 0.0;
  if (e == cudaSuccess && f0) e = cudaMemcpyAsync(&hf, fout, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return sfail(TC_ERR_CUDA, std::string("tc_complete_static: ") + cudaGetErrorString(e));
  if (herr != DEV_OK) return sfail(TC_ERR_CUDA, "device-side check failed (code " + std::to_string(herr) + ")");
  if (f0) {
    *f0 = hf;
    if (!std::isfinite(hf)) return sfail(TC_ERR_NUMERIC, "objective is not finite");
  }
  return TC_OK;
}

}  // namespace

extern "C" tc_status tc_complete_static(const tc_params* p, const void* G, const uint8_t* mask, const void* Y0,
                                        const void* X0, int32_t n_iters, void* W, double* f0, void* cuda_stream) {
  tc::set_last_error("");
  if (!p) return sfail(TC_ERR_ARG, "params is NULL");
  if (!G || !mask || !Y0 || !W) return sfail(TC_ERR_ARG, "G, mask, Y0 and W are required (device pointers)");
  if (n_iters < 0) return sfail(TC_ERR_ARG, "n_iters must be >= 0");
  if (p->n1 < 1 || p->n2 < 1 || p->n3 < 1 || p->n1 > (1 << 24) || p->n2 > 4096 || p->n3 > 4096)
    return sfail(TC_ERR_ARG, "sizes out of range");
  if (p->r < 1 || p->r > 32 || p->r > p->n1 || p->r > p->n2)
    return sfail(TC_ERR_ARG, "r must satisfy 1 <= r <= min(n1, n2, 32)");
  if (!(p->mu >= 0) || !(p->rho1 >= 0) || !(p->rho2 >= 0) || !std::isfinite(p->mu) || !std::isfinite(p->rho1) ||
      !std::isfinite(p->rho2))
    return sfail(TC_ERR_ARG, "mu, rho1, rho2 must be finite and >= 0");
  if (p->flags != 0 || p->step != TC_STEP_EXACT || p->eps != 0.0)
    return sfail(TC_ERR_UNSUPPORTED, "tc_complete_static runs exact steps for a fixed number of iterations only");
  if (!std::isfinite(p->pinv_rtol) || p->pinv_rtol >= 1.0) return sfail(TC_ERR_ARG, "pinv_rtol must be < 1");
  if (p->precision != TC_FP64 && p->precision != TC_FP32) return sfail(TC_ERR_UNSUPPORTED, "precision not built");
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    // the call reads results back to host variables and synchronises the
    // stream, neither of which a stream capture allows
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess)
      return sfail(TC_ERR_CUDA, "cudaStreamIsCapturing failed on the given stream");
    if (cs != cudaStreamCaptureStatusNone)
      return sfail(TC_ERR_STATE, "tc_complete_static must not be called on a stream that is being captured");
  }
  // every buffer must be device memory of the current device (a host pointer
  // would be dereferenced by the kernels)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return sfail(TC_ERR_CUDA, "cudaGetDevice failed");
  const struct {
    const void* ptr;
    const char* name;
  } bufs[] = {{G, "G"}, {mask, "mask"}, {Y0, "Y0"}, {X0, "X0"}, {W, "W"}};
  for (const auto& b : bufs) {
    if (!b.ptr) continue;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, b.ptr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return sfail(TC_ERR_ARG, std::string(b.name) + " is not a pointer the CUDA runtime knows");
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
      return sfail(TC_ERR_ARG, std::string(b.name) + " must be device memory of the current device");
  }
  if (p->precision == TC_FP64) return run_static<double>(*p, G, mask, Y0, X0, n_iters, W, f0, st);
  return run_static<float>(*p, G, mask, Y0, X0, n_iters, W, f0, st);
}
