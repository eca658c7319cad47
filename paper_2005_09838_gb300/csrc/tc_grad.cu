// Differentiation form of the library: loss and gradient of the factor model
// (the adjoint kernels of k_grad.cuh and the slab kernel's MODE_GRAD), behind
// the C ABI tc_grad_init / tc_grad_eval / tc_grad_free.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "tc_kernels.cuh"
#include "tctf2r.h"

namespace tc {
void set_last_error(const std::string& msg);
}

namespace {

using namespace tc;

template <typename T>
using GSlabFn = void (*)(Dev<T>, T*, int, int);

inline int grad_pad_rank(int r) { return r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : r <= 16 ? 16 : 32; }

template <typename T>
using GFn = void (*)(Dev<T>, cx<T>*);

template <typename T>
GFn<T> pick_dcon(int rp) {
  switch (rp) {
    case 2: return k_dcon<T, 2>;
    case 4: return k_dcon<T, 4>;
    case 8: return k_dcon<T, 8>;
    case 16: return k_dcon<T, 16>;
    default: return k_dcon<T, 32>;
  }
}
template <typename T>
GFn<T> pick_qcon_g(int rp) {
  switch (rp) {
    case 2: return k_qcon<T, 2>;
    case 4: return k_qcon<T, 4>;
    case 8: return k_qcon<T, 8>;
    case 16: return k_qcon<T, 16>;
    default: return k_qcon<T, 32>;
  }
}

// Slab kernel for MODE_GRAD: the shared-memory transform for n3 in {112, 168}
// (FP32), the register transform for n3 = 7 (FP64), else the direct DFT.
template <typename T>
struct GradSlab {
  GSlabFn<T> f = nullptr;
  int threads = 256;
  size_t smem = 0;
  bool in_smem = true;
  size_t scratch_bytes = 0;
};

template <typename T>
GradSlab<T> pick_grad_slab(int n2, int n3, int optin) {
  GradSlab<T> g;
  if constexpr (sizeof(T) == 4) {
    if (n3 == 168 || n3 == 112) {
      const SlabFLayout lay = slab_f_layout<T>(n2, n3);
      if (lay.total <= (size_t)optin) {
        fft::upload_tables<T>();
        g.f = (n3 == 168) ? k_slab_f<T, 168, 12, 7, MODE_GRAD> : k_slab_f<T, 112, 8, 7, MODE_GRAD>;
        g.threads = kSlabFThreads;
        g.smem = lay.total;
        return g;
      }
    }
  } else {
    if (n3 == 7) {
      const SlabLayout lay = slab_layout<T>(n2, 7, true, true);
      if (lay.total <= (size_t)optin) {
        fft::upload_tables<T>();
        g.f = k_slab<T, 7, MODE_GRAD>;
        g.threads = std::max(std::min((n2 + 31) / 32 * 32, slab_max_threads(7)), 32);
        g.smem = lay.total;
        return g;
      }
    }
  }
  SlabLayout lay = slab_layout<T>(n2, n3, false, true);
  g.f = k_slab<T, 0, MODE_GRAD>;
  g.threads = 256;
  if (lay.total > (size_t)optin) {
    g.in_smem = false;
    lay = slab_layout<T>(n2, n3, false, false);
    g.scratch_bytes = lay.slab_bytes;
  }
  g.smem = lay.total;
  return g;
}

}  // namespace

struct tc_grad {
  virtual ~tc_grad() {}
  virtual tc_status eval(const void* X, const void* Y, double* loss, void* dX, void* dY, bool on_device,
                         std::string& err) = 0;
  int device = 0;
};

namespace {

#define TCG_TRY(expr)                                                        \
  do {                                                                       \
    cudaError_t e_ = (expr);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      err = std::string(#expr) + ": " + cudaGetErrorString(e_);              \
      return (e_ == cudaErrorMemoryAllocation) ? TC_ERR_NOMEM : TC_ERR_CUDA; \
    }                                                                        \
  } while (0)

template <typename T>
struct GradEngine final : tc_grad {
  ~GradEngine() override {
    for (void* q : allocs_) cudaFree(q);
  }

  template <typename U>
  U* alloc(size_t elems, std::string& err) {
    if (!err.empty()) return nullptr;
    void* q = nullptr;
    const size_t bytes = elems * sizeof(U) > 0 ? elems * sizeof(U) : 16;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed";
      return nullptr;
    }
    allocs_.push_back(q);
    return static_cast<U*>(q);
  }

  tc_status init(const tc_params& p, const void* G, const uint8_t* mask, bool on_device, cudaStream_t stream,
                 std::string& err) {
    stream_ = stream;
    n1_ = (int)p.n1;
    n2_ = (int)p.n2;
    n3_ = (int)p.n3;
    r_ = p.r;
    S_ = n3_ / 2 + 1;
    rp_ = grad_pad_rank(r_);
    const int mw = (n2_ + 31) / 32;
    const size_t N = (size_t)n1_ * n2_ * n3_;
    TCG_TRY(cudaGetDevice(&device));
    int optin = 0;
    TCG_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    optin -= kStaticSmemReserve;  // room for the kernels' static shared memory
    if constexpr (sizeof(T) == 8) fft::upload_tables<T>();

    T* Gint = alloc<T>(N, err);
    uint32_t* maskbits = alloc<uint32_t>((size_t)n1_ * n3_ * mw, err);
    cx<T>* Rt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    cx<T>* Zt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    cx<T>* Xt = alloc<cx<T>>((size_t)S_ * r_ * n1_, err);
    cx<T>* Yt = alloc<cx<T>>((size_t)S_ * r_ * n2_, err);
    GX_ = alloc<cx<T>>((size_t)S_ * r_ * n1_, err);
    GY_ = alloc<cx<T>>((size_t)S_ * r_ * n2_, err);
    cx<T>* twg = alloc<cx<T>>((size_t)n3_, err);
    double* part = alloc<double>((size_t)n1_ * 4, err);
    double* part_k = alloc<double>((size_t)S_ * kRhoChunks, err);
    int* derr = alloc<int>(1, err);
    xin_ = alloc<T>((size_t)n1_ * r_ * n3_, err);
    yin_ = alloc<T>((size_t)r_ * n2_ * n3_, err);
    if (!err.empty()) return TC_ERR_NOMEM;

    slab_ = pick_grad_slab<T>(n2_, n3_, optin);
    if (!slab_.in_smem) {
      T* scratch = alloc<T>(slab_.scratch_bytes / sizeof(T) * (size_t)n1_ + 16, err);
      if (!err.empty()) return TC_ERR_NOMEM;
      d_.scratch = scratch;
    }
    TCG_TRY(allow_dynamic_smem((const void*)slab_.f, slab_.smem));
    qcon_ = pick_qcon_g<T>(rp_);
    dcon_ = pick_dcon<T>(rp_);
    qsmem_ = qcon_smem_bytes<T>(n2_, r_, rp_);
    dsmem_ = dcon_smem_bytes<T>(n1_, r_, rp_);
    d_.yx_global = dsmem_ > (size_t)optin ? 1 : 0;
    if (d_.yx_global) dsmem_ = dcon_smem_bytes<T>(n1_, r_, rp_, false);
    if (qsmem_ > (size_t)optin || dsmem_ > (size_t)optin) {
      err = "shared memory of the gradient kernels exceeds the device limit for these sizes";
      return TC_ERR_UNSUPPORTED;
    }
    TCG_TRY(allow_dynamic_smem((const void*)qcon_, qsmem_));
    TCG_TRY(allow_dynamic_smem((const void*)dcon_, dsmem_));

    std::vector<cx<T>> tw(n3_);
    for (int m = 0; m < n3_; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)n3_;
      tw[m] = cx<T>{(T)std::cos(a), (T)(-std::sin(a))};
    }
    TCG_TRY(cudaMemcpyAsync(twg, tw.data(), tw.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, stream_));

    d_.n1 = n1_;
    d_.n2 = n2_;
    d_.n3 = n3_;
    d_.S = S_;
    d_.r = r_;
    d_.mw = mw;
    d_.rho1 = (T)p.rho1;
    d_.G = Gint;
    d_.mask = maskbits;
    d_.Rt = Rt;
    d_.Zt = Zt;
    d_.Xt = Xt;
    d_.Yt = Yt;
    d_.twg = twg;
    d_.part = part;
    d_.part_k = part_k;
    d_.err = derr;
    TCG_TRY(cudaMemsetAsync(derr, 0, sizeof(int), stream_));
    TCG_TRY(cudaMemsetAsync(part, 0, sizeof(double) * 4 * n1_, stream_));

    const T* dG = static_cast<const T*>(G);
    const uint8_t* dM = mask;
    void* tG = nullptr;
    void* tM = nullptr;
    if (!on_device) {
      TCG_TRY(cudaMalloc(&tG, N * sizeof(T)));
      TCG_TRY(cudaMalloc(&tM, N));
      TCG_TRY(cudaMemcpyAsync(tG, G, N * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TCG_TRY(cudaMemcpyAsync(tM, mask, N, cudaMemcpyHostToDevice, stream_));
      dG = static_cast<const T*>(tG);
      dM = static_cast<const uint8_t*>(tM);
    }
    k_pack<T><<<n1_ * n3_, 256, 0, stream_>>>(dG, dM, Gint, maskbits, n1_, n2_, n3_, mw);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t se = cudaStreamSynchronize(stream_);
    if (tG) cudaFree(tG);
    if (tM) cudaFree(tM);
    if (le != cudaSuccess || se != cudaSuccess) {
      err = std::string("initialisation kernels failed: ") + cudaGetErrorString(le != cudaSuccess ? le : se);
      return TC_ERR_CUDA;
    }
    return TC_OK;
  }

  // loss (always) and the spatial gradients (when dX / dY are given)
  tc_status eval(const void* X, const void* Y, double* loss, void* dX, void* dY, bool on_device,
                 std::string& err) override {
    const size_t nx = (size_t)n1_ * r_ * n3_, ny = (size_t)r_ * n2_ * n3_;
    const T* xs = static_cast<const T*>(X);
    const T* ys = static_cast<const T*>(Y);
    if (!on_device) {
      TCG_TRY(cudaMemcpyAsync(xin_, X, nx * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TCG_TRY(cudaMemcpyAsync(yin_, Y, ny * sizeof(T), cudaMemcpyHostToDevice, stream_));
      xs = xin_;
      ys = yin_;
    }
    const int fgrid = 4 * 152;
    k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(xs, d_.Xt, n1_, r_, n3_, 0, d_.twg);
    k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(ys, d_.Yt, n2_, r_, n3_, 1, d_.twg);
    {
      const size_t tot = (size_t)n1_ * S_ * n2_;
      k_synth_init<T><<<(unsigned)std::min<size_t>((tot + 255) / 256, 8 * 152), 256, 0, stream_>>>(d_);
    }
    slab_.f<<<n1_, slab_.threads, slab_.smem, stream_>>>(d_, nullptr, slab_.in_smem ? 1 : 0, 0);  // R~, ||E||^2
    if (d_.rho1 != T(0)) k_rho1_term<T><<<dim3(S_, kRhoChunks), 256, 0, stream_>>>(d_);  // ||H Z~_k||^2 from Z~
    if (dX || dY) {
      if (d_.rho1 != T(0)) {
        // R~ += rho1 H^T H Z~: the contractions below then carry the rho1 term too
        const size_t tot = (size_t)n1_ * S_ * n2_;
        k_grad_hth<T><<<(unsigned)std::min<size_t>((tot + 255) / 256, 16 * 152), 256, 0, stream_>>>(d_);
      }
      qcon_<<<dim3(S_, (n1_ + 31) / 32), kSliceThreads, qsmem_, stream_>>>(d_, GX_);  // R~ Y~^H
      dcon_<<<dim3(S_, (n2_ + 31) / 32), kYThreads, dsmem_, stream_>>>(d_, GY_);     // X~^H R~
      T* ox = static_cast<T*>(dX);
      T* oy = static_cast<T*>(dY);
      if (!on_device) {
        ox = dX ? xin_ : nullptr;
        oy = dY ? yin_ : nullptr;
      }
      if (ox) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(GX_, ox, n1_, r_, n3_, 0, d_.twg);
      if (oy) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(GY_, oy, n2_, r_, n3_, 1, d_.twg);
      if (!on_device) {
        if (dX) TCG_TRY(cudaMemcpyAsync(dX, xin_, nx * sizeof(T), cudaMemcpyDeviceToHost, stream_));
        if (dY) TCG_TRY(cudaMemcpyAsync(dY, yin_, ny * sizeof(T), cudaMemcpyDeviceToHost, stream_));
      }
    }
    TCG_TRY(cudaGetLastError());
    std::vector<double> part(4 * (size_t)n1_), pk((size_t)S_ * kRhoChunks);
    TCG_TRY(cudaMemcpyAsync(part.data(), d_.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    if (d_.rho1 != T(0))
      TCG_TRY(cudaMemcpyAsync(pk.data(), d_.part_k, pk.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    int herr = 0;
    TCG_TRY(cudaMemcpyAsync(&herr, d_.err, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    TCG_TRY(cudaStreamSynchronize(stream_));
    if (herr != DEV_OK) {
      err = "device-side check failed (code " + std::to_string(herr) + ")";
      return TC_ERR_CUDA;
    }
    double e2 = 0.0;
    for (int i = 0; i < n1_; ++i) e2 += part[4 * (size_t)i];
    double h2 = 0.0;  // sum over all n3 slices of ||H Z~_k||^2 (half spectrum, mirrored slices twice)
    if (d_.rho1 != T(0))
      for (int k = 0; k < S_; ++k) {
        double v = 0.0;
        for (int q = 0; q < kRhoChunks; ++q) v += pk[(size_t)k * kRhoChunks + q];
        h2 += ((k == 0 || 2 * k == n3_) ? 1.0 : 2.0) * v;
      }
    const double f = 0.5 * e2 + 0.5 * (double)d_.rho1 * h2 / (double)n3_;
    if (!std::isfinite(f)) {
      err = "loss is not finite";
      return TC_ERR_NUMERIC;
    }
    *loss = f;
    return TC_OK;
  }

  cudaStream_t stream_ = nullptr;
  int n1_ = 0, n2_ = 0, n3_ = 0, r_ = 0, S_ = 0, rp_ = 8;
  Dev<T> d_{};
  GradSlab<T> slab_;
  GFn<T> qcon_ = nullptr;
  GFn<T> dcon_ = nullptr;
  size_t qsmem_ = 0, dsmem_ = 0;
  cx<T>* GX_ = nullptr;
  cx<T>* GY_ = nullptr;
  T* xin_ = nullptr;
  T* yin_ = nullptr;
  std::vector<void*> allocs_;
};

}  // namespace

extern "C" {

tc_status tc_grad_init(tc_grad** out, const tc_params* p, const void* G, const uint8_t* mask,
                       int32_t inputs_on_device, void* cuda_stream) {
  if (!out) {
    tc::set_last_error("out is NULL");
    return TC_ERR_ARG;
  }
  *out = nullptr;
  if (!p || !G || !mask) {
    tc::set_last_error("params, G and mask are required");
    return TC_ERR_ARG;
  }
  if (p->n1 < 1 || p->n2 < 1 || p->n3 < 1 || p->n2 > 4096 || p->n3 > 4096 || p->n1 > (1 << 24) ||
      (double)p->n1 * (double)p->n2 * (double)p->n3 > 4.0e9 || p->r < 1 || p->r > 32 || p->r > p->n1 ||
      p->r > p->n2) {
    tc::set_last_error("sizes out of range (those of tc_init)");
    return TC_ERR_ARG;
  }
  if (!(p->rho1 >= 0) || !std::isfinite(p->rho1)) {
    tc::set_last_error("rho1 must be finite and >= 0");
    return TC_ERR_ARG;
  }
  if (p->precision != TC_FP64 && p->precision != TC_FP32) {
    tc::set_last_error("precision not built for the differentiation form");
    return TC_ERR_UNSUPPORTED;
  }
  std::string err;
  tc_status st;
  tc_grad* g = nullptr;
  if (p->precision == TC_FP64) {
    auto* e = new (std::nothrow) GradEngine<double>();
    if (!e) return TC_ERR_NOMEM;
    st = e->init(*p, G, mask, inputs_on_device != 0, static_cast<cudaStream_t>(cuda_stream), err);
    g = e;
  } else {
    auto* e = new (std::nothrow) GradEngine<float>();
    if (!e) return TC_ERR_NOMEM;
    st = e->init(*p, G, mask, inputs_on_device != 0, static_cast<cudaStream_t>(cuda_stream), err);
    g = e;
  }
  if (st != TC_OK) {
    delete g;
    tc::set_last_error(err);
    return st;
  }
  *out = g;
  return TC_OK;
}

tc_status tc_grad_eval(tc_grad* g, const void* X, const void* Y, double* loss, void* dX, void* dY,
                       int32_t on_device) {
  if (!g || !X || !Y || !loss) {
    tc::set_last_error("g, X, Y and loss are required");
    return TC_ERR_ARG;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  std::string err;
  tc_status st = g->eval(X, Y, loss, dX, dY, on_device != 0, err);
  if (prev != g->device) cudaSetDevice(prev);
  if (st != TC_OK) tc::set_last_error(err);
  return st;
}

tc_status tc_grad_free(tc_grad* g) {
  if (!g) return TC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  const int dev = g->device;
  if (prev != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  delete g;
  if (prev != dev) cudaSetDevice(prev);
  return TC_OK;
}

}  // extern "C"
