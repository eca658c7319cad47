// Host engine of one precision: owns the device state of a context, launches
// the kernels of tc_kernels.cuh and captures one iteration as a CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tc_engine.h"
#include "tc_kernels.cuh"

namespace tc {

#define TC_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      err = std::string(#expr) + ": " + cudaGetErrorString(e_);                 \
      poisoned_ = true;                                                          \
      return (e_ == cudaErrorMemoryAllocation) ? TC_ERR_NOMEM : TC_ERR_CUDA;     \
    }                                                                            \
  } while (0)

template <typename T>
using SlabFn = void (*)(Dev<T>, T*, int);

// Slab-kernel instances per specialised tube length (L = 0: generic).
template <typename T, int L>
inline void slab_table(SlabFn<T> f[4]) {
  f[MODE_ITER] = k_slab<T, L, MODE_ITER>;
  f[MODE_INIT] = k_slab<T, L, MODE_INIT>;
  f[MODE_W] = k_slab<T, L, MODE_W>;
  f[MODE_R] = k_slab<T, L, MODE_R>;
}

// Which register-FFT lengths each precision instantiates.
template <typename T>
bool pick_slab(int n3, SlabFn<T> f[4]);

template <typename T>
using YFn = void (*)(Dev<T>);

template <typename T>
inline YFn<T> pick_ystep(int r, int* rp) {
  if (r <= 2) { *rp = 2; return k_ystep<T, 2>; }
  if (r <= 4) { *rp = 4; return k_ystep<T, 4>; }
  if (r <= 8) { *rp = 8; return k_ystep<T, 8>; }
  if (r <= 16) { *rp = 16; return k_ystep<T, 16>; }
  *rp = 32;
  return k_ystep<T, 32>;
}

template <typename T>
void upload_twiddles(cudaStream_t s);

template <typename T>
class Engine final : public EngineBase {
 public:
  ~Engine() override { release(); }

  void release() override {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    cap_stream_ = nullptr;
    for (void* p : allocs_) cudaFree(p);
    allocs_.clear();
  }

  tc_status init(const tc_params& p, const void* G, const uint8_t* mask, const void* Y0, const void* X0,
                 bool on_device, cudaStream_t stream, std::string& err) override {
    p_ = p;
    stream_ = stream;
    n1_ = (int)p.n1;
    n2_ = (int)p.n2;
    n3_ = (int)p.n3;
    r_ = p.r;
    S_ = n3_ / 2 + 1;
    words_ = (n2_ + 31) / 32;
    const size_t N = (size_t)n1_ * n2_ * n3_;
    TC_CUDA_TRY(cudaGetDevice(&device_));
    int optin = 0;
    TC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device_));
    upload_twiddles<T>(stream_);
    TC_CUDA_TRY(cudaGetLastError());

    // ---- state buffers ---------------------------------------------------------
    T* Gint = alloc<T>(N, err);
    uint32_t* maskbits = alloc<uint32_t>((size_t)n1_ * n3_ * words_, err);
    cx<T>* Rt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    cx<T>* Xt = alloc<cx<T>>((size_t)S_ * r_ * n1_, err);
    cx<T>* Q = alloc<cx<T>>((size_t)S_ * r_ * n1_, err);
    cx<T>* Tb = alloc<cx<T>>((size_t)S_ * r_ * n1_, err);
    cx<T>* Yt = alloc<cx<T>>((size_t)S_ * r_ * n2_, err);
    cx<T>* Mm = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
    cx<T>* Gp = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
    T* winv = alloc<T>((size_t)2 * n2_, err);
    T* hinv = alloc<T>((size_t)n1_, err);
    cx<T>* twg = alloc<cx<T>>((size_t)n3_, err);
    double* part = alloc<double>((size_t)n1_ * 4, err);
    double* part_k = alloc<double>((size_t)S_, err);
    int* derr = alloc<int>(1, err);
    if (!err.empty()) return TC_ERR_NOMEM;

    // ---- slab kernel choice and shared memory -------------------------------------
    specialised_ = pick_slab<T>(n3_, slab_) && ((n2_ + 31) / 32 * 32 <= kSlabMaxThreads);
    if (!specialised_) slab_table<T, 0>(slab_);
    slab_threads_ = specialised_ ? (n2_ + 31) / 32 * 32 : 256;
    SlabLayout lay = slab_layout<T>(n2_, n3_, r_, specialised_, true);
    slabs_in_smem_ = lay.total <= (size_t)optin;
    if (!slabs_in_smem_) {
      lay = slab_layout<T>(n2_, n3_, r_, specialised_, false);
      T* scratch = alloc<T>(lay.slab_bytes / sizeof(T) * (size_t)n1_ + 16, err);
      if (!err.empty()) return TC_ERR_NOMEM;
      d_.scratch = scratch;
    } else {
      d_.scratch = nullptr;
    }
    slab_smem_ = lay.total;
    for (int m = 0; m < 4; ++m)
      TC_CUDA_TRY(cudaFuncSetAttribute(slab_[m], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab_smem_));
    xstep_smem_ = xstep_smem_bytes<T>(r_);
    TC_CUDA_TRY(cudaFuncSetAttribute(k_xstep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xstep_smem_));
    ystep_ = pick_ystep<T>(r_, &rp_);
    ystep_smem_ = (size_t)(kYThreads / 32 + 2) * rp_ * 32 * sizeof(cx<T>);
    TC_CUDA_TRY(cudaFuncSetAttribute(ystep_, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ystep_smem_));

    // ---- host tables (FP64, rounded to T) -------------------------------------------
    {
      const double mu = p.mu, rho1 = p.rho1, rho2 = p.rho2;
      std::vector<T> w(2 * (size_t)n2_);
      // runs starting at j = 0 (first entry has one neighbour when n2 > 1)
      double inv = 1.0 / (1.0 + mu + rho2 * (n2_ > 1 ? 1.0 : 0.0));
      w[0] = (T)inv;
      for (int q = 1; q < n2_; ++q) {
        inv = 1.0 / (1.0 + mu + 2.0 * rho2 - rho2 * rho2 * inv);
        w[q] = (T)inv;
      }
      inv = 1.0 / (1.0 + mu + 2.0 * rho2);
      w[n2_] = (T)inv;
      for (int q = 1; q < n2_; ++q) {
        inv = 1.0 / (1.0 + mu + 2.0 * rho2 - rho2 * rho2 * inv);
        w[n2_ + q] = (T)inv;
      }
      std::vector<T> h(n1_);
      // H_rho1 = I + rho1 H^T H: diagonal 1 + rho1 deg_i, off-diagonal -rho1
      double hi = 0.0;
      for (int i = 0; i < n1_; ++i) {
        const int deg = (i > 0) + (i + 1 < n1_);
        const double den = 1.0 + rho1 * deg - (i > 0 ? rho1 * rho1 * hi : 0.0);
        hi = 1.0 / den;
        h[i] = (T)hi;
      }
      std::vector<cx<T>> tw(n3_);
      for (int m = 0; m < n3_; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)n3_;
        tw[m] = cx<T>{(T)std::cos(a), (T)(-std::sin(a))};
      }
      TC_CUDA_TRY(cudaMemcpyAsync(winv, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaMemcpyAsync(hinv, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaMemcpyAsync(twg, tw.data(), tw.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaStreamSynchronize(stream_));  // host vectors go out of scope
    }

    d_.n1 = n1_;
    d_.n2 = n2_;
    d_.n3 = n3_;
    d_.S = S_;
    d_.r = r_;
    d_.words = words_;
    d_.mu = (T)p.mu;
    d_.rho1 = (T)p.rho1;
    d_.rho2 = (T)p.rho2;
    d_.G = Gint;
    d_.mask = maskbits;
    d_.Rt = Rt;
    d_.Xt = Xt;
    d_.Yt = Yt;
    d_.Q = Q;
    d_.Tb = Tb;
    d_.Mm = Mm;
    d_.Gp = Gp;
    d_.winv = winv;
    d_.hinv = hinv;
    d_.twg = twg;
    d_.part = part;
    d_.part_k = part_k;
    d_.err = derr;
    d_.rtol = (p.pinv_rtol > 0) ? p.pinv_rtol : (double)r_ * 2.220446049250313e-16;
    d_.pinv_fallbacks_enabled = 1;
    TC_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(int), stream_));

    // ---- inputs ------------------------------------------------------------------------
    const T* dG = static_cast<const T*>(G);
    const uint8_t* dM = mask;
    const T* dY = static_cast<const T*>(Y0);
    const T* dX = static_cast<const T*>(X0);
    std::vector<void*> tmp;
    auto stage = [&](const void* src, size_t bytes) -> void* {
      void* dst = nullptr;
      if (cudaMalloc(&dst, bytes) != cudaSuccess) return nullptr;
      tmp.push_back(dst);
      if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream_) != cudaSuccess) return nullptr;
      return dst;
    };
    if (!on_device) {
      dG = static_cast<const T*>(stage(G, N * sizeof(T)));
      dM = static_cast<const uint8_t*>(stage(mask, N));
      dY = static_cast<const T*>(stage(Y0, (size_t)r_ * n2_ * n3_ * sizeof(T)));
      dX = X0 ? static_cast<const T*>(stage(X0, (size_t)n1_ * r_ * n3_ * sizeof(T))) : nullptr;
      if (!dG || !dM || !dY || (X0 && !dX)) {
        for (void* q : tmp) cudaFree(q);
        err = "staging of host inputs failed";
        return TC_ERR_NOMEM;
      }
    }
    k_pack<T><<<n1_ * n3_, 256, 0, stream_>>>(dG, dM, Gint, maskbits, n1_, n2_, n3_, words_);
    const int fgrid = 4 * 152;
    k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(dY, Yt, n2_, r_, n3_, 1);
    if (dX) {
      k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(dX, Xt, n1_, r_, n3_, 0);
    } else {
      cudaMemsetAsync(Xt, 0, (size_t)S_ * r_ * n1_ * sizeof(cx<T>), stream_);
    }
    launch_slab(MODE_INIT, nullptr, stream_);
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(stream_);
    for (void* q : tmp) cudaFree(q);
    if (le != cudaSuccess || se != cudaSuccess) {
      err = std::string("initialisation kernels failed: ") + cudaGetErrorString(le != cudaSuccess ? le : se);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    return check_dev_err(err);
  }

  tc_status iterate(int n, int* done, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    if (n > 0 && !graph_exec_) {
      tc_status st = capture(err);
      if (st != TC_OK) return st;
    }
    for (int i = 0; i < n; ++i) TC_CUDA_TRY(cudaGraphLaunch(graph_exec_, stream_));
    if (done) *done = n;
    return TC_OK;
  }

  tc_status objective(double* f0, double* resid_obs, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    launch_slab(MODE_R, nullptr, stream_);
    launch_slab(MODE_W, nullptr, stream_);
    k_rho1_term<T><<<S_, 256, 0, stream_>>>(d_);
    TC_CUDA_TRY(cudaGetLastError());
    std::vector<double> part((size_t)n1_ * 4), pk(S_);
    TC_CUDA_TRY(cudaMemcpyAsync(part.data(), d_.part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    TC_CUDA_TRY(cudaMemcpyAsync(pk.data(), d_.part_k, pk.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
    TC_CUDA_TRY(cudaStreamSynchronize(stream_));
    tc_status st = check_dev_err(err);
    if (st != TC_OK) return st;
    double sr = 0, so = 0, sw = 0, sk = 0, sh = 0;
    for (int i = 0; i < n1_; ++i) {
      sr += part[(size_t)i * 4 + 0];
      so += part[(size_t)i * 4 + 1];
      sw += part[(size_t)i * 4 + 2];
      sk += part[(size_t)i * 4 + 3];
    }
    for (int k = 0; k < S_; ++k) {
      const double c = (k == 0 || 2 * k == n3_) ? 1.0 : 2.0;
      sh += c * pk[k];
    }
    const double f = 0.5 * sr + 0.5 * p_.mu * sw + 0.5 * p_.rho2 * sk + 0.5 * p_.rho1 * sh / (double)n3_;
    *f0 = f;
    if (resid_obs) *resid_obs = std::sqrt(so);
    if (!std::isfinite(f)) {
      err = "objective is not finite";
      return TC_ERR_NUMERIC;
    }
    return TC_OK;
  }

  tc_status result(void* W, void* X, void* Y, bool on_device, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    const size_t N = (size_t)n1_ * n2_ * n3_;
    const size_t nx = (size_t)n1_ * r_ * n3_, ny = (size_t)r_ * n2_ * n3_;
    T* dW = nullptr;
    T* dXo = nullptr;
    T* dYo = nullptr;
    std::vector<void*> tmp;
    auto dev_buf = [&](void* user, size_t elems) -> T* {
      if (!user) return nullptr;
      if (on_device) return static_cast<T*>(user);
      void* q = nullptr;
      if (cudaMalloc(&q, elems * sizeof(T)) != cudaSuccess) return nullptr;
      tmp.push_back(q);
      return static_cast<T*>(q);
    };
    dW = dev_buf(W, N);
    dXo = dev_buf(X, nx);
    dYo = dev_buf(Y, ny);
    if ((W && !dW) || (X && !dXo) || (Y && !dYo)) {
      for (void* q : tmp) cudaFree(q);
      err = "allocation of read-back buffers failed";
      return TC_ERR_NOMEM;
    }
    if (dW) launch_slab(MODE_W, dW, stream_);
    const int fgrid = 4 * 152;
    if (dXo) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(d_.Xt, dXo, n1_, r_, n3_, 0);
    if (dYo) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(d_.Yt, dYo, n2_, r_, n3_, 1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device) {
      if (W) e = cudaMemcpyAsync(W, dW, N * sizeof(T), cudaMemcpyDeviceToHost, stream_);
      if (e == cudaSuccess && X) e = cudaMemcpyAsync(X, dXo, nx * sizeof(T), cudaMemcpyDeviceToHost, stream_);
      if (e == cudaSuccess && Y) e = cudaMemcpyAsync(Y, dYo, ny * sizeof(T), cudaMemcpyDeviceToHost, stream_);
    }
    cudaError_t se = cudaStreamSynchronize(stream_);
    for (void* q : tmp) cudaFree(q);
    if (e != cudaSuccess || se != cudaSuccess) {
      err = std::string("read-back failed: ") + cudaGetErrorString(e != cudaSuccess ? e : se);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    return check_dev_err(err);
  }

  tc_status profile(int n, double* ms, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    cudaEvent_t ev[4];
    for (int i = 0; i < 4; ++i) TC_CUDA_TRY(cudaEventCreate(&ev[i]));
    double acc[3] = {0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n && e == cudaSuccess; ++it) {
      cudaEventRecord(ev[0], stream_);
      k_xstep<T><<<S_, kSliceThreads, xstep_smem_, stream_>>>(d_);
      cudaEventRecord(ev[1], stream_);
      dim3 yg(S_, (n2_ + 31) / 32);
      ystep_<<<yg, kYThreads, ystep_smem_, stream_>>>(d_);
      cudaEventRecord(ev[2], stream_);
      launch_slab(MODE_ITER, nullptr, stream_);
      cudaEventRecord(ev[3], stream_);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
      for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
        acc[q] += t;
      }
    }
    for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) {
      err = std::string("profiled iteration failed: ") + cudaGetErrorString(e);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    for (int q = 0; q < 3; ++q) ms[q] = acc[q] / n;
    return check_dev_err(err);
  }

 private:
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

  void launch_slab(int mode, T* Wout, cudaStream_t s) {
    slab_[mode]<<<n1_, slab_threads_, slab_smem_, s>>>(d_, Wout, slabs_in_smem_ ? 1 : 0);
  }

  void launch_iteration(cudaStream_t s) {
    k_xstep<T><<<S_, kSliceThreads, xstep_smem_, s>>>(d_);
    dim3 yg(S_, (n2_ + 31) / 32);
    ystep_<<<yg, kYThreads, ystep_smem_, s>>>(d_);
    launch_slab(MODE_ITER, nullptr, s);
  }

  tc_status capture(std::string& err) {
    if (!cap_stream_) TC_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    TC_CUDA_TRY(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
    launch_iteration(cap_stream_);
    cudaError_t le = cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(cap_stream_, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      err = std::string("graph capture failed: ") + cudaGetErrorString(le != cudaSuccess ? le : ce);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&graph_exec_, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      err = std::string("graph instantiation failed: ") + cudaGetErrorString(ie);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    return TC_OK;
  }

  tc_status check_dev_err(std::string& err) {
    int h = 0;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, d_.err, sizeof(int), cudaMemcpyDeviceToHost, stream_));
    TC_CUDA_TRY(cudaStreamSynchronize(stream_));
    if (h != DEV_OK) {
      err = "device-side check failed (code " + std::to_string(h) + ")";
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    return TC_OK;
  }

  tc_params p_{};
  cudaStream_t stream_ = nullptr;
  cudaStream_t cap_stream_ = nullptr;
  cudaGraphExec_t graph_exec_ = nullptr;
  int device_ = 0;
  int n1_ = 0, n2_ = 0, n3_ = 0, r_ = 0, S_ = 0, words_ = 0;
  bool poisoned_ = false;
  bool specialised_ = false;
  bool slabs_in_smem_ = true;
  int slab_threads_ = 256;
  size_t slab_smem_ = 0, xstep_smem_ = 0, ystep_smem_ = 0;
  int rp_ = 8;
  SlabFn<T> slab_[4] = {nullptr, nullptr, nullptr, nullptr};
  YFn<T> ystep_ = nullptr;
  Dev<T> d_{};
  std::vector<void*> allocs_;
};

}  // namespace tc
