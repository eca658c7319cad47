// Host engine of one precision: owns the device state of a context, launches
// the kernels and captures one iteration (four kernels) as a CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <limits>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
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
using SlabFn = void (*)(Dev<T>, T*, int, int);

template <typename T, int L>
inline void slab_table(SlabFn<T> f[3]) {
  f[MODE_ITER] = k_slab<T, L, MODE_ITER>;
  f[MODE_W] = k_slab<T, L, MODE_W>;
  f[MODE_R] = k_slab<T, L, MODE_R>;
}

// Generic-length slab kernels with TL rows / slices per transform item.
template <typename T, int TL>
inline void slab_table_tl(SlabFn<T> f[3]) {
  f[MODE_ITER] = k_slab<T, 0, MODE_ITER, TL>;
  f[MODE_W] = k_slab<T, 0, MODE_W, TL>;
  f[MODE_R] = k_slab<T, 0, MODE_R, TL>;
}

template <typename T, int L, int N1, int N2>
inline void slab_f_table(SlabFn<T> f[3]) {
  f[MODE_ITER] = k_slab_f<T, L, N1, N2, MODE_ITER>;
  f[MODE_W] = k_slab_f<T, L, N1, N2, MODE_W>;
  f[MODE_R] = k_slab_f<T, L, N1, N2, MODE_R>;
}

// Launch configuration of the slab kernel.
template <typename T>
struct SlabCfg {
  SlabFn<T> f[3];
  int threads;
  size_t smem;
};

// Slab kernels specialised for the tube length n3, instantiated per precision
// (defined per translation unit); false when none applies to (n2, n3) within
// the shared-memory limit optin.
template <typename T>
bool pick_slab(int n2, int n3, int optin, SlabCfg<T>& cfg);

template <typename T>
using YFn = void (*)(Dev<T>);
template <typename T>
using QFn = void (*)(Dev<T>, cx<T>*);

template <typename T>
inline int pad_rank(int r) {
  return r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : r <= 16 ? 16 : 32;
}

// xsh: X~' of the slice staged in shared memory (r n1 fits), else read through L1
template <typename T>
inline YFn<T> pick_ystep(int rp, bool xsh = true) {
  switch (rp) {
    case 2: return xsh ? k_ystep<T, 2, false, true> : k_ystep<T, 2, false, false>;
    case 4: return xsh ? k_ystep<T, 4, false, true> : k_ystep<T, 4, false, false>;
    case 8: return xsh ? k_ystep<T, 8, false, true> : k_ystep<T, 8, false, false>;
    case 16: return xsh ? k_ystep<T, 16, false, true> : k_ystep<T, 16, false, false>;
    default: return xsh ? k_ystep<T, 32, false, true> : k_ystep<T, 32, false, false>;
  }
}

template <typename T>
using XFn = void (*)(Dev<T>, const cx<T>*, int);

// Type of the r x r solves: FP64 storage (df64 arithmetic, see
// gauss_jordan_inplace_df) in an FP32 engine for r > 16, whose Grams (the DC
// slice above all) are too ill-conditioned for an FP32 inverse, and for every
// r in the precision form; the working precision otherwise.
template <typename T>
inline bool solve64(int rp, bool mixed) {
  return sizeof(T) == 4 && (mixed || rp == 32);
}

// Default cutoff of the pseudo-inverse: r times the epsilon of the solve type.
template <typename T>
inline double default_rtol(int r, int rp, bool mixed) {
  return (double)r * (solve64<T>(rp, mixed) ? std::numeric_limits<double>::epsilon()
                                             : (double)std::numeric_limits<T>::epsilon());
}

template <typename T>
inline XLayout xstep_layout_for(int n1, int n2, int r, int rp, bool mixed, bool in_smem) {
  return solve64<T>(rp, mixed) ? xstep_layout<T, double>(n1, n2, r, in_smem) : xstep_layout<T>(n1, n2, r, in_smem);
}

template <typename T, typename TS = T>
inline XFn<T> pick_xstep(int rp) {
  switch (rp) {
    case 2: return k_xstep<T, 2, TS>;
    case 4: return k_xstep<T, 4, TS>;
    case 8: return k_xstep<T, 8, TS>;
    case 16: return k_xstep<T, 16, TS>;
    default: return k_xstep<T, 32, TS>;
  }
}

// Tensor-core Q contraction of the precision form (TC_TF32 / TC_BF16 over
// FP32 data, r > 16): the kernel and its dynamic shared memory, or nullptr
// where it is not built (FP64 data).
template <typename T>
inline XFn<T> pick_xstep_for(int rp, bool mixed) {
  return solve64<T>(rp, mixed) ? pick_xstep<T, double>(rp) : pick_xstep<T>(rp);
}

// Tensor-core kernels of the precision form (TC_TF32 / TC_BF16 over FP32
// data, r > 16): Q contraction, partial D of the Y-step, Z~ synthesis, with
// their dynamic shared memory.  False where they are not built (FP64 data).
template <typename T>
struct TcKernels {
  QFn<T> qcon = nullptr;
  YFn<T> dcon = nullptr, zsyn = nullptr;
  size_t qsm = 0, dsm = 0, zsm = 0;
};
template <typename T>
bool pick_tc(int precision, bool split, TcKernels<T>& k);
template <>
bool pick_tc<float>(int precision, bool split, TcKernels<float>& k);
template <>
bool pick_tc<double>(int precision, bool split, TcKernels<double>& k);

template <typename T>
inline QFn<T> pick_qcon(int rp) {
  switch (rp) {
    case 2: return k_qcon<T, 2>;
    case 4: return k_qcon<T, 4>;
    case 8: return k_qcon<T, 8>;
    case 16: return k_qcon<T, 16>;
    default: return k_qcon<T, 32>;
  }
}

template <typename T>
void upload_twiddles();

template <typename T>
class Engine final : public EngineBase {
 public:
  ~Engine() override { release(); }

  void release() override {
    if (graph_exec_) cudaGraphExecDestroy(graph_exec_);
    graph_exec_ = nullptr;
    if (cap_stream_) cudaStreamDestroy(cap_stream_);
    cap_stream_ = nullptr;
    if (aux_stream_) cudaStreamDestroy(aux_stream_);
    aux_stream_ = nullptr;
    for (cudaEvent_t* e : {&ev_fork_, &ev_join_}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
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
    mw_ = (n2_ + 31) / 32;  // mask words per row
    rp_ = pad_rank<T>(r_);
    const size_t N = (size_t)n1_ * n2_ * n3_;
    TC_CUDA_TRY(cudaGetDevice(&device_));
    int optin = 0;
    TC_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device_));
    optin -= kStaticSmemReserve;  // room for the kernels' static shared memory
    upload_twiddles<T>();
    TC_CUDA_TRY(cudaGetLastError());

    // ---- state buffers -----------------------------------------------------------
    const size_t nx = (size_t)S_ * r_ * n1_, ny = (size_t)S_ * r_ * n2_, nrr = (size_t)S_ * r_ * r_;
    T* Gint = alloc<T>(N, err);
    uint32_t* maskbits = alloc<uint32_t>((size_t)n1_ * n3_ * mw_, err);
    cx<T>* Rt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    cx<T>* Zt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    const int ytiles = (n2_ + 31) / 32;
    cx<double>* Ag = alloc<cx<double>>((size_t)S_ * ytiles * (r_ * (r_ + 1) / 2), err);
    cx<T>* Xt = alloc<cx<T>>(nx, err);
    Q_ = alloc<cx<T>>(nx, err);
    cx<T>* Tb = alloc<cx<T>>(nx, err);
    cx<T>* Yt = alloc<cx<T>>(ny, err);
    cx<T>* Dg = alloc<cx<T>>(nrr, err);
    cx<T>* Gp = alloc<cx<T>>(nrr, err);
    // FP64 t G^+ of the real slices (DC, Nyquist) of an FP32 engine
    cx<double>* Gp64 = sizeof(T) == 4 ? alloc<cx<double>>((size_t)2 * r_ * r_, err) : nullptr;
    T* winv = alloc<T>((size_t)6 * n2_, err);
    T* hinv = alloc<T>((size_t)2 * n1_, err);
    cx<T>* twg = alloc<cx<T>>((size_t)n3_, err);
    double* part = alloc<double>((size_t)n1_ * 4, err);
    double* part_k = alloc<double>((size_t)S_ * kRhoChunks, err);
    int* derr = alloc<int>(1, err);
    // stopping test (eps > 0): change maxima, flag, counter; |dW| partial sums; Z~ changes
    unsigned long long* conv = nullptr;
    double* part_dw = nullptr;
    cx<T>* dZt = nullptr;
    if (p.eps > 0) {
      conv = alloc<unsigned long long>(8, err);
      part_dw = alloc<double>((size_t)n1_, err);
      dZt = alloc<cx<T>>((size_t)n1_ * S_ * n2_, err);
    }
    if (!err.empty()) return TC_ERR_NOMEM;
    if (conv) TC_CUDA_TRY(cudaMemsetAsync(conv, 0, 8 * sizeof(unsigned long long), stream_));

    // ---- kernel variants and shared memory -------------------------------------------
    SlabCfg<T> cfg{};
    specialised_ = pick_slab<T>(n2_, n3_, optin, cfg);
    d_.scratch = nullptr;
    if (specialised_) {
      for (int m = 0; m < 3; ++m) slab_[m] = cfg.f[m];
      slab_threads_ = cfg.threads;
      slab_smem_ = cfg.smem;
      slabs_in_smem_ = true;
    } else {
      slab_table<T, 0>(slab_);
      slab_threads_ = 256;
      SlabLayout lay = slab_layout<T>(n2_, n3_, false, true);
      slabs_in_smem_ = lay.total <= (size_t)optin;
      if (!slabs_in_smem_) {
        lay = slab_layout<T>(n2_, n3_, false, false);
        T* scratch = alloc<T>(lay.slab_bytes / sizeof(T) * (size_t)n1_ + 16, err);
        if (!err.empty()) return TC_ERR_NOMEM;
        d_.scratch = scratch;
      }
      slab_smem_ = lay.total;
    }
    for (int m = 0; m < 3; ++m)
      TC_CUDA_TRY(allow_dynamic_smem((const void*)slab_[m], slab_smem_));

    // precision form: r x r solves in FP64, contractions on the tensor cores for r > 16
    mixed_ = p.precision == TC_TF32 || p.precision == TC_BF16;
    auto xlay = [&](bool in_smem) { return xstep_layout_for<T>(n1_, n2_, r_, rp_, mixed_, in_smem); };
    XLayout xl = xlay(true);
    xarrays_in_smem_ = xl.total <= (size_t)optin;
    if (!xarrays_in_smem_) xl = xlay(false);
    xstep_smem_ = xl.total;
    if (xstep_smem_ > (size_t)optin) {
      err = "X-step shared memory exceeds the device limit";
      return TC_ERR_UNSUPPORTED;
    }
    xstep_ = pick_xstep_for<T>(rp_, mixed_);
    TC_CUDA_TRY(allow_dynamic_smem((const void*)xstep_, xstep_smem_));
    // the X-step as four kernels spread over the GPU (k_xbg, k_xbc, k_xg, k_xc in
    // k_xsplit.cuh; A^+ by k_xa on a graph branch) for r > 8 in FP32 engines and
    // r > 16 in the FP64 engine; below that one CTA per slice is faster (the
    // r x r work is small and the extra launches and barriers dominate: 35 us
    // against 49 us for the 144 x 288 x 168, r = 8 workload)
    const bool s64 = solve64<T>(rp_, mixed_);
    // FP32 engines: room for the FP64 real-slice solve of k_xc (real_gram_solve_store)
    const size_t xa_bytes = (s64 || sizeof(T) == 4) ? xa_smem_bytes<double>(r_) : xa_smem_bytes<T>(r_);
    xsplit_ = (sizeof(T) == 4 ? rp_ >= 16 : rp_ == 32) && xbc_smem_bytes<T>(n1_) <= (size_t)optin &&
              xbg_smem_bytes<T>(r_) <= (size_t)optin &&
              xa_bytes <= (size_t)optin && xg_smem_bytes<T>(r_) <= (size_t)optin;
    // one-CTA X-step: A^+ of the next X-step formed by k_xa on a graph branch after
    // each Y-step (beside Z~ synthesis and the slab kernel), off the critical path
    apre_ = !xsplit_ && xa_bytes <= (size_t)optin;
    d_.apre = apre_ ? 1 : 0;
    if (apre_) {
      xa_threads_ = 64;
      while (xa_threads_ < r_ * r_ && xa_threads_ < kXaThreads) xa_threads_ *= 2;
      d_.Apg = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
      d_.Pg = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
      d_.certA = alloc<int>((size_t)S_, err);
      d_.tstep = alloc<T>((size_t)S_, err);
      if (!err.empty()) return TC_ERR_NOMEM;
      xa_smem_ = xa_bytes;
      xa_fn_ = s64 ? k_xa<T, double> : k_xa<T, T>;
      TC_CUDA_TRY(allow_dynamic_smem((const void*)xa_fn_, xa_smem_));
    }
    if (xsplit_) {
      gch_ = (n1_ + kXgRows - 1) / kXgRows;
      d_.gch = gch_;
      d_.Apg = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
      d_.Pg = alloc<cx<T>>((size_t)S_ * r_ * r_, err);
      d_.certA = alloc<int>((size_t)S_, err);
      d_.tstep = alloc<T>((size_t)S_, err);
      d_.Gpart = alloc<cx<T>>((size_t)S_ * gch_ * 3 * r_ * r_, err);
      if (!err.empty()) return TC_ERR_NOMEM;
      xa_smem_ = xa_bytes;
      xa_threads_ = kXaThreads;
      xa_fn_ = s64 ? k_xa<T, double> : k_xa<T, T>;
      xc_fn_ = s64 ? k_xc<T, double> : k_xc<T, T>;
      xbg_smem_ = xbg_smem_bytes<T>(r_);
      xbc_smem_ = xbc_smem_bytes<T>(n1_);
      xg_smem_ = xg_smem_bytes<T>(r_);
      TC_CUDA_TRY(allow_dynamic_smem((const void*)xa_fn_, xa_smem_));
      TC_CUDA_TRY(allow_dynamic_smem((const void*)xc_fn_, xa_smem_));
      TC_CUDA_TRY(allow_dynamic_smem((const void*)k_xbg<T>, xbg_smem_));
      TC_CUDA_TRY(allow_dynamic_smem((const void*)k_xbc<T>, xbc_smem_));
      TC_CUDA_TRY(allow_dynamic_smem((const void*)k_xg<T>, xg_smem_));
    }
    ystep_smem_ = ystep_smem_bytes<T>(n1_, r_, rp_);
    d_.yx_global = ystep_smem_ > (size_t)optin ? 1 : 0;
    if (d_.yx_global) ystep_smem_ = ystep_smem_bytes<T>(n1_, r_, rp_, false);
    ystep_ = pick_ystep<T>(rp_, !d_.yx_global);
    qcon_ = pick_qcon<T>(rp_);
    qcon_smem_ = qcon_smem_bytes<T>(n2_, r_, rp_);
    qgrid_ = dim3(S_, (n1_ + 31) / 32);
    qthreads_ = kSliceThreads;
    if (mixed_ && rp_ == 32 && pick_tc<T>(p.precision, (p.flags & TC_FLAG_SINGLE_PASS) == 0, tck_)) {
      tcy_ = true;
      qcon_ = tck_.qcon;
      qcon_smem_ = tck_.qsm;
      qgrid_ = dim3(S_, (n1_ + 127) / 128);
      qthreads_ = 256;
      ystep_ = k_ystep<T, 32, true>;
      ystep_smem_ = ystep_smem_bytes<T>(n1_, r_, rp_, false, true);
      // split the n1 reduction of D so that the grid covers the SMs about twice
      int nsm = 0;
      TC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device_));
      const int ntj = (n2_ + 127) / 128;
      ksplit_ = std::max(1, std::min((2 * nsm + S_ * ntj - 1) / (S_ * ntj), (n1_ + 31) / 32));
      d_.ksplit = ksplit_;
      Dpart_ = alloc<cx<T>>((size_t)S_ * ksplit_ * r_ * n2_, err);
      if (!err.empty()) return TC_ERR_NOMEM;
      d_.Dpart = Dpart_;
      if (tck_.dsm > (size_t)optin || tck_.zsm > (size_t)optin) {
        err = "shared memory of the tensor-core kernels exceeds the device limit";
        return TC_ERR_UNSUPPORTED;
      }
      TC_CUDA_TRY(allow_dynamic_smem((const void*)tck_.dcon, tck_.dsm));
      TC_CUDA_TRY(allow_dynamic_smem((const void*)tck_.zsyn, tck_.zsm));
    }
    if (ystep_smem_ > (size_t)optin || qcon_smem_ > (size_t)optin) {
      err = "shared memory of the slice kernels exceeds the device limit for these sizes";
      return TC_ERR_UNSUPPORTED;
    }
    TC_CUDA_TRY(allow_dynamic_smem((const void*)ystep_, ystep_smem_));
    TC_CUDA_TRY(allow_dynamic_smem((const void*)qcon_, qcon_smem_));

    // ---- host tables (FP64, rounded to T) ----------------------------------------------
    {
      const double mu = p.mu, rho1 = p.rho1, rho2 = p.rho2;
      // W-step runs: inverse LU pivots by position in the run
      std::vector<T> w(6 * (size_t)n2_);
      wstep_tables<T>(w.data(), n2_, mu, rho2);
      // H_rho1 = I + rho1 H^T H: diagonal 1 + rho1 deg_i, off-diagonal -rho1
      std::vector<T> h(2 * (size_t)n1_);
      double hi = 0.0;
      for (int i = 0; i < n1_; ++i) {
        const int deg = (i > 0) + (i + 1 < n1_);
        const double den = 1.0 + rho1 * deg - (i > 0 ? rho1 * rho1 * hi : 0.0);
        hi = 1.0 / den;
        h[i] = (T)hi;
        h[n1_ + i] = (T)(rho1 * hi);
      }
      std::vector<cx<T>> tw(n3_);
      for (int m = 0; m < n3_; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)n3_;
        tw[m] = cx<T>{(T)std::cos(a), (T)(-std::sin(a))};
      }
      TC_CUDA_TRY(cudaMemcpyAsync(winv, w.data(), w.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaMemcpyAsync(hinv, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaMemcpyAsync(twg, tw.data(), tw.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaStreamSynchronize(stream_));  // the host vectors go out of scope
    }

    d_.n1 = n1_;
    d_.n2 = n2_;
    d_.n3 = n3_;
    d_.S = S_;
    d_.r = r_;
    d_.mw = mw_;
    d_.mu = (T)p.mu;
    d_.rho1 = (T)p.rho1;
    d_.rho2 = (T)p.rho2;
    d_.G = Gint;
    d_.mask = maskbits;
    d_.Rt = Rt;
    d_.Zt = Zt;
    d_.Ag = Ag;
    d_.ytiles = ytiles;
    d_.Xt = Xt;
    d_.Yt = Yt;
    d_.Dg = Dg;
    d_.Gp = Gp;
    d_.Tb = Tb;
    d_.winv = winv;
    d_.hinv = hinv;
    d_.twg = twg;
    d_.part = part;
    d_.part_k = part_k;
    d_.err = derr;
    d_.rtol = (p.pinv_rtol > 0) ? p.pinv_rtol : default_rtol<T>(r_, rp_, mixed_);
    d_.rtol64 = (p.pinv_rtol > 0) ? p.pinv_rtol : (double)r_ * std::numeric_limits<double>::epsilon();
    d_.Gp64 = Gp64;
    d_.scaled = (p.step == TC_STEP_SCALED) ? 1 : 0;
    d_.alpha = (T)p.alpha;
    d_.beta = (T)p.beta;
    // ||H_rho1||_2 = 1 + rho1 lambda_max(H^T H); H^T H is the path Laplacian on n1
    // nodes with lambda_max = 2 + 2 cos(pi / n1)
    d_.hnorm = (T)(1.0 + p.rho1 * (n1_ > 1 ? 2.0 + 2.0 * std::cos(M_PI / (double)n1_) : 0.0));
    d_.conv = conv;
    d_.part_dw = part_dw;
    d_.dZt = dZt;
    d_.eps = p.eps;
    TC_CUDA_TRY(cudaMemsetAsync(derr, 0, sizeof(int), stream_));

    // ---- inputs --------------------------------------------------------------------------
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
        cudaStreamSynchronize(stream_);
        for (void* q : tmp) cudaFree(q);
        err = "staging of host inputs failed";
        return TC_ERR_NOMEM;
      }
    }
    k_pack<T><<<n1_ * n3_, 256, 0, stream_>>>(dG, dM, Gint, maskbits, n1_, n2_, n3_, mw_);
    const int fgrid = 4 * 152;
    k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(dY, Yt, n2_, r_, n3_, 1, twg);
    if (dX) {
      k_factor_dft<T><<<fgrid, 256, 0, stream_>>>(dX, Xt, n1_, r_, n3_, 0, twg);
    } else {
      cudaMemsetAsync(Xt, 0, nx * sizeof(cx<T>), stream_);
    }
    k_synth_init<T><<<fgrid, 256, 0, stream_>>>(d_);                    // Z~0 = X~0 Y~0
    k_gram_tiles<T><<<dim3(S_, ytiles), 256, 0, stream_>>>(d_);         // A of the first X-step
    if (xsplit_ || apre_) xa_fn_<<<S_, xa_threads_, xa_smem_, stream_>>>(d_);  // its A^+
    if (!specialised_) {
      // tile of the generic transform for this shape: each candidate runs the
      // initial slab pass (it only depends on G and Z~0, so every run writes the
      // same R~0), timed twice; the fastest is kept
      tc_status st = tune_slab_tile(err);
      if (st != TC_OK) return st;
    }
    launch_slab(MODE_ITER, nullptr, 1, stream_);  // R~0 = DFT3(P_Omega(G) - Z0)
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(stream_);
    for (void* q : tmp) cudaFree(q);
    if (le != cudaSuccess || se != cudaSuccess) {
      err = std::string("initialisation kernels failed: ") + cudaGetErrorString(le != cudaSuccess ? le : se);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    tc_status st = check_dev_err(err);
    if (st != TC_OK) return st;
    // the iteration graph is built and uploaded here, so that tc_iterate only
    // launches it
    st = capture(err);
    if (st != TC_OK) return st;
    TC_CUDA_TRY(cudaGraphUpload(graph_exec_, stream_));
    return TC_OK;
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
    unsigned long long h0[8] = {}, h1[8] = {};
    if (done && d_.conv) {
      tc_status st = read_conv(h0, err);
      if (st != TC_OK) return st;
    }
    for (int i = 0; i < n; ++i) TC_CUDA_TRY(cudaGraphLaunch(graph_exec_, stream_));
    if (done) {
      if (d_.conv) {
        tc_status st = read_conv(h1, err);
        if (st != TC_OK) return st;
        *done = (int)(h1[3] - h0[3]);  // iterations run before the stopping test fired
      } else {
        *done = n;
      }
    }
    return TC_OK;
  }

  tc_status convergence(double* changes, int* stopped, long long* iters_run, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    if (!d_.conv) {
      err = "the stopping test is off (eps = 0)";
      return TC_ERR_STATE;
    }
    unsigned long long h[8];
    tc_status st = read_conv(h, err);
    if (st != TC_OK) return st;
    for (int q = 0; q < 3; ++q) {
      double v;
      std::memcpy(&v, &h[4 + q], sizeof(double));
      changes[q] = v;
    }
    *stopped = h[2] != 0ull;
    *iters_run = (long long)h[3];
    return TC_OK;
  }

  tc_status objective(double* f0, double* resid_obs, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    launch_slab(MODE_R, nullptr, 0, stream_);
    launch_slab(MODE_W, nullptr, 0, stream_);
    k_rho1_term<T><<<dim3(S_, kRhoChunks), 256, 0, stream_>>>(d_);
    TC_CUDA_TRY(cudaGetLastError());
    std::vector<double> part((size_t)n1_ * 4), pk((size_t)S_ * kRhoChunks);
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
      double v = 0.0;
      for (int q = 0; q < kRhoChunks; ++q) v += pk[(size_t)k * kRhoChunks + q];
      sh += c * v;
    }
    // f0 of Eq. (TETP-optim): ||Z - W||^2 = ||R||^2; the rho1 term by Parseval
    // from the factors (Eq. (HunfZ2))
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
    std::vector<void*> tmp;
    auto dev_buf = [&](void* user, size_t elems) -> T* {
      if (!user) return nullptr;
      if (on_device) return static_cast<T*>(user);
      void* q = nullptr;
      if (cudaMalloc(&q, elems * sizeof(T)) != cudaSuccess) return nullptr;
      tmp.push_back(q);
      return static_cast<T*>(q);
    };
    T* dW = dev_buf(W, N);
    T* dXo = dev_buf(X, nx);
    T* dYo = dev_buf(Y, ny);
    if ((W && !dW) || (X && !dXo) || (Y && !dYo)) {
      for (void* q : tmp) cudaFree(q);
      err = "allocation of read-back buffers failed";
      return TC_ERR_NOMEM;
    }
    if (dW) launch_slab(MODE_W, dW, 0, stream_);
    const int fgrid = 4 * 152;
    if (dXo) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(d_.Xt, dXo, n1_, r_, n3_, 0, d_.twg);
    if (dYo) k_factor_idft<T><<<fgrid, 256, 0, stream_>>>(d_.Yt, dYo, n2_, r_, n3_, 1, d_.twg);
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

  tc_status capture_iteration(cudaGraph_t* out, std::string& err) override {
    if (!cap_stream_) TC_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream_, cudaStreamNonBlocking));
    *out = nullptr;
    const cudaError_t pre = cudaGetLastError();  // an error left by an earlier call of this thread
    if (pre != cudaSuccess) {
      err = std::string("pending error before graph capture: ") + cudaGetErrorString(pre);
      return TC_ERR_CUDA;
    }
    if ((xsplit_ || apre_) && !aux_stream_) {
      TC_CUDA_TRY(cudaStreamCreateWithFlags(&aux_stream_, cudaStreamNonBlocking));
      TC_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming));
      TC_CUDA_TRY(cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming));
    }
    TC_CUDA_TRY(cudaStreamBeginCapture(cap_stream_, cudaStreamCaptureModeThreadLocal));
    const char* at = "qcon";
    launch_qcon(cap_stream_);
    cudaError_t le = cudaPeekAtLastError();
    if (le == cudaSuccess) {
      at = "xstep";
      launch_xstep(cap_stream_);
      le = cudaPeekAtLastError();
    }
    bool forked = false;
    if (le == cudaSuccess) {
      at = "ystep";
      // with the four-kernel X-step, A^+ of the next iteration (k_xa) needs only
      // the tile Grams the Y-step writes: a branch of the graph beside the rest
      // of the iteration (Z~ synthesis, slab kernel)
      forked = launch_ystep(cap_stream_, (xsplit_ || apre_) ? aux_stream_ : nullptr);
      le = cudaPeekAtLastError();
    }
    if (le == cudaSuccess) {
      at = "slab";
      launch_slab(MODE_ITER, nullptr, 0, cap_stream_);
      le = cudaPeekAtLastError();
    }
    if (forked) {
      const cudaError_t je = cudaStreamWaitEvent(cap_stream_, ev_join_, 0);
      if (le == cudaSuccess) le = je;
    }
    if (le == cudaSuccess && d_.rk) {
      at = "rank";
      launch_rank(cap_stream_);  // step 5, after the A^+ branch has joined
      le = cudaPeekAtLastError();
    }
    if (le == cudaSuccess && d_.conv) {
      at = "check";
      k_check<T><<<1, 32, 0, cap_stream_>>>(d_);
      le = cudaPeekAtLastError();
    }
    cudaGetLastError();
    cudaError_t ce = cudaStreamEndCapture(cap_stream_, out);
    if (le != cudaSuccess || ce != cudaSuccess) {
      if (*out) cudaGraphDestroy(*out);
      *out = nullptr;
      err = std::string("graph capture failed (") + at + "): " + cudaGetErrorString(le != cudaSuccess ? le : ce);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    return TC_OK;
  }
  tc_status set_rank_rule(double tol, int patience, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    if (tol > 0.0 && !rk_) {
      rk_ = alloc<int>((size_t)S_, err);
      rcnt_ = alloc<int>((size_t)S_, err);
      rscr_ = alloc<cx<T>>((size_t)S_ * r_ * (n1_ + n2_), err);
      if (!err.empty()) return TC_ERR_NOMEM;
      std::vector<int> full((size_t)S_, r_);
      TC_CUDA_TRY(cudaMemcpyAsync(rk_, full.data(), full.size() * sizeof(int), cudaMemcpyHostToDevice, stream_));
      TC_CUDA_TRY(cudaMemsetAsync(rcnt_, 0, (size_t)S_ * sizeof(int), stream_));
      TC_CUDA_TRY(cudaStreamSynchronize(stream_));  // the host vector goes out of scope
      rank_smem_ = rank_smem_bytes(r_);
      TC_CUDA_TRY(allow_dynamic_smem((const void*)k_rank<T>, rank_smem_));
    }
    d_.rk = tol > 0.0 ? rk_ : nullptr;
    d_.rcnt = rcnt_;
    d_.rscr = rscr_;
    d_.rank_tol = tol;
    d_.rank_patience = patience;
    if (rcnt_) TC_CUDA_TRY(cudaMemsetAsync(rcnt_, 0, (size_t)S_ * sizeof(int), stream_));
    // the captured iteration carries d_ by value: capture it again
    if (graph_exec_) {
      TC_CUDA_TRY(cudaStreamSynchronize(stream_));
      cudaGraphExecDestroy(graph_exec_);
      graph_exec_ = nullptr;
    }
    tc_status st = capture(err);
    if (st != TC_OK) return st;
    TC_CUDA_TRY(cudaGraphUpload(graph_exec_, stream_));
    return TC_OK;
  }

  tc_status ranks(int* out, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    std::vector<int> h((size_t)S_, r_);
    if (rk_) {
      TC_CUDA_TRY(cudaMemcpyAsync(h.data(), rk_, h.size() * sizeof(int), cudaMemcpyDeviceToHost, stream_));
      TC_CUDA_TRY(cudaStreamSynchronize(stream_));
    }
    for (int k = 0; k < n3_; ++k) out[k] = h[k < S_ ? k : n3_ - k];  // r_k = r_{n3-k} (conjugate slices)
    return TC_OK;
  }

  int slab_tile() const override { return slab_tile_; }
  cudaStream_t stream() const override { return stream_; }
  bool poisoned() const override { return poisoned_; }

  tc_status profile(int n, double* ms, std::string& err) override {
    if (poisoned_) {
      err = "context poisoned by an earlier error";
      return TC_ERR_STATE;
    }
    constexpr int K = 4;
    cudaEvent_t ev[K + 1];
    for (int i = 0; i <= K; ++i) TC_CUDA_TRY(cudaEventCreate(&ev[i]));
    double acc[K] = {0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n && e == cudaSuccess; ++it) {
      cudaEventRecord(ev[0], stream_);
      launch_qcon(stream_);
      cudaEventRecord(ev[1], stream_);
      launch_xstep(stream_);
      cudaEventRecord(ev[2], stream_);
      launch_ystep(stream_, nullptr, false);  // A^+ of the next X-step is formed below, untimed
      cudaEventRecord(ev[3], stream_);
      launch_slab(MODE_ITER, nullptr, 0, stream_);
      cudaEventRecord(ev[4], stream_);
      // in the captured iteration k_xa runs beside the slab kernel; here after it
      if (xsplit_ || apre_) xa_fn_<<<S_, xa_threads_, xa_smem_, stream_>>>(d_);
      if (d_.rk) launch_rank(stream_);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[K]);
      for (int q = 0; q < K && e == cudaSuccess; ++q) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
        acc[q] += t;
      }
    }
    for (int i = 0; i <= K; ++i) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) {
      err = std::string("profiled iteration failed: ") + cudaGetErrorString(e);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    for (int q = 0; q < K; ++q) ms[q] = acc[q] / n;
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

  tc_status tune_slab_tile(std::string& err) {
    const int cand[3] = {2, 4, 8};
    SlabFn<T> tab[3][3];
    slab_table_tl<T, 2>(tab[0]);
    slab_table_tl<T, 4>(tab[1]);
    slab_table_tl<T, 8>(tab[2]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TC_CUDA_TRY(cudaEventCreate(&e0));
    TC_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int pick = 1;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
      for (int m = 0; m < 3 && e == cudaSuccess; ++m) e = allow_dynamic_smem((const void*)tab[c][m], slab_smem_);
      for (int m = 0; m < 3; ++m) slab_[m] = tab[c][m];
      float ms = 1e30f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, stream_);
        if (e == cudaSuccess) launch_slab(MODE_ITER, nullptr, 1, stream_);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, stream_);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (e == cudaSuccess && ms < best) {
        best = ms;
        pick = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
      err = std::string("tuning of the generic slab kernel failed: ") + cudaGetErrorString(e);
      poisoned_ = true;
      return TC_ERR_CUDA;
    }
    for (int m = 0; m < 3; ++m) slab_[m] = tab[pick][m];
    slab_tile_ = cand[pick];
    return TC_OK;
  }

  void launch_slab(int mode, T* Wout, int init, cudaStream_t s) {
    slab_[mode]<<<n1_, slab_threads_, slab_smem_, s>>>(d_, Wout, slabs_in_smem_ ? 1 : 0, init);
  }
  void launch_qcon(cudaStream_t s) { qcon_<<<qgrid_, qthreads_, qcon_smem_, s>>>(d_, Q_); }
  // With the four-kernel X-step, A^+ (k_xa) is formed after every change of Y~
  // (initialisation, Y-step), so the X-step starts with it in place.
  void launch_xstep(cudaStream_t s) {
    if (xsplit_) {
      k_xbg<T><<<dim3(S_, (n1_ + kXbRows - 1) / kXbRows), 256, xbg_smem_, s>>>(d_, Q_);
      k_xbc<T><<<dim3(S_, (r_ + 7) / 8), 256, xbc_smem_, s>>>(d_);
      k_xg<T><<<dim3(S_, gch_), 256, xg_smem_, s>>>(d_);
      xc_fn_<<<S_, kXaThreads, xa_smem_, s>>>(d_);
      return;
    }
    xstep_<<<S_, xstep_threads(rp_), xstep_smem_, s>>>(d_, Q_, xarrays_in_smem_ ? 1 : 0);
  }
  // Y-step, then (four-kernel X-step) A^+ of the next X-step from the new tile
  // Grams.  With a branch stream (graph capture) A^+ is formed there, beside
  // the rest of the iteration; the return value says whether it was, and the
  // caller then joins on ev_join_.  Without one it follows on s.
  bool launch_ystep(cudaStream_t s, cudaStream_t branch = nullptr, bool with_xa = true) {
    const int tw = 32 * ystep_cpl(rp_);
    dim3 g(S_, (n2_ + tw - 1) / tw);
    if (tcy_) tck_.dcon<<<dim3(S_, (n2_ + 127) / 128, ksplit_), 256, tck_.dsm, s>>>(d_);
    ystep_<<<g, kYThreads, ystep_smem_, s>>>(d_);
    bool forked = false;
    if ((xsplit_ || apre_) && with_xa) {
      if (branch && cudaEventRecord(ev_fork_, s) == cudaSuccess &&
          cudaStreamWaitEvent(branch, ev_fork_, 0) == cudaSuccess) {
        xa_fn_<<<S_, xa_threads_, xa_smem_, branch>>>(d_);
        forked = cudaEventRecord(ev_join_, branch) == cudaSuccess;
      } else {
        xa_fn_<<<S_, xa_threads_, xa_smem_, s>>>(d_);
      }
    }
    if (tcy_) tck_.zsyn<<<dim3(S_, (n1_ + 127) / 128, (n2_ + 63) / 64), 256, tck_.zsm, s>>>(d_);
    return forked;
  }

  // One TCTF2R iteration: Q = R~Y~^H, X-step (+ Y-step r x r work), Y-step,
  // then the slab kernel (Z, W-step, R~).
  // Step 5 (rank vector): the rank kernel, then the tile Grams of Y~ and A^+ of
  // the next X-step again (the rank kernel may have rotated Y~).
  void launch_rank(cudaStream_t s) {
    k_rank<T><<<S_, 256, rank_smem_, s>>>(d_);
    k_gram_tiles<T><<<dim3(S_, d_.ytiles), 256, 0, s>>>(d_);
    if (xsplit_ || apre_) xa_fn_<<<S_, xa_threads_, xa_smem_, s>>>(d_);
  }

  void launch_iteration(cudaStream_t s) {
    launch_qcon(s);
    launch_xstep(s);
    launch_ystep(s);
    launch_slab(MODE_ITER, nullptr, 0, s);
    if (d_.rk) launch_rank(s);
    if (d_.conv) k_check<T><<<1, 32, 0, s>>>(d_);  // step 6
  }

  tc_status read_conv(unsigned long long* h, std::string& err) {
    TC_CUDA_TRY(cudaMemcpyAsync(h, d_.conv, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream_));
    TC_CUDA_TRY(cudaStreamSynchronize(stream_));
    return TC_OK;
  }

  tc_status capture(std::string& err) {
    cudaGraph_t g = nullptr;
    tc_status st = capture_iteration(&g, err);
    if (st != TC_OK) return st;
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
  int n1_ = 0, n2_ = 0, n3_ = 0, r_ = 0, S_ = 0, mw_ = 0, rp_ = 8;
  bool poisoned_ = false;
  bool specialised_ = false;
  bool slabs_in_smem_ = true;
  bool xarrays_in_smem_ = true;
  bool mixed_ = false;
  bool xsplit_ = false;  // X-step as four kernels
  bool apre_ = false;    // one-CTA X-step with A^+ from k_xa on a graph branch
  int slab_tile_ = 0;    // rows / slices per item of the generic transform (0: specialised length)
  int* rk_ = nullptr;    // step 5: slice ranks, counters and work (allocated when the rule is first on)
  int* rcnt_ = nullptr;
  cx<T>* rscr_ = nullptr;
  size_t rank_smem_ = 0;
  int xa_threads_ = kXaThreads;
  YFn<T> xa_fn_ = nullptr, xc_fn_ = nullptr;
  int gch_ = 0;
  size_t xa_smem_ = 0, xbg_smem_ = 0, xbc_smem_ = 0, xg_smem_ = 0;
  cudaStream_t aux_stream_ = nullptr;  // graph branch of k_xa during capture
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr;
  bool tcy_ = false;  // tensor-core Y-step (D partials, update, Z~ synthesis)
  TcKernels<T> tck_;
  int ksplit_ = 1;
  cx<T>* Dpart_ = nullptr;
  dim3 qgrid_;
  int qthreads_ = kSliceThreads;
  int slab_threads_ = 256;
  size_t slab_smem_ = 0, xstep_smem_ = 0, ystep_smem_ = 0, qcon_smem_ = 0;
  SlabFn<T> slab_[3] = {nullptr, nullptr, nullptr};
  XFn<T> xstep_ = nullptr;
  YFn<T> ystep_ = nullptr;
  QFn<T> qcon_ = nullptr;
  cx<T>* Q_ = nullptr;
  Dev<T> d_{};
  std::vector<void*> allocs_;
};

}  // namespace tc
