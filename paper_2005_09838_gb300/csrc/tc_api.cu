// C ABI of the TCTF2R library (declared in include/tctf2r.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "tc_engine.h"
#include "tctf2r.h"

struct tc_ctx {
  tc::EngineBase* eng = nullptr;
  int device = 0;
  int64_t n3 = 0;
};

namespace {

thread_local std::string g_last_error;

tc_status fail(tc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

tc_status validate(const tc_params* p) {
  if (!p) return fail(TC_ERR_ARG, "params is NULL");
  if (p->n1 < 1 || p->n2 < 1 || p->n3 < 1) return fail(TC_ERR_ARG, "n1, n2, n3 must be >= 1");
  if (p->n1 > (1 << 24) || p->n2 > 4096 || p->n3 > 4096)
    return fail(TC_ERR_ARG, "sizes beyond the supported range (n1 <= 2^24, n2 <= 4096, n3 <= 4096)");
  const double N = (double)p->n1 * (double)p->n2 * (double)p->n3;
  if (N > 4.0e9) return fail(TC_ERR_ARG, "n1*n2*n3 exceeds 4e9 entries");
  if (p->r < 1 || p->r > 32 || p->r > p->n1 || p->r > p->n2)
    return fail(TC_ERR_ARG, "r must satisfy 1 <= r <= min(n1, n2, 32)");
  if (!(p->mu >= 0) || !(p->rho1 >= 0) || !(p->rho2 >= 0) || !std::isfinite(p->mu) || !std::isfinite(p->rho1) ||
      !std::isfinite(p->rho2))
    return fail(TC_ERR_ARG, "mu, rho1, rho2 must be finite and >= 0");
  if (p->precision != TC_FP64 && p->precision != TC_FP32 && p->precision != TC_TF32 && p->precision != TC_BF16)
    return fail(TC_ERR_ARG, "unknown precision");
  const bool mixed = p->precision == TC_TF32 || p->precision == TC_BF16;
  if ((p->flags & ~(int32_t)TC_FLAG_SINGLE_PASS) != 0 || (!mixed && p->flags != 0))
    return fail(TC_ERR_ARG, "unknown flags, or TC_FLAG_SINGLE_PASS without TC_TF32 / TC_BF16");
  if (p->step != TC_STEP_EXACT && p->step != TC_STEP_SCALED) return fail(TC_ERR_ARG, "unknown step rule");
  if (p->step == TC_STEP_SCALED &&
      (!(p->alpha > 0) || !(p->beta > 0) || !std::isfinite(p->alpha) || !std::isfinite(p->beta)))
    return fail(TC_ERR_ARG, "scaled steps need finite alpha > 0 and beta > 0");
  if (!(p->eps >= 0) || !std::isfinite(p->eps)) return fail(TC_ERR_ARG, "eps must be finite and >= 0");
  if (!std::isfinite(p->pinv_rtol) || p->pinv_rtol >= 1.0) return fail(TC_ERR_ARG, "pinv_rtol must be < 1");
  return TC_OK;
}

}  // namespace

namespace tc {
// Lets other translation units of the library report through tc_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace tc

extern "C" {

const char* tc_last_error(void) { return g_last_error.c_str(); }

const char* tc_version(void) { return "tctf2r-gb300 0.1 (sm_103a)"; }

tc_status tc_init(tc_ctx** out, const tc_params* p, const void* G, const uint8_t* mask, const void* Y0,
                  const void* X0, int32_t inputs_on_device, void* cuda_stream) {
  g_last_error.clear();
  if (!out) return fail(TC_ERR_ARG, "out is NULL");
  *out = nullptr;
  tc_status st = validate(p);
  if (st != TC_OK) return st;
  if (!G || !mask || !Y0) return fail(TC_ERR_ARG, "G, mask and Y0 are required");
  tc_ctx* c = new (std::nothrow) tc_ctx();
  if (!c) return fail(TC_ERR_NOMEM, "host allocation failed");
  c->n3 = p->n3;
  c->eng = (p->precision == TC_FP64) ? tc::make_engine_f64() : tc::make_engine_f32();
  if (!c->eng) {
    delete c;
    return fail(TC_ERR_NOMEM, "host allocation failed");
  }
  cudaGetDevice(&c->device);
  std::string err;
  st = c->eng->init(*p, G, mask, Y0, X0, inputs_on_device != 0, static_cast<cudaStream_t>(cuda_stream), err);
  if (st != TC_OK) {
    c->eng->release();
    delete c->eng;
    delete c;
    return fail(st, err);
  }
  *out = c;
  return TC_OK;
}

tc_status tc_iterate(tc_ctx* c, int32_t n_iters, int32_t* done) {
  g_last_error.clear();
  if (done) *done = 0;
  if (!c) return fail(TC_ERR_ARG, "ctx is NULL");
  if (n_iters < 0) return fail(TC_ERR_ARG, "n_iters must be >= 0");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  int d = 0;
  tc_status st = c->eng->iterate(n_iters, done ? &d : nullptr, err);
  if (prev != c->device) cudaSetDevice(prev);
  if (done) *done = d;
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_objective(tc_ctx* c, double* f0, double* resid_obs) {
  g_last_error.clear();
  if (!c || !f0) return fail(TC_ERR_ARG, "ctx and f0 are required");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  tc_status st = c->eng->objective(f0, resid_obs, err);
  if (prev != c->device) cudaSetDevice(prev);
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_result(tc_ctx* c, void* W, void* X, void* Y, int32_t dst_on_device) {
  g_last_error.clear();
  if (!c) return fail(TC_ERR_ARG, "ctx is NULL");
  if (!W && !X && !Y) return fail(TC_ERR_ARG, "no output requested");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  tc_status st = c->eng->result(W, X, Y, dst_on_device != 0, err);
  if (prev != c->device) cudaSetDevice(prev);
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_profile(tc_ctx* c, int32_t n_iters, double* ms) {
  g_last_error.clear();
  if (!c || !ms) return fail(TC_ERR_ARG, "ctx and ms are required");
  if (n_iters < 1) return fail(TC_ERR_ARG, "n_iters must be >= 1");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  tc_status st = c->eng->profile(n_iters, ms, err);
  if (prev != c->device) cudaSetDevice(prev);
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_convergence(tc_ctx* c, double* changes, int32_t* stopped, int64_t* iters_run) {
  g_last_error.clear();
  if (!c || !changes) return fail(TC_ERR_ARG, "ctx and changes are required");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  int s = 0;
  long long it = 0;
  tc_status st = c->eng->convergence(changes, &s, &it, err);
  if (prev != c->device) cudaSetDevice(prev);
  if (stopped) *stopped = s;
  if (iters_run) *iters_run = it;
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_rank_rule(tc_ctx* c, double tol, int32_t patience) {
  g_last_error.clear();
  if (!c) return fail(TC_ERR_ARG, "ctx is required");
  if (!(tol >= 0.0) || !(tol < 1.0)) return fail(TC_ERR_ARG, "tol must satisfy 0 <= tol < 1");
  if (patience < 1) return fail(TC_ERR_ARG, "patience must be >= 1");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  tc_status st = c->eng->set_rank_rule(tol, patience, err);
  if (prev != c->device) cudaSetDevice(prev);
  return st == TC_OK ? st : fail(st, err);
}

tc_status tc_ranks(tc_ctx* c, int32_t* ranks) {
  g_last_error.clear();
  if (!c || !ranks) return fail(TC_ERR_ARG, "ctx and ranks are required");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  std::string err;
  std::vector<int> h((size_t)c->n3);
  tc_status st = c->eng->ranks(h.data(), err);
  if (prev != c->device) cudaSetDevice(prev);
  if (st != TC_OK) return fail(st, err);
  for (size_t k = 0; k < h.size(); ++k) ranks[k] = (int32_t)h[k];
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Batched form: many contexts advanced by one CUDA graph per iteration.  The
// graph holds one child graph per instance (its captured iteration) in K
// independent chains; instance i runs in chain i mod K, so independent
// completions of different sizes fill the GPU together.  The
// first iterations try each candidate K once or twice (each trial is a real
// iteration of every instance, so the results do not depend on the choice)
// and keep the fastest.
// ---------------------------------------------------------------------------
struct tc_batch {
  std::vector<tc_ctx*> ctxs;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<int> cand;              // branch counts of the candidate graphs
  std::vector<cudaGraphExec_t> exec;  // one per candidate
  std::vector<float> best_ms;         // best trial time per candidate
  std::vector<int> trials;
  int chosen = -1;
  cudaGraphExec_t loop = nullptr;     // after tuning: n iterations in one launch (device-side loop)
  bool loop_failed = false;           // conditional nodes unavailable: one launch per iteration
  unsigned int* left = nullptr;       // device counter of the iterations still to run
  long long launches = 0;             // graph launches made by tc_batch_iterate
  std::vector<cudaGraph_t> child;     // one captured iteration per instance
  std::vector<cudaEvent_t> ctx_ev;
  cudaEvent_t t0 = nullptr, t1 = nullptr, done = nullptr;

  void release() {
    if (loop) cudaGraphExecDestroy(loop);
    loop = nullptr;
    if (left) cudaFree(left);
    left = nullptr;
    for (auto e : exec)
      if (e) cudaGraphExecDestroy(e);
    for (auto g : child)
      if (g) cudaGraphDestroy(g);
    for (auto e : ctx_ev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {t0, t1, done})
      if (e) cudaEventDestroy(e);
    exec.clear();
    child.clear();
    ctx_ev.clear();
    t0 = t1 = done = nullptr;
  }
};

namespace {

constexpr int kBatchTrials = 2;

// The batched graph: one child graph per instance (its own captured
// iteration), chained K ways; chain j runs instances j, j + K, ...
tc_status batch_build(tc_batch* b, int K, cudaGraphExec_t* out, std::string& err) {
  cudaGraph_t parent = nullptr;
  cudaError_t e = cudaGraphCreate(&parent, 0);
  std::vector<cudaGraphNode_t> last(K, nullptr);
  for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i) {
    const int j = (int)(i % K);
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddChildGraphNode(&node, parent, last[j] ? &last[j] : nullptr, last[j] ? 1 : 0, b->child[i]);
    last[j] = node;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, parent, 0);
  if (parent) cudaGraphDestroy(parent);
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = std::string("batched graph build failed: ") + cudaGetErrorString(e);
    return TC_ERR_CUDA;
  }
  return TC_OK;
}

// Device-side loop of the batched completion: before the launch the counter
// holds n >= 1; each pass of the while body runs one iteration of every
// instance and then this one-thread kernel, which counts down and keeps the
// loop going while iterations remain (the count only decreases, so the loop
// ends after n passes).
__global__ void k_batch_set(unsigned int* left, unsigned int n) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *left = n;
}
__global__ void k_batch_count(unsigned int* left, cudaGraphConditionalHandle h) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned int n = *left;
    const unsigned int rest = n > 1u ? n - 1u : 0u;
    *left = rest;
    cudaGraphSetConditional(h, rest > 0u ? 1u : 0u);
  }
}

// The loop graph: a while node whose body is the batched iteration with K
// chains (as batch_build) followed by k_batch_count.
tc_status batch_build_loop(tc_batch* b, int K, cudaGraphExec_t* out, std::string& err) {
  cudaGraph_t parent = nullptr;
  cudaError_t e = cudaGraphCreate(&parent, 0);
  cudaGraphConditionalHandle h{};
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, parent, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, parent, nullptr, nullptr, 0, &cp);
  cudaGraph_t body = (e == cudaSuccess) ? cp.conditional.phGraph_out[0] : nullptr;
  std::vector<cudaGraphNode_t> last(K, nullptr);
  for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i) {
    const int j = (int)(i % K);
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddChildGraphNode(&node, body, last[j] ? &last[j] : nullptr, last[j] ? 1 : 0, b->child[i]);
    last[j] = node;
  }
  std::vector<cudaGraphNode_t> tails;
  for (auto n : last)
    if (n) tails.push_back(n);
  if (e == cudaSuccess) {
    cudaKernelNodeParams kp{};
    void* args[] = {&b->left, &h};
    kp.func = (void*)k_batch_count;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    cudaGraphNode_t knode = nullptr;
    e = cudaGraphAddKernelNode(&knode, body, tails.data(), tails.size(), &kp);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, parent, 0);
  if (parent) cudaGraphDestroy(parent);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    err = std::string("device-side loop of the batch not available: ") + cudaGetErrorString(e);
    return TC_ERR_CUDA;
  }
  return TC_OK;
}

}  // namespace

tc_status tc_batch_create(tc_batch** out, tc_ctx* const* ctxs, int32_t count, void* cuda_stream) {
  g_last_error.clear();
  if (!out) return fail(TC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || count < 1) return fail(TC_ERR_ARG, "ctxs must hold count >= 1 contexts");
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return fail(TC_ERR_ARG, "a context is NULL");
    if (ctxs[i]->device != dev) return fail(TC_ERR_ARG, "all contexts must live on the current device");
    if (ctxs[i]->eng->poisoned()) return fail(TC_ERR_STATE, "a context is poisoned by an earlier error");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(TC_ERR_ARG, "a context appears twice");
  }
  tc_batch* b = new (std::nothrow) tc_batch();
  if (!b) return fail(TC_ERR_NOMEM, "host allocation failed");
  b->ctxs.assign(ctxs, ctxs + count);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->device = dev;
  for (int K : {1, 4, 16, count})
    if (K <= count && std::find(b->cand.begin(), b->cand.end(), K) == b->cand.end()) b->cand.push_back(K);
  std::string err;
  cudaError_t e = cudaSuccess;
  b->ctx_ev.assign(count, nullptr);
  for (int i = 0; i < count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ctx_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->t1);
  if (e != cudaSuccess) {
    b->release();
    delete b;
    return fail(TC_ERR_CUDA, std::string("batch set-up failed: ") + cudaGetErrorString(e));
  }
  b->child.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    tc_status st = b->ctxs[i]->eng->capture_iteration(&b->child[i], err);
    if (st != TC_OK) {
      b->release();
      delete b;
      return fail(st, err);
    }
  }
  b->exec.assign(b->cand.size(), nullptr);
  for (size_t c = 0; c < b->cand.size(); ++c) {
    tc_status st = batch_build(b, b->cand[c], &b->exec[c], err);
    if (st != TC_OK) {
      b->release();
      delete b;
      return fail(st, err);
    }
  }
  b->best_ms.assign(b->cand.size(), 1e30f);
  b->trials.assign(b->cand.size(), 0);
  if (b->cand.size() == 1) b->chosen = 0;
  if (cudaMalloc(&b->left, sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    b->release();
    delete b;
    return fail(TC_ERR_NOMEM, "allocation of the batch counter failed");
  }
  *out = b;
  return TC_OK;
}

tc_status tc_batch_iterate(tc_batch* b, int32_t n_iters) {
  g_last_error.clear();
  if (!b) return fail(TC_ERR_ARG, "batch is NULL");
  if (n_iters < 0) return fail(TC_ERR_ARG, "n_iters must be >= 0");
  if (n_iters == 0) return TC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaError_t e = cudaSuccess;
  // after the work already queued on every context's stream
  for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ctx_ev[i], b->ctxs[i]->eng->stream());
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0);
  }
  for (int it = 0; it < n_iters && e == cudaSuccess; ++it) {
    if (b->chosen >= 0 && !b->loop && !b->loop_failed) {
      std::string lerr;
      b->loop_failed = batch_build_loop(b, b->cand[b->chosen], &b->loop, lerr) != TC_OK;
    }
    if (b->chosen >= 0 && b->loop) {
      // the remaining iterations in one launch: the loop runs on the device
      k_batch_set<<<1, 32, 0, b->stream>>>(b->left, (unsigned int)(n_iters - it));
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaGraphLaunch(b->loop, b->stream);
      ++b->launches;
      break;
    }
    if (b->chosen < 0) {
      // tuning: the candidate with the fewest trials, timed on its own
      size_t c = 0;
      for (size_t q = 1; q < b->cand.size(); ++q)
        if (b->trials[q] < b->trials[c]) c = q;
      e = cudaEventRecord(b->t0, b->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(b->exec[c], b->stream);
      ++b->launches;
      if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b->t1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->t0, b->t1);
      if (e != cudaSuccess) break;
      b->best_ms[c] = std::min(b->best_ms[c], ms);
      if (++b->trials[c] >= kBatchTrials &&
          *std::min_element(b->trials.begin(), b->trials.end()) >= kBatchTrials)
        b->chosen = (int)(std::min_element(b->best_ms.begin(), b->best_ms.end()) - b->best_ms.begin());
    } else {
      e = cudaGraphLaunch(b->exec[b->chosen], b->stream);
      ++b->launches;
    }
  }
  // every context's later calls come after the batch
  if (e == cudaSuccess) e = cudaEventRecord(b->done, b->stream);
  for (size_t i = 0; i < b->ctxs.size() && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(b->ctxs[i]->eng->stream(), b->done, 0);
  if (prev != b->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return fail(TC_ERR_CUDA, std::string("batched iteration failed: ") + cudaGetErrorString(e));
  return TC_OK;
}

tc_status tc_batch_branches(tc_batch* b, int32_t* branches) {
  g_last_error.clear();
  if (!b || !branches) return fail(TC_ERR_ARG, "batch and branches are required");
  *branches = (b->chosen < 0) ? 0 : b->cand[b->chosen];
  return TC_OK;
}

tc_status tc_batch_launches(tc_batch* b, int64_t* launches, int32_t* device_loop) {
  g_last_error.clear();
  if (!b || !launches) return fail(TC_ERR_ARG, "batch and launches are required");
  *launches = b->launches;
  if (device_loop) *device_loop = b->loop ? 1 : 0;
  return TC_OK;
}

tc_status tc_tile(tc_ctx* c, int32_t* slab_tile) {
  g_last_error.clear();
  if (!c || !slab_tile) return fail(TC_ERR_ARG, "ctx and slab_tile are required");
  *slab_tile = c->eng->slab_tile();
  return TC_OK;
}

tc_status tc_batch_free(tc_batch* b) {
  if (!b) return TC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  b->release();
  if (prev != b->device) cudaSetDevice(prev);
  delete b;
  return TC_OK;
}

tc_status tc_free(tc_ctx* c) {
  if (!c) return TC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  c->eng->release();
  delete c->eng;
  if (prev != c->device) cudaSetDevice(prev);
  delete c;
  return TC_OK;
}

}  // extern "C"
