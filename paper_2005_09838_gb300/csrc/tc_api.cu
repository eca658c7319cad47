// C ABI of the TCTF2R library (declared in include/tctf2r.h).
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <string>

#include "tc_engine.h"
#include "tctf2r.h"

struct tc_ctx {
  tc::EngineBase* eng = nullptr;
  int device = 0;
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
  if (p->flags != 0) return fail(TC_ERR_ARG, "flags must be 0");
  if (p->precision != TC_FP64 && p->precision != TC_FP32) {
    if (p->precision == TC_TF32 || p->precision == TC_BF16)
      return fail(TC_ERR_UNSUPPORTED, "TF32/BF16 precision is not built");
    return fail(TC_ERR_ARG, "unknown precision");
  }
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
