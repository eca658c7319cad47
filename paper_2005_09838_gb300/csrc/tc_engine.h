// Host-side engine interface shared by the C ABI layer and the per-precision
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "tctf2r.h"

namespace tc {

struct EngineBase {
  virtual ~EngineBase() {}
  virtual tc_status init(const tc_params& p, const void* G, const uint8_t* mask, const void* Y0, const void* X0,
                         bool on_device, cudaStream_t stream, std::string& err) = 0;
  virtual tc_status iterate(int n, int* done, std::string& err) = 0;
  virtual tc_status objective(double* f0, double* resid_obs, std::string& err) = 0;
  virtual tc_status result(void* W, void* X, void* Y, bool on_device, std::string& err) = 0;
  virtual tc_status profile(int n, double* ms, std::string& err) = 0;
  virtual tc_status convergence(double* changes, int* stopped, long long* iters_run, std::string& err) = 0;
  // step 5 (rank vector): tol = 0 turns the rule off; ranks gets n3 values
  virtual tc_status set_rank_rule(double tol, int patience, std::string& err) = 0;
  virtual tc_status ranks(int* out, std::string& err) = 0;
  // tile of the generic-length transform chosen at init (0: specialised length)
  virtual int slab_tile() const = 0;
  virtual void release() = 0;
  // one iteration captured as a graph (the caller owns and destroys it)
  virtual tc_status capture_iteration(cudaGraph_t* out, std::string& err) = 0;
  virtual cudaStream_t stream() const = 0;
  virtual bool poisoned() const = 0;
};

EngineBase* make_engine_f32();
EngineBase* make_engine_f64();

}  // namespace tc
