// FP32 slab kernels for n3 = 112: shared-memory transform with M = 56 = 8 x 7.
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_112(int n2, int optin, SlabCfg<float>& cfg) {
  const SlabFLayout lay = slab_f_layout<float>(n2, 112);
  if (lay.total > (size_t)optin) return false;
  fft::upload_tables<float>();
  slab_f_table<float, 112, 8, 7>(cfg.f);
  cfg.threads = kSlabFThreads;
  cfg.smem = lay.total;
  return true;
}

}  // namespace tc
