// FP32 slab kernels for n3 = 168: shared-memory transform with M = 84 = 12 x 7.
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_168(int n2, int optin, SlabCfg<float>& cfg) {
  const SlabFLayout lay = slab_f_layout<float>(n2, 168);
  if (lay.total > (size_t)optin) return false;
  fft::upload_tables<float>();
  slab_f_table<float, 168, 12, 7>(cfg.f);
  cfg.threads = kSlabFThreads;
  cfg.smem = lay.total;
  return true;
}

}  // namespace tc
