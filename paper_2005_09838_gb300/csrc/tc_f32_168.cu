// FP32 slab kernels with the register FFT of length 168.
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_168(SlabFn<float> f[3]) {
  fft::upload_tables<float>();
  slab_table<float, 168>(f);
  return true;
}

}  // namespace tc
