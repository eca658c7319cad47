// FP32 slab kernels with the register FFT of length 112.
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_112(SlabFn<float> f[3]) {
  fft::upload_tables<float>();
  slab_table<float, 112>(f);
  return true;
}

}  // namespace tc
