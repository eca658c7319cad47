// FP32 engine: generic slab kernel here; the register-FFT slab kernels live in
// their own translation units (compiled in parallel).
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_112(SlabFn<float> f[3]);
bool slab_setup_f32_168(SlabFn<float> f[3]);

template <>
bool pick_slab<float>(int n3, SlabFn<float> f[3]) {
  switch (n3) {
    case 112: return slab_setup_f32_112(f);
    case 168: return slab_setup_f32_168(f);
    default: return false;
  }
}

template <>
void upload_twiddles<float>() {}

EngineBase* make_engine_f32() { return new Engine<float>(); }

}  // namespace tc
