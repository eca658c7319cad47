// FP32 engine: generic slab kernel here; the slab kernels specialised for a
// tube length live in their own translation units (compiled in parallel).
#include "tc_engine.cuh"

namespace tc {

bool slab_setup_f32_112(int n2, int optin, SlabCfg<float>& cfg);
bool slab_setup_f32_168(int n2, int optin, SlabCfg<float>& cfg);

template <>
bool pick_slab<float>(int n2, int n3, int optin, SlabCfg<float>& cfg) {
  switch (n3) {
    case 112: return slab_setup_f32_112(n2, optin, cfg);
    case 168: return slab_setup_f32_168(n2, optin, cfg);
    default: return false;
  }
}

template <>
void upload_twiddles<float>() {}

EngineBase* make_engine_f32() { return new Engine<float>(); }

}  // namespace tc
