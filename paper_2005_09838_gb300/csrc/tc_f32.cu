// FP32 engine: generic slab kernel here; the slab kernels specialised for a
// tube length live in their own translation units (compiled in parallel).
#include "tc_engine.cuh"
#include "k_tc.cuh"

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

template <>
bool pick_tc<float>(int precision, bool split, TcKernels<float>& k) {
  using namespace umma;
  if (precision == TC_TF32) {
    if (split) {
      k = {k_qcon_tc<kTF32, true>, k_dcon_tc<kTF32, true>, k_zsyn_tc<kTF32, true>, qcon_tc_smem<kTF32, true>(),
           dcon_tc_smem<kTF32, true>(), zsyn_tc_smem<kTF32, true>()};
    } else {
      k = {k_qcon_tc<kTF32, false>, k_dcon_tc<kTF32, false>, k_zsyn_tc<kTF32, false>, qcon_tc_smem<kTF32, false>(),
           dcon_tc_smem<kTF32, false>(), zsyn_tc_smem<kTF32, false>()};
    }
    return true;
  }
  if (precision == TC_BF16) {
    if (split) {
      k = {k_qcon_tc<kBF16, true>, k_dcon_tc<kBF16, true>, k_zsyn_tc<kBF16, true>, qcon_tc_smem<kBF16, true>(),
           dcon_tc_smem<kBF16, true>(), zsyn_tc_smem<kBF16, true>()};
    } else {
      k = {k_qcon_tc<kBF16, false>, k_dcon_tc<kBF16, false>, k_zsyn_tc<kBF16, false>, qcon_tc_smem<kBF16, false>(),
           dcon_tc_smem<kBF16, false>(), zsyn_tc_smem<kBF16, false>()};
    }
    return true;
  }
  return false;
}

EngineBase* make_engine_f32() { return new Engine<float>(); }

}  // namespace tc
