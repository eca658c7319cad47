// FP64 engine (register FFT for n3 = 7, generic transform otherwise).
#include "tc_engine.cuh"

namespace tc {

template <>
bool pick_slab<double>(int n2, int n3, int optin, SlabCfg<double>& cfg) {
  if (n3 != 7) return false;
  const SlabLayout lay = slab_layout<double>(n2, 7, true, true);
  if (lay.total > (size_t)optin) return false;
  slab_table<double, 7>(cfg.f);
  // one thread per tube (up to the register budget) and at least one per W-step row
  cfg.threads = std::max(std::min((n2 + 31) / 32 * 32, slab_max_threads(7)), 32);
  cfg.smem = lay.total;
  return true;
}

template <>
void upload_twiddles<double>() { fft::upload_tables<double>(); }

template <>
bool pick_tc<double>(int, bool, TcKernels<double>&) {
  return false;
}

EngineBase* make_engine_f64() { return new Engine<double>(); }

}  // namespace tc
