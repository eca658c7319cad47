// FP64 engine (register FFT for n3 = 7, generic transform otherwise).
#include "tc_engine.cuh"

namespace tc {

template <>
bool pick_slab<double>(int n3, SlabFn<double> f[3]) {
  switch (n3) {
    case 7: slab_table<double, 7>(f); return true;
    default: return false;
  }
}

template <>
void upload_twiddles<double>() { fft::upload_tables<double>(); }

EngineBase* make_engine_f64() { return new Engine<double>(); }

}  // namespace tc
