// float instantiation of the TCTF2R engine.
#include <cmath>
#include <vector>

#include "tc_engine.cuh"

namespace tc {

template <>
bool pick_slab<float>(int n3, SlabFn<float> f[4]) {
  switch (n3) {
    case 112: slab_table<float, 112>(f); return true;
    case 168: slab_table<float, 168>(f); return true;
    default:
      return false;
  }
}

template <>
void upload_twiddles<float>(cudaStream_t) {
  std::vector<cx<float>> tab(fft::kTableSize);
  for (int i = 0; i < fft::kNumLengths; ++i) {
    const int L = fft::kLengths[i];
    const int off = fft::table_offset(L);
    for (int m = 0; m < L; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)L;
      tab[off + m] = cx<float>{(float)std::cos(a), (float)(-std::sin(a))};
    }
  }
  cudaMemcpyToSymbol(fft::c_tw_f32, tab.data(), tab.size() * sizeof(cx<float>));
}

EngineBase* make_engine_f32() { return new Engine<float>(); }

}  // namespace tc
