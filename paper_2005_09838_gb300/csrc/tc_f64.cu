// double instantiation of the TCTF2R engine.
#include <cmath>
#include <vector>

#include "tc_engine.cuh"

namespace tc {

template <>
bool pick_slab<double>(int n3, SlabFn<double> f[4]) {
  switch (n3) {
    case 7: slab_table<double, 7>(f); return true;
    default:
      return false;
  }
}

template <>
void upload_twiddles<double>(cudaStream_t) {
  std::vector<cx<double>> tab(fft::kTableSize);
  for (int i = 0; i < fft::kNumLengths; ++i) {
    const int L = fft::kLengths[i];
    const int off = fft::table_offset(L);
    for (int m = 0; m < L; ++m) {
      const double a = 2.0 * M_PI * (double)m / (double)L;
      tab[off + m] = cx<double>{(double)std::cos(a), (double)(-std::sin(a))};
    }
  }
  cudaMemcpyToSymbol(fft::c_tw_f64, tab.data(), tab.size() * sizeof(cx<double>));
}

EngineBase* make_engine_f64() { return new Engine<double>(); }

}  // namespace tc
