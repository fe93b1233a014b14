// ns_k2_f32b.cu -- size-specialised kernels (float, N in {96, 128, 192}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f32b(int N, K2Entry<float>* e) {
  switch (N) {
    case 96:
      *e = make_k2_entry<float, 96>();
      return true;
    case 128:
      *e = make_k2_entry<float, 128>();
      return true;
    case 192:
      *e = make_k2_entry<float, 192>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
