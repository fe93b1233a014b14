// ns_k2_f32d.cu -- size-specialised kernels (float, N in {384, 512, 768}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f32d(int N, K2Entry<float>* e) {
  switch (N) {
    case 384:
      *e = make_k2_entry<float, 384>();
      return true;
    case 512:
      *e = make_k2_entry<float, 512>();
      return true;
    case 768:
      *e = make_k2_entry<float, 768>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
