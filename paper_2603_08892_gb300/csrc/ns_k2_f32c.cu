// ns_k2_f32c.cu -- size-specialised kernels (float, N in {256}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f32c(int N, K2Entry<float>* e) {
  switch (N) {
    case 256:
      *e = make_k2_entry<float, 256>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
