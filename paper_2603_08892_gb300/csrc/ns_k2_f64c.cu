// ns_k2_f64c.cu -- size-specialised kernels (double, N in {384, 512, 768}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f64c(int N, K2Entry<double>* e) {
  switch (N) {
    case 384:
      *e = make_k2_entry<double, 384>();
      return true;
    case 512:
      *e = make_k2_entry<double, 512>();
      return true;
    case 768:
      *e = make_k2_entry<double, 768>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
