// ns_k2_f64b.cu -- size-specialised kernels (double, N in {96, 128, 192, 256}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f64b(int N, K2Entry<double>* e) {
  switch (N) {
    case 96:
      *e = make_k2_entry<double, 96>();
      return true;
    case 128:
      *e = make_k2_entry<double, 128>();
      return true;
    case 192:
      *e = make_k2_entry<double, 192>();
      return true;
    case 256:
      *e = make_k2_entry<double, 256>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
