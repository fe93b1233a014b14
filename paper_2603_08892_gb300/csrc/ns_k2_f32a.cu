// ns_k2_f32a.cu -- size-specialised kernels (float, N in {8, 12, 16, 24, 32, 48, 64}).
// One translation unit per group of sizes so the build compiles them in parallel.
#include "ns_kernels2.cuh"

namespace ns {

bool k2_lookup_f32a(int N, K2Entry<float>* e) {
  switch (N) {
    case 8:
      *e = make_k2_entry<float, 8>();
      return true;
    case 12:
      *e = make_k2_entry<float, 12>();
      return true;
    case 16:
      *e = make_k2_entry<float, 16>();
      return true;
    case 24:
      *e = make_k2_entry<float, 24>();
      return true;
    case 32:
      *e = make_k2_entry<float, 32>();
      return true;
    case 48:
      *e = make_k2_entry<float, 48>();
      return true;
    case 64:
      *e = make_k2_entry<float, 64>();
      return true;
    default:
      return false;
  }
}

}  // namespace ns
