// ns_batch_f64.cu -- FP64 instantiation of the persistent batched kernel (own translation
// unit so the two precisions compile in parallel).
#include "ns_batch.cuh"

using namespace nsb;

int ns_batch_step_f64(ns_batch* b, const double* dt, int nsteps) {
  return batch_step_t<double>(b, dt, nsteps);
}

// resident CTAs per SM of the FP64 persistent kernel (for the schedule tuner)
int ns_batch_max_ctas_f64() {
  int q = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, k_batch<double>, BCfg<double>::NT, BCfg<double>::SM);
  return q;
}
