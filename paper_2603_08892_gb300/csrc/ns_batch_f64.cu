// ns_batch_f64.cu -- FP64 instantiation of the persistent batched kernel (own translation
// unit so the two precisions compile in parallel).
#include "ns_batch.cuh"

int ns_batch_step_f64(ns_batch* b, const double* dt, int nsteps) {
  return batch_step_t<double>(b, dt, nsteps);
}
