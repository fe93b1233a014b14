// ns_batch_grid_f32.cu -- the grid schedule of the batched ensembles in FP32: one kernel per kind
// of pass and member size (ns_batch.cuh), compiled in a translation unit of their own so the
// build stays parallel.
#define NS_BATCH_GRID_DEFS
#include "ns_batch.cuh"

namespace nsb {
template cudaError_t launch_class_any<float>(int, const BatchMem<float>*, const int*, int, int, cudaStream_t);
}  // namespace nsb
