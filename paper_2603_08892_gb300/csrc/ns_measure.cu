// ns_measure.cu -- FP32 / FP64 CUDA-core FMA throughput of the device (the denominator of the
// secondary, arithmetic roofline of the FFT passes).  Every thread runs 8 independent FMA
// chains; the grid fills every SM.  No counterpart in the paper: measurement only.
#include <cuda_runtime.h>

#include "ns.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x) * T(1e-3) + T(i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(-1.2345)) out[0] = s;  // keeps the chains live; never taken for these inputs
}

template <typename T>
int fma_peak(int device, int iters, double* flops) {
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return NS_ERR_CUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = NS_ERR_CUDA;
  const int blocks = nsm * 8, threads = 256;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) goto done;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
  k_fma_peak<T><<<blocks, threads>>>(out, iters / 8, T(0.999999), T(1e-6));  // warm-up
  cudaEventRecord(e0);
  k_fma_peak<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
  cudaEventRecord(e1);
  if (cudaEventSynchronize(e1) != cudaSuccess) goto done;
  if (cudaGetLastError() != cudaSuccess) goto done;
  cudaEventElapsedTime(&ms, e0, e1);
  *flops = 2.0 * 8.0 * (double)blocks * threads * iters / (ms * 1e-3);
  rc = NS_OK;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaSetDevice(prev);
  return rc;
}

}  // namespace

extern "C" int ns_fma_peak(int device, int precision, double* flops_per_s) {
  if (!flops_per_s || (precision != NS_FP32 && precision != NS_FP64)) return NS_ERR_INVALID_ARG;
  return precision == NS_FP32 ? fma_peak<float>(device, 1 << 15, flops_per_s)
                              : fma_peak<double>(device, 1 << 10, flops_per_s);
}
