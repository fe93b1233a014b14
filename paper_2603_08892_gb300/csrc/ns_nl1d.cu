// ns_nl1d.cu -- the one-dimensional quadratic model of Sec. 3.3 (Eq. model-1d, "nl1d"):
// dS/dt = -sign(S) S^2 on [0, 2 pi), pseudo-spectral on N points with the truncation
// |k| < kmax (Sec. 3.2) and the RK2 of Sec. 4.1 (midpoint; no viscosity).  A demonstration of
// where the aliases of the quadratic term land: one block per field, FP64, direct DFTs against a
// shared twiddle table (N need not be 2^a 3^b: the paper's example has N = 22), every step in
// one launch with the state in shared memory.
#include <cuda_runtime.h>

#include <cmath>

#include "ns.h"

namespace {

constexpr int kNl1dMaxN = 2048;

// shared layout: twiddles c[N], s[N] (cos, sin of 2 pi m / N); spectra S, H, F as (re, im)
// arrays of M + 1 = N/2 + 1; the physical field x[N]
struct Nl1dSmem {
  double *c, *s, *Sr, *Si, *Hr, *Hi, *Fr, *Fi, *x;
  __device__ Nl1dSmem(double* b, int N) {
    const int M1 = N / 2 + 1;
    c = b; s = c + N;
    Sr = s + N; Si = Sr + M1;
    Hr = Si + M1; Hi = Hr + M1;
    Fr = Hi + M1; Fi = Fr + M1;
    x = Fi + M1;
  }
  static size_t bytes(int N) { return sizeof(double) * (3 * (size_t)N + 6 * (size_t)(N / 2 + 1)); }
};

// half spectrum (k = 0 .. N/2, 1/N on the forward transform) of the real x, truncated to k < kmax
__device__ void nl1d_forward(const Nl1dSmem& m, int N, double kmax, double* Rr, double* Ri) {
  for (int k = threadIdx.x; k <= N / 2; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    if ((double)k < kmax) {
      for (int j = 0; j < N; ++j) {
        const int t = (int)(((long long)j * k) % N);
        re += m.x[j] * m.c[t];
        im -= m.x[j] * m.s[t];
      }
      re /= N;
      im /= N;
    }
    Rr[k] = re;
    Ri[k] = im;
  }
  __syncthreads();
}

// x = the real field of the half spectrum R (the k = 0 and N/2 entries taken as real)
__device__ void nl1d_inverse(const Nl1dSmem& m, int N, const double* Rr, const double* Ri) {
  const int M = N / 2;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double v = 0.0;
    for (int k = 1; k < M; ++k) {
      const int t = (int)(((long long)j * k) % N);
      v += Rr[k] * m.c[t] - Ri[k] * m.s[t];
    }
    m.x[j] = Rr[0] + 2.0 * v + ((j & 1) ? -Rr[M] : Rr[M]);
  }
  __syncthreads();
}

// F = T FFT[-sign(S) S^2] of the half spectrum R (Eq. model-1d; the product on the grid)
__device__ void nl1d_nonlinear(const Nl1dSmem& m, int N, double kmax, const double* Rr,
                               const double* Ri) {
  nl1d_inverse(m, N, Rr, Ri);
  for (int j = threadIdx.x; j < N; j += blockDim.x) m.x[j] = -m.x[j] * fabs(m.x[j]);
  __syncthreads();
  nl1d_forward(m, N, kmax, m.Fr, m.Fi);
}

__global__ void __launch_bounds__(256) k_nl1d(int N, double kmax, double dt, int nsteps,
                                              const double* __restrict__ s0, double* out) {
  extern __shared__ double sm_nl1d[];
  const Nl1dSmem m(sm_nl1d, N);
  const int M = N / 2;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sincospi(2.0 * i / N, &m.s[i], &m.c[i]);
    m.x[i] = s0[(size_t)blockIdx.x * N + i];
  }
  __syncthreads();
  nl1d_forward(m, N, kmax, m.Sr, m.Si);  // the truncated initial state
  for (int n = 0; n < nsteps; ++n) {
    nl1d_nonlinear(m, N, kmax, m.Sr, m.Si);
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
      m.Hr[k] = m.Sr[k] + 0.5 * dt * m.Fr[k];
      m.Hi[k] = m.Si[k] + 0.5 * dt * m.Fi[k];
    }
    __syncthreads();
    nl1d_nonlinear(m, N, kmax, m.Hr, m.Hi);
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
      m.Sr[k] += dt * m.Fr[k];
      m.Si[k] += dt * m.Fi[k];
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k <= M; k += blockDim.x) {
    out[((size_t)blockIdx.x * (M + 1) + k) * 2] = m.Sr[k];
    out[((size_t)blockIdx.x * (M + 1) + k) * 2 + 1] = m.Si[k];
  }
}

}  // namespace

extern "C" int ns_nl1d(int N, double kmax, double dt, int nsteps, int nbatch, const double* s0,
                       double* out) {
  if (N < 4 || N > kNl1dMaxN || (N & 1) || !(kmax > 0.0) || kmax > N / 2 || !(dt > 0.0) ||
      !std::isfinite(dt) || nsteps < 0 || nbatch < 1 || nbatch > 65535 || !s0 || !out)
    return NS_ERR_INVALID_ARG;
  const size_t in_b = sizeof(double) * (size_t)nbatch * N;
  const size_t out_b = sizeof(double) * (size_t)nbatch * (N / 2 + 1) * 2;
  const size_t smem = Nl1dSmem::bytes(N);
  double *d_in = nullptr, *d_out = nullptr;
  int rc = NS_ERR_CUDA;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_nl1d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    goto done;
  if ((e = cudaMalloc(&d_in, in_b)) != cudaSuccess || (e = cudaMalloc(&d_out, out_b)) != cudaSuccess) goto done;
  if ((e = cudaMemcpy(d_in, s0, in_b, cudaMemcpyHostToDevice)) != cudaSuccess) goto done;
  k_nl1d<<<nbatch, 256, smem>>>(N, kmax, dt, nsteps, d_in, d_out);
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  if ((e = cudaMemcpy(out, d_out, out_b, cudaMemcpyDeviceToHost)) != cudaSuccess) goto done;
  rc = NS_OK;
done:
  if (rc != NS_OK && e == cudaErrorMemoryAllocation) rc = NS_ERR_OOM;
  cudaFree(d_in);
  cudaFree(d_out);
  return rc;
}
