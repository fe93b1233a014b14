// ns_kernels.cuh -- the CUDA kernels of one pseudo-spectral Navier-Stokes evaluation.
//
// Data layout in HBM (complex values of type cpx<T>, T = float or double):
//   state / acc   [3][kz][ky][kx]      spectral, kx = 0..N/2-1 contiguous
//   mixed         [5][z][ky][kx]       after the inverse z transform: u_x, u_y, u_z,
//                                      d_z u_x, d_z u_y (phase shift already applied)
//   Ft            [3][z][ky][kx]       FFT_xy of u x omega (mixed space)
//   scratch       [6][g][y][kx]        y-transformed planes of the current plane group
//                                      (L2-resident for small groups; the group size is
//                                      autotuned and may be the whole grid)
// One evaluation of the nonlinear term = slab pass over all planes (k_yinv -> k_xrow ->
// k_yfwd per plane group) followed by one pencil pass (k_pencil) that ends the forward
// transform and applies the whole spectral stage of Sec. 4 in the same HBM pass.
#pragma once

#include "ns_fft.cuh"

namespace ns {

enum PencilMode {
  MODE_INIT = 0,     // S_next = S0 (state)
  MODE_RK2_1 = 1,    // S_next = (S0 + dt/2 N) E_{dt/2}
  MODE_RK2_2 = 2,    // S = S0 E_dt + dt E_{dt/2} N -> state;      S_next = S
  MODE_RK4_1 = 3,    // acc = S0 E_dt + dt/6 E_dt N;               S_next = (S0 + dt/2 N) E_{dt/2}
  MODE_RK4_2 = 4,    // acc += dt/3 E_{dt/2} N;                    S_next = S0 E_{dt/2} + dt/2 N
  MODE_RK4_3 = 5,    // acc += dt/3 E_{dt/2} N;                    S_next = S0 E_dt + dt E_{dt/2} N
  MODE_RK4_4 = 6,    // S = acc + dt/6 N -> state;                 S_next = S
  MODE_ROG_1 = 7,    // A = S0 E_dt + dt/2 E_{dt/2} N -> state;    S_next = (S0 + dt N) E_dt
  MODE_ROG_2 = 8,    // S = A + dt/2 E_{dt/2} N -> state;          S_next = S
  MODE_NL = 9,       // acc = N
  MODE_PROJECT = 10  // state = N (input is a velocity: truncation + projection only)
};

// XMODE_ADJ_WR / XMODE_ADJ_RU: adjoint slab passes, u x omega replaced by omega x r and
// r x u (r: the mixed fields of the cotangent, in SlabArgs::mixedB)
enum XMode { XMODE_NONLINEAR = 0, XMODE_C2R = 1, XMODE_R2C = 2, XMODE_ADJ_WR = 3, XMODE_ADJ_RU = 4 };
__host__ __device__ __forceinline__ bool xmode_cross(int m) {
  return m == XMODE_NONLINEAR || m == XMODE_ADJ_WR || m == XMODE_ADJ_RU;
}

enum ErrBits { ERR_FFT_SHAPE = 1, ERR_LAUNCH_SHAPE = 2 };

__device__ __forceinline__ int kof(int i, int N) { return i < (N >> 1) ? i : i - N; }

// ----------------------------------------------------------------------------------------
// Tables (FP64 arithmetic, rounded to T)
// ----------------------------------------------------------------------------------------
// Truncation mask T at mode k (Sec. 3.2; Sec. 4.2 for the double aliases).  trunc 1, cubic:
// max_i |k_i| <= Kimax.  Otherwise spherical: |k|^2 <= K2max; trunc 2 also drops the modes a
// double alias can reach: |k + N e|^2 <= 4 K2max for some e with exactly one zero component,
// whose closest member gives (N - |k_i|)^2 + (N - |k_j|)^2 + k_l^2 for the pair (i, j).
__device__ __forceinline__ bool trunc_keep(int trunc, int kx, int ky, int kz, int N, int K2max, int Kimax) {
  if (trunc == 1) return max(abs(kx), max(abs(ky), abs(kz))) <= Kimax;
  const long long x2 = (long long)kx * kx, y2 = (long long)ky * ky, z2 = (long long)kz * kz;
  if (x2 + y2 + z2 > (long long)K2max) return false;
  if (trunc != 2) return true;
  const long long ax = N - abs(kx), ay = N - abs(ky), az = N - abs(kz), m4 = 4LL * K2max;
  return ax * ax + ay * ay + z2 > m4 && ax * ax + az * az + y2 > m4 && ay * ay + az * az + x2 > m4;
}

template <typename T>
__global__ void k_twiddle(cpx<T>* tw, int N) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)N, &s, &c);
  tw[k] = mk<T>((T)c, (T)(-s));
}

// out[j * N + i] = exp(-nu k(i)^2 tau_j), j = 0, 1
template <typename T>
__global__ void k_ifac(T* out, int N, double nu, double tau0, double tau1) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double k = (double)kof(i, N);
  out[i] = (T)exp(-nu * k * k * tau0);
  out[N + i] = (T)exp(-nu * k * k * tau1);
}

// out[(s * 3 + d) * N + i] = exp(i k(i) delta[s][d])  (Sec. 4.2, Eq. shift_operator_3d)
template <typename T>
__global__ void k_shift_tables(cpx<T>* out, int N, const double* __restrict__ delta, int nshift) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nshift * 3 * N) return;
  int i = idx % N, sd = idx / N;
  double a = (double)kof(i, N) * delta[sd];
  double s, c;
  sincos(a, &s, &c);
  out[idx] = mk<T>((T)c, (T)s);
}

// ----------------------------------------------------------------------------------------
// Pencil pass: z transforms + spectral stage
// ----------------------------------------------------------------------------------------
template <typename T>
struct PencilArgs {
  int N, M, TX;
  FFTPlan pz;
  const cpx<T>* tw;
  int nF;                // number of nonlinear inputs (0, 1, 2)
  const cpx<T>* F[2];    // [3][N][N][M]
  const cpx<T>* dsh[2];  // shift tables of the inputs ([3][N]) or null (no shift)
  T wF[2];               // weights of the inputs (1/N^3 or 1/(2 N^3))
  int mode;
  T dt;
  const T* ifac;         // [2][N]: tau = dt, dt/2
  cpx<T>* state;
  cpx<T>* acc;
  const cpx<T>* src;     // MODE_INIT source (state or a temporary)
  int trunc, K2max, Kimax;
  const cpx<T>* force;   // [3][D] dense table of the forcing term, or null
  cpx<T>* shell;         // [3][D] S_next at the forcing table's modes, or null
  int fK;                // forcing table half-width (D = (2fK+1)^2 (fK+1))
  int nOut;
  const cpx<T>* osh[2];  // shift tables of the outputs
  cpx<T>* out[2];        // [5][N][N][M]
  int* err;
  double* epart;         // [tiles][2]: sums of w |S|^2 and w k^2 |S|^2 of the written state, or null
  int iy0;               // first ky row of the launch (rank-range passes; 0 for a whole field)
};

template <typename T>
__device__ __forceinline__ cpx<T> phase3(const cpx<T>* tab, int N, int ix, int iy, int iz) {
  return (ldg(&tab[ix]) * ldg(&tab[N + iy])) * ldg(&tab[2 * N + iz]);
}

template <typename T>
__device__ __forceinline__ void load_tile(cpx<T>* dst, const cpx<T>* __restrict__ src, int N,
                                          int M, int TX, int iy, int x0) {
  const int n = N * TX;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int z = e / TX, x = e - z * TX;
    dst[e] = src[((size_t)z * N + iy) * M + x0 + x];
  }
}

template <typename T>
__device__ __forceinline__ void store_tile(cpx<T>* __restrict__ dst, const cpx<T>* src, int N,
                                           int M, int TX, int iy, int x0) {
  const int n = N * TX;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    int z = e / TX, x = e - z * TX;
    dst[((size_t)z * N + iy) * M + x0 + x] = src[e];
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_pencil(PencilArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int N = a.N, M = a.M, TX = a.TX;
  const int ntx = M / TX;
  const int iy = a.iy0 + blockIdx.x / ntx;
  const int x0 = (blockIdx.x % ntx) * TX;
  const int tile = N * TX;
  cpx<T>* b[4] = {buf, buf + tile, buf + 2 * tile, buf + 3 * tile};
  const size_t fstride = (size_t)N * N * M;
  const int ky = kof(iy, N);

  // 1) forward z transforms of the nonlinear inputs, de-shift, weights
  if (a.nF > 0) {
    for (int c = 0; c < 3; ++c) {
      load_tile(b[c], a.F[0] + c * fstride, N, M, TX, iy, x0);
      __syncthreads();
      fft_lines(b[c], a.pz, TX, TX, 1, true, a.tw, T(-1), a.err);
      if (a.nF > 1) {
        load_tile(b[3], a.F[1] + c * fstride, N, M, TX, iy, x0);
        __syncthreads();
        fft_lines(b[3], a.pz, TX, TX, 1, true, a.tw, T(-1), a.err);
      }
      for (int e = threadIdx.x; e < tile; e += blockDim.x) {
        int iz = e / TX, x = e - iz * TX;
        cpx<T> v = b[c][e];
        if (a.dsh[0]) v = mul_conj(v, phase3(a.dsh[0], N, x0 + x, iy, iz));
        v = a.wF[0] * v;
        if (a.nF > 1) {
          cpx<T> w = b[3][e];
          if (a.dsh[1]) w = mul_conj(w, phase3(a.dsh[1], N, x0 + x, iy, iz));
          v = v + a.wF[1] * w;
        }
        b[c][e] = v;
      }
      __syncthreads();
    }
  }

  // 2) pointwise: N(0) = 0, truncation T, projection P, forcing, stage combine
  const T dt = a.dt, hdt = T(0.5) * a.dt;
  const int D1 = 2 * a.fK + 1;
  const int D = D1 * D1 * (a.fK + 1);
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int iz = e / TX, x = e - iz * TX;
    const int kx = x0 + x, kz = kof(iz, N);
    const size_t g = ((size_t)iz * N + iy) * M + kx;
    cpx<T> nv[3];
    if (a.nF > 0) {
      const int k2 = kx * kx + ky * ky + kz * kz;
      const bool keep = trunc_keep(a.trunc, kx, ky, kz, N, a.K2max, a.Kimax) && (k2 != 0);
      if (keep) {
        cpx<T> v0 = b[0][e], v1 = b[1][e], v2 = b[2][e];
        const T fx = (T)kx, fy = (T)ky, fz = (T)kz;
        const T ik2 = T(1) / (T)k2;
        cpx<T> kd = mk<T>(fx * v0.x + fy * v1.x + fz * v2.x, fx * v0.y + fy * v1.y + fz * v2.y);
        nv[0] = v0 - (fx * ik2) * kd;
        nv[1] = v1 - (fy * ik2) * kd;
        nv[2] = v2 - (fz * ik2) * kd;
      } else {
        nv[0] = nv[1] = nv[2] = mk<T>(0, 0);
      }
      if (a.force && kx <= a.fK && abs(ky) <= a.fK && abs(kz) <= a.fK) {
        const int fi = ((kz + a.fK) * D1 + (ky + a.fK)) * (a.fK + 1) + kx;
#pragma unroll
        for (int c = 0; c < 3; ++c) nv[c] = nv[c] + a.force[c * D + fi];
      }
    }
    T E1 = 1, Eh = 1;
    if (a.mode != MODE_INIT && a.mode != MODE_NL && a.mode != MODE_PROJECT) {
      E1 = a.ifac[kx] * a.ifac[iy] * a.ifac[iz];
      Eh = a.ifac[N + kx] * a.ifac[N + iy] * a.ifac[N + iz];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t gi = g + c * fstride;
      cpx<T> sn = mk<T>(0, 0);
      switch (a.mode) {
        case MODE_INIT:
          sn = a.src[gi];
          break;
        case MODE_RK2_1: {
          cpx<T> s0 = a.state[gi];
          sn = Eh * (s0 + hdt * nv[c]);
        } break;
        case MODE_RK2_2: {
          cpx<T> s0 = a.state[gi];
          sn = E1 * s0 + (dt * Eh) * nv[c];
          a.state[gi] = sn;
        } break;
        case MODE_RK4_1: {
          cpx<T> s0 = a.state[gi];
          a.acc[gi] = E1 * s0 + (dt / T(6) * E1) * nv[c];
          sn = Eh * (s0 + hdt * nv[c]);
        } break;
        case MODE_RK4_2: {
          cpx<T> s0 = a.state[gi];
          a.acc[gi] = a.acc[gi] + (dt / T(3) * Eh) * nv[c];
          sn = Eh * s0 + hdt * nv[c];
        } break;
        case MODE_RK4_3: {
          cpx<T> s0 = a.state[gi];
          a.acc[gi] = a.acc[gi] + (dt / T(3) * Eh) * nv[c];
          sn = E1 * s0 + (dt * Eh) * nv[c];
        } break;
        case MODE_RK4_4: {
          sn = a.acc[gi] + (dt / T(6)) * nv[c];
          a.state[gi] = sn;
        } break;
        case MODE_ROG_1: {
          cpx<T> s0 = a.state[gi];
          a.state[gi] = E1 * s0 + (hdt * Eh) * nv[c];
          sn = E1 * (s0 + dt * nv[c]);
        } break;
        case MODE_ROG_2: {
          sn = a.state[gi] + (hdt * Eh) * nv[c];
          a.state[gi] = sn;
        } break;
        case MODE_NL:
          a.acc[gi] = nv[c];
          break;
        case MODE_PROJECT:
          a.state[gi] = nv[c];
          break;
      }
      b[c][e] = sn;
      if (a.shell && kx <= a.fK && abs(ky) <= a.fK && abs(kz) <= a.fK) {
        const int fi = ((kz + a.fK) * D1 + (ky + a.fK)) * (a.fK + 1) + kx;
        a.shell[c * D + fi] = sn;
      }
    }
  }
  __syncthreads();

  // 3) outputs: shift, z-derivatives, inverse z transforms
  for (int o = 0; o < a.nOut; ++o) {
    for (int f = 0; f < 5; ++f) {
      const int c = f < 3 ? f : f - 3;
      for (int e = threadIdx.x; e < tile; e += blockDim.x) {
        const int iz = e / TX, x = e - iz * TX;
        cpx<T> v = b[c][e];
        if (a.osh[o]) v = v * phase3(a.osh[o], N, x0 + x, iy, iz);
        if (f >= 3) v = mul_si(v, (T)kof(iz, N));  // i kz v
        b[3][e] = v;
      }
      __syncthreads();
      fft_lines(b[3], a.pz, TX, TX, 1, true, a.tw, T(1), a.err);
      store_tile(a.out[o] + f * fstride, b[3], N, M, TX, iy, x0);
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------------------------------
// Slab pass: y transforms and the x rows with the real-space cross product
// ----------------------------------------------------------------------------------------
template <typename T>
struct SlabArgs {
  int N, M, z0, G;
  FFTPlan py, px;
  const cpx<T>* tw;
  const cpx<T>* mixed;  // [5][N][N][M]
  const cpx<T>* mixedB; // [5][N][N][M] cotangent fields r (adjoint modes; first 3 used)
  cpx<T>* scr;          // [6][G][N][M]
  cpx<T>* Ft;           // [3][N][N][M]
  T* rio;               // physical rows [3][N][N][N] (C2R output / R2C input)
  int TY, RX, xmode;
  int* err;
  void* umax;           // or null: max_x |u_i(x)| of the velocity rows, i = 0..2, folded in
                        // with atomicMax on the IEEE bits (unsigned / unsigned long long [3])
  // modes of Ft no pencil pass reads (skip_tx > 0: the compile-time y-forward leaves them
  // unwritten): those of pencil tiles of skip_tx columns outside the truncation (trunc, K2max,
  // Kimax) and outside the forcing block |k| <= fK (fK < 0: no forcing)
  int skip_tx, trunc, K2max, Kimax, fK;
};

// Block maxima m0..m2 (non-negative) folded into umax[0..2], one atomic per value per block:
// the bit patterns of non-negative IEEE numbers order like the numbers, so an unsigned
// atomicMax is a max of the values.  scratch: 3 (blockDim.x / 32) values of shared memory
// that are free during the call; every thread of the block calls it (blockDim.x is a
// multiple of 32).
template <typename T>
__device__ void block_max3(T m0, T m1, T m2, T* scratch, void* umax) {
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    scratch[3 * w] = m0;
    scratch[3 * w + 1] = m1;
    scratch[3 * w + 2] = m2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    T m = T(0);
    for (int i = 0; i < nw; ++i) m = fmax(m, scratch[3 * i + threadIdx.x]);
    if (sizeof(T) == 4)
      atomicMax(static_cast<unsigned*>(umax) + threadIdx.x, __float_as_uint((float)m));
    else
      atomicMax(static_cast<unsigned long long*>(umax) + threadIdx.x,
                (unsigned long long)__double_as_longlong((double)m));
  }
  __syncthreads();
}

// inverse y transforms; forms omega = i k x u from the mixed fields (nonlinear mode) or
// passes the velocity only (C2R mode).  grid (M/TY, G)
template <typename T>
__global__ void __launch_bounds__(512) k_yinv(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int N = a.N, M = a.M, TY = a.TY;
  const int x0 = blockIdx.x * TY, zg = blockIdx.y, z = a.z0 + zg;
  const int tile = N * TY;
  const size_t fstride = (size_t)N * N * M;
  const int nf = xmode_cross(a.xmode) ? 6 : 3;
  for (int e = threadIdx.x; e < tile; e += blockDim.x) {
    const int iy = e / TY, x = e - iy * TY;
    const size_t g = ((size_t)z * N + iy) * M + x0 + x;
    cpx<T> ux = a.mixed[g], uy = a.mixed[g + fstride], uz = a.mixed[g + 2 * fstride];
    // slots 0..2 and 3..5 of the pair whose cross product the x rows form
    int su = 0, sw = 3, sr = -1;
    if (a.xmode == XMODE_ADJ_WR) { sw = 0; sr = 3; su = -1; }
    if (a.xmode == XMODE_ADJ_RU) { sr = 0; su = 3; sw = -1; }
    if (su >= 0) {
      buf[su * tile + e] = ux;
      buf[(su + 1) * tile + e] = uy;
      buf[(su + 2) * tile + e] = uz;
    }
    if (nf == 6 && sw >= 0) {
      cpx<T> dzx = a.mixed[g + 3 * fstride], dzy = a.mixed[g + 4 * fstride];
      const T kx = (T)(x0 + x), ky = (T)kof(iy, N);
      buf[sw * tile + e] = mul_si(uz, ky) - dzy;                  // w_x = i ky uz - dz uy
      buf[(sw + 1) * tile + e] = dzx - mul_si(uz, kx);            // w_y = dz ux - i kx uz
      buf[(sw + 2) * tile + e] = mul_si(uy, kx) - mul_si(ux, ky); // w_z = i kx uy - i ky ux
    }
    if (sr >= 0) {
      buf[sr * tile + e] = a.mixedB[g];
      buf[(sr + 1) * tile + e] = a.mixedB[g + fstride];
      buf[(sr + 2) * tile + e] = a.mixedB[g + 2 * fstride];
    }
  }
  __syncthreads();
  for (int f = 0; f < nf; ++f) fft_lines(buf + f * tile, a.py, TY, TY, 1, true, a.tw, T(1), a.err);
  const size_t sstride = (size_t)a.G * N * M;
  for (int f = 0; f < nf; ++f) {
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int iy = e / TY, x = e - iy * TY;
      a.scr[f * sstride + ((size_t)zg * N + iy) * M + x0 + x] = buf[f * tile + e];
    }
  }
}

// forward y transforms of the 3 components of the x-transformed product.  grid (M/TY, G)
template <typename T>
__global__ void __launch_bounds__(512) k_yfwd(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int N = a.N, M = a.M, TY = a.TY;
  const int x0 = blockIdx.x * TY, zg = blockIdx.y, z = a.z0 + zg;
  const int tile = N * TY;
  const size_t fstride = (size_t)N * N * M;
  const size_t sstride = (size_t)a.G * N * M;
  for (int f = 0; f < 3; ++f) {
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int iy = e / TY, x = e - iy * TY;
      buf[f * tile + e] = a.scr[f * sstride + ((size_t)zg * N + iy) * M + x0 + x];
    }
  }
  __syncthreads();
  for (int f = 0; f < 3; ++f) fft_lines(buf + f * tile, a.py, TY, TY, 1, true, a.tw, T(-1), a.err);
  for (int f = 0; f < 3; ++f) {
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
      const int iy = e / TY, x = e - iy * TY;
      a.Ft[f * fstride + ((size_t)z * N + iy) * M + x0 + x] = buf[f * tile + e];
    }
  }
}

// Hermitian half spectrum X_0..X_{M-1} (X_M = 0) -> Z'_k whose inverse M-point DFT is the
// packed real row z_m = x_{2m} + i x_{2m+1}, x_j = sum_{k=0}^{N-1} X_k exp(2 pi i jk/N).
template <typename T>
__device__ __forceinline__ void c2r_pre(cpx<T>* row, int M, const cpx<T>* __restrict__ tw,
                                        int k) {
  if (k == 0) {
    const T r = row[0].x;
    row[0] = mk<T>(r, r);
    if (M % 2 == 0 && M > 1) {
      // k = M/2: X_{M-k} = X_k; e^{2 pi i k/N} = e^{i pi/2} = i
      cpx<T> X = row[M / 2];
      cpx<T> A = X + conjg(X), B = X - conjg(X);
      row[M / 2] = A - B;  // A + i * i * B
    }
    return;
  }
  const int km = M - k;
  cpx<T> Xk = row[k], Xm = row[km];
  cpx<T> w = conjg(ldg(&tw[k]));  // e^{+2 pi i k / N}
  cpx<T> A = Xk + conjg(Xm), B = Xk - conjg(Xm);
  row[k] = A + mul_si(w * B, T(1));
  // for M-k: e^{2 pi i (M-k)/N} = -e^{-2 pi i k/N} = -tw[k]
  cpx<T> A2 = Xm + conjg(Xk), B2 = Xm - conjg(Xk);
  row[km] = A2 - mul_si(ldg(&tw[k]) * B2, T(1));
}

// Z_k (forward M-point DFT of the packed real row) -> X_k = sum_j x_j e^{-2 pi i jk/N}, k < M
template <typename T>
__device__ __forceinline__ void r2c_post(cpx<T>* row, int M, const cpx<T>* __restrict__ tw,
                                         int k) {
  if (k == 0) {
    const cpx<T> Z = row[0];
    row[0] = mk<T>(Z.x + Z.y, T(0));
    if (M % 2 == 0 && M > 1) {
      // k = M/2: W^k = e^{-i pi/2} = -i
      cpx<T> Zk = row[M / 2];
      cpx<T> A = Zk + conjg(Zk), B = Zk - conjg(Zk);
      // X = A/2 - i/2 (-i) B = A/2 - B/2
      row[M / 2] = T(0.5) * (A - B);
    }
    return;
  }
  const int km = M - k;
  cpx<T> Zk = row[k], Zm = row[km];
  cpx<T> W = ldg(&tw[k]);  // e^{-2 pi i k/N}
  cpx<T> A = Zk + conjg(Zm), B = Zk - conjg(Zm);
  row[k] = T(0.5) * (A - mul_si(W * B, T(1)));
  // W^{M-k} = -conj(W)
  cpx<T> A2 = Zm + conjg(Zk), B2 = Zm - conjg(Zk);
  row[km] = T(0.5) * (A2 + mul_si(conjg(W) * B2, T(1)));
}

// x rows: c2r of 6 fields, u x omega, r2c of 3 fields (nonlinear mode); c2r of 3 fields to
// physical rows (C2R); r2c of 3 physical rows (R2C).  grid ceil(G*N / RX)
template <typename T>
__global__ void __launch_bounds__(512) k_xrow(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int N = a.N, M = a.M, RX = a.RX;
  const int rows_total = a.G * N;
  const int r0 = blockIdx.x * RX;
  const int nr = min(RX, rows_total - r0);
  if (nr <= 0) return;
  const int tile = RX * M;
  const size_t sstride = (size_t)a.G * N * M;
  const int nin = xmode_cross(a.xmode) ? 6 : 3;
  const size_t plane = (size_t)N * N;

  // load
  for (int f = 0; f < nin; ++f) {
    for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
      const int r = e / M, k = e - r * M;
      if (a.xmode == XMODE_R2C) {
        const int rr = r0 + r, zg = rr / N, y = rr - zg * N;
        const T* src = a.rio + (size_t)f * plane * N + ((size_t)(a.z0 + zg) * N + y) * N;
        buf[f * tile + e] = mk<T>(src[2 * k], src[2 * k + 1]);
      } else {
        buf[f * tile + e] = a.scr[f * sstride + (size_t)(r0 + r) * M + k];
      }
    }
  }
  // zero unused rows so the FFT batch is well defined
  for (int f = 0; f < nin; ++f)
    for (int e = nr * M + threadIdx.x; e < tile; e += blockDim.x) buf[f * tile + e] = mk<T>(0, 0);
  __syncthreads();

  if (a.xmode != XMODE_R2C) {
    const int npair = M / 2 + 1;
    for (int e = threadIdx.x; e < nin * RX * npair; e += blockDim.x) {
      const int fr = e / npair, k = e - fr * npair;
      if (k == 0 || k < M - k) c2r_pre(buf + fr * M, M, a.tw, k);
    }
    __syncthreads();
    for (int f = 0; f < nin; ++f) fft_lines(buf + f * tile, a.px, RX, 1, M, false, a.tw, T(1), a.err);
  }

  if (a.xmode == XMODE_C2R) {
    for (int f = 0; f < 3; ++f) {
      for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
        const int r = e / M, k = e - r * M;
        const int rr = r0 + r, zg = rr / N, y = rr - zg * N;
        T* dst = a.rio + (size_t)f * plane * N + ((size_t)(a.z0 + zg) * N + y) * N;
        cpx<T> v = buf[f * tile + e];
        dst[2 * k] = v.x;
        dst[2 * k + 1] = v.y;
      }
    }
    return;
  }

  if (xmode_cross(a.xmode)) {
    // (fields 0..2) x (fields 3..5) on the packed real rows, written over fields 0..2
    T* re = reinterpret_cast<T*>(buf);
    const int rt = 2 * tile;  // reals per field
    T m0 = 0, m1 = 0, m2 = 0;
    for (int e = threadIdx.x; e < 2 * nr * M; e += blockDim.x) {
      const T u0 = re[e], u1 = re[rt + e], u2 = re[2 * rt + e];
      const T w0 = re[3 * rt + e], w1 = re[4 * rt + e], w2 = re[5 * rt + e];
      m0 = fmax(m0, fabs(u0));
      m1 = fmax(m1, fabs(u1));
      m2 = fmax(m2, fabs(u2));
      re[e] = u1 * w2 - u2 * w1;
      re[rt + e] = u2 * w0 - u0 * w2;
      re[2 * rt + e] = u0 * w1 - u1 * w0;
    }
    __syncthreads();
    // CFL: max |u_i| of the rows (omega, fields 3..5, is no longer needed: scratch)
    if (a.umax && a.xmode == XMODE_NONLINEAR) block_max3<T>(m0, m1, m2, re + 3 * rt, a.umax);
  }

  // forward r2c of fields 0..2
  for (int f = 0; f < 3; ++f) fft_lines(buf + f * tile, a.px, RX, 1, M, false, a.tw, T(-1), a.err);
  {
    const int npair = M / 2 + 1;
    for (int e = threadIdx.x; e < 3 * RX * npair; e += blockDim.x) {
      const int fr = e / npair, k = e - fr * npair;
      if (k == 0 || k < M - k) r2c_post(buf + fr * M, M, a.tw, k);
    }
  }
  __syncthreads();
  for (int f = 0; f < 3; ++f) {
    for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
      const int r = e / M, k = e - r * M;
      a.scr[f * sstride + (size_t)(r0 + r) * M + k] = buf[f * tile + e];
    }
  }
}

// ----------------------------------------------------------------------------------------
// Forcing amplitude (Sec. 2 / 6.1; reading: an Euler step of the forcing injects eps*dt)
// ----------------------------------------------------------------------------------------
template <typename T>
__global__ void k_force_coef(const cpx<double>* __restrict__ pj, const cpx<double>* __restrict__ pj1,
                             double theta, const cpx<T>* __restrict__ shell, int fK, double dt,
                             double eps, cpx<T>* force, double* coef_out) {
  __shared__ double sb[256], sc[256];
  const int D1 = 2 * fK + 1, D = D1 * D1 * (fK + 1);
  double b = 0, c = 0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const int kx = i % (fK + 1);
    const double w = kx == 0 ? 1.0 : 2.0;
    for (int comp = 0; comp < 3; ++comp) {
      cpx<double> p0 = pj[comp * D + i], p1 = pj1[comp * D + i];
      double fx = (1.0 - theta) * p0.x + theta * p1.x;
      double fy = (1.0 - theta) * p0.y + theta * p1.y;
      cpx<T> s = shell[comp * D + i];
      b += w * ((double)s.x * fx + (double)s.y * fy);
      c += w * (fx * fx + fy * fy);
    }
  }
  sb[threadIdx.x] = b;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sb[threadIdx.x] += sb[threadIdx.x + s];
      sc[threadIdx.x] += sc[threadIdx.x + s];
    }
    __syncthreads();
  }
  const double B = sb[0], C = 0.5 * dt * sc[0];
  const double q = sqrt(B * B + 4.0 * C * eps);
  const double amp = (B >= 0.0) ? 2.0 * eps / (B + q) : 2.0 * eps / (B - q);
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    for (int comp = 0; comp < 3; ++comp) {
      cpx<double> p0 = pj[comp * D + i], p1 = pj1[comp * D + i];
      double fx = (1.0 - theta) * p0.x + theta * p1.x;
      double fy = (1.0 - theta) * p0.y + theta * p1.y;
      force[comp * D + i] = mk<T>((T)(amp * fx), (T)(amp * fy));
    }
  }
  if (threadIdx.x == 0 && coef_out) coef_out[0] = amp;
}

// ----------------------------------------------------------------------------------------
// Reductions (FP64 across threads and blocks; per thread FP64, or compensated FP32 for FP32
// states; fixed-order tree: bitwise reproducible)
// ----------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_energy(const cpx<T>* __restrict__ S, int N, double nu,
                                                double* partial) {
  __shared__ double se[256], sd[256];
  const int M = N / 2;
  const size_t nmode = (size_t)N * N * M;
  double e = 0, d = 0;
  if constexpr (sizeof(T) == 4) {
    // FP32 state: the terms in FP32 and each thread's share (about a hundred modes) summed
    // with compensated (Kahan) FP32 additions, then the partial sums reduced in FP64 (FP64
    // arithmetic per mode is ALU-bound on this GPU)
    float es = 0.f, ec = 0.f, ds = 0.f, dc = 0.f;
    auto kahan = [](float& sum, float& comp, float x) {
      const float y = x - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    };
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nmode;
         i += (size_t)gridDim.x * blockDim.x) {
      const int kx = (int)(i % M);
      const size_t r = i / M;
      const int iy = (int)(r % N), iz = (int)(r / N);
      const int ky = kof(iy, N), kz = kof(iz, N);
      float a2 = 0.f;
      for (int c = 0; c < 3; ++c) {
        const cpx<T> v = S[i + c * nmode];
        a2 = fmaf((float)v.x, (float)v.x, fmaf((float)v.y, (float)v.y, a2));
      }
      const float te = (kx == 0 ? 1.f : 2.f) * a2;
      kahan(es, ec, te);
      kahan(ds, dc, te * (float)(kx * kx + ky * ky + kz * kz));
    }
    e = (double)es - (double)ec;
    d = (double)ds - (double)dc;
  } else {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nmode;
         i += (size_t)gridDim.x * blockDim.x) {
      const int kx = (int)(i % M);
      const size_t r = i / M;
      const int iy = (int)(r % N), iz = (int)(r / N);
      const int ky = kof(iy, N), kz = kof(iz, N);
      const double w = kx == 0 ? 1.0 : 2.0;
      double a2 = 0;
      for (int c = 0; c < 3; ++c) {
        cpx<T> v = S[i + c * nmode];
        a2 += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
      }
      e += w * a2;
      d += w * (double)(kx * kx + ky * ky + kz * kz) * a2;
    }
  }
  se[threadIdx.x] = e;
  sd[threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      se[threadIdx.x] += se[threadIdx.x + s];
      sd[threadIdx.x] += sd[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = 0.5 * se[0];
    partial[2 * blockIdx.x + 1] = nu * sd[0];
  }
}

// out = (f0 * sum_i partial[2i], f1 * sum_i partial[2i+1]) in a fixed order (one block)
static __global__ void k_sum_pairs(const double* partial, int nblk, double* out, double f0 = 1.0,
                                   double f1 = 1.0) {
  __shared__ double s0[256], s1[256];
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s0[threadIdx.x] += s0[threadIdx.x + s];
      s1[threadIdx.x] += s1[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = f0 * s0[0];
    out[1] = f1 * s1[0];
  }
}

// spectrum partials: block b accumulates its modes into smem bins, writes partial[b][bin]
// Binned quadratic forms of the half spectrum, weights 1/2 at kx = 0 and 1 elsewhere (so a
// bin holds half the full-spectrum sum): q = 0, |S|^2 (energy spectrum); q = 1, 2 Re(S* . B)
// (nonlinear transfer T(k) for B = N); q = 2, 2 nu k^2 |S|^2 (dissipation spectrum).
template <typename T>
__global__ void __launch_bounds__(256) k_spectrum(const cpx<T>* __restrict__ S, int N, int kind,
                                                  int nbins, double* partial, int q = 0,
                                                  const cpx<T>* __restrict__ B = nullptr,
                                                  double nu = 0.0) {
  extern __shared__ double bins[];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) bins[i] = 0.0;
  __syncthreads();
  const int M = N / 2;
  const size_t nmode = (size_t)N * N * M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nmode;
       i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % M);
    const size_t r = i / M;
    const int iy = (int)(r % N), iz = (int)(r / N);
    const int ky = kof(iy, N), kz = kof(iz, N);
    double a2 = 0;
    for (int c = 0; c < 3; ++c) {
      const cpx<T> v = S[i + c * nmode];
      if (q == 1) {
        const cpx<T> b = B[i + c * nmode];
        a2 += 2.0 * ((double)v.x * (double)b.x + (double)v.y * (double)b.y);
      } else {
        a2 += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
      }
    }
    if (q == 2) a2 *= 2.0 * nu * (double)(kx * kx + ky * ky + kz * kz);
    if (a2 == 0.0) continue;
    const double w = kx == 0 ? 0.5 : 1.0;
    int bin;
    if (kind == 0) {
      bin = (int)floor(sqrt((double)(kx * kx + ky * ky + kz * kz)) + 0.5);
    } else if (kind == 1) {
      bin = kx;
    } else if (kind == 2) {
      bin = abs(ky);
    } else {
      bin = abs(kz);
    }
    if (bin < nbins) atomicAdd(&bins[bin], w * a2);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) partial[(size_t)blockIdx.x * nbins + i] = bins[i];
}

static __global__ void k_spectrum_final(const double* partial, int nblk, int nbins, double* out) {
  int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= nbins) return;
  double s = 0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * nbins + bin];
  out[bin] = s;
}

// ----------------------------------------------------------------------------------------
// Adjoint step building blocks (pointwise on [3][N][N][M] spectral arrays)
// ----------------------------------------------------------------------------------------
enum EwOp {
  EW_ROG_S1 = 0,   // o = E_dt (x + dt y)                         (S1 = E(S0 + dt N0))
  EW_ROG_SN = 1,   // o = E_dt x + dt/2 E_{dt/2} (y + z)          (S = E S0 + dt/2 Eh (N0 + N1))
  EW_RHO = 2,      // o = dt/2 E_{dt/2} x
  EW_SIGMA = 3,    // o = dt E_dt x
  EW_LAMBDA = 4,   // o = E_dt (x + y) + z
  EW_ADD = 5,      // o = x + y
  EW_LOSS = 6,     // o = 2 nu k^2 x        (gradient of eps = nu <S, k^2 S>_w)
  EW_SCALE = 7,    // o = c x
  EW_CURL_ADD = 8  // o = x + i k x y
};

template <typename T>
__global__ void k_elementwise(int op, int N, T dt, T c, const T* __restrict__ ifac,
                              const cpx<T>* x, const cpx<T>* y, const cpx<T>* z, cpx<T>* o) {
  const int M = N / 2;
  const size_t nmode = (size_t)N * N * M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nmode;
       i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % M);
    const size_t r = i / M;
    const int iy = (int)(r % N), iz = (int)(r / N);
    const T E1 = ifac[kx] * ifac[iy] * ifac[iz];
    const T Eh = ifac[N + kx] * ifac[N + iy] * ifac[N + iz];
    const T fx = (T)kx, fy = (T)kof(iy, N), fz = (T)kof(iz, N);
    if (op == EW_CURL_ADD) {
      const cpx<T> y0 = y[i], y1 = y[i + nmode], y2 = y[i + 2 * nmode];
      o[i] = x[i] + mul_si(fy * y2 - fz * y1, T(1));
      o[i + nmode] = x[i + nmode] + mul_si(fz * y0 - fx * y2, T(1));
      o[i + 2 * nmode] = x[i + 2 * nmode] + mul_si(fx * y1 - fy * y0, T(1));
      continue;
    }
    for (int q = 0; q < 3; ++q) {
      const size_t j = i + q * nmode;
      cpx<T> v;
      switch (op) {
        case EW_ROG_S1: v = E1 * (x[j] + dt * y[j]); break;
        case EW_ROG_SN: v = E1 * x[j] + (T(0.5) * dt * Eh) * (y[j] + z[j]); break;
        case EW_RHO: v = (T(0.5) * dt * Eh) * x[j]; break;
        case EW_SIGMA: v = (dt * E1) * x[j]; break;
        case EW_LAMBDA: v = E1 * (x[j] + y[j]) + z[j]; break;
        case EW_ADD: v = x[j] + y[j]; break;
        case EW_LOSS: v = (T(2) * c * (fx * fx + fy * fy + fz * fz)) * x[j]; break;
        default: v = c * x[j]; break;
      }
      o[j] = v;
    }
  }
}

// dense forcing table [3][D] <-> spectral array at the table's modes
template <typename T>
__global__ void k_shell_gather(const cpx<T>* __restrict__ S, int N, int fK, cpx<T>* shell) {
  const int D1 = 2 * fK + 1, D = D1 * D1 * (fK + 1), M = N / 2;
  const size_t nmode = (size_t)N * N * M;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const int kx = i % (fK + 1), ky = (i / (fK + 1)) % D1 - fK, kz = i / ((fK + 1) * D1) - fK;
    const size_t g = ((size_t)((kz + N) % N) * N + (size_t)((ky + N) % N)) * M + kx;
    for (int c = 0; c < 3; ++c) shell[c * D + i] = S[g + c * nmode];
  }
}
template <typename T>
__global__ void k_shell_add(cpx<T>* S, int N, int fK, const cpx<T>* __restrict__ tab) {
  const int D1 = 2 * fK + 1, D = D1 * D1 * (fK + 1), M = N / 2;
  const size_t nmode = (size_t)N * N * M;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const int kx = i % (fK + 1), ky = (i / (fK + 1)) % D1 - fK, kz = i / ((fK + 1) * D1) - fK;
    const size_t g = ((size_t)((kz + N) % N) * N + (size_t)((ky + N) % N)) * M + kx;
    for (int c = 0; c < 3; ++c) S[g + c * nmode] = S[g + c * nmode] + tab[c * D + i];
  }
}

// adjoint of S -> a(S) f at one stage applied to rho: table = (da/db) Re<f, rho>_w f with
// da/db = -|a| / sqrt(b^2 + 4 c eps), b = Re<S, f>_w, c = dt/2 <f, f>_w
template <typename T>
__global__ void k_force_vjp(const cpx<double>* __restrict__ pj, const cpx<double>* __restrict__ pj1,
                            double theta, const cpx<T>* __restrict__ shS,
                            const cpx<T>* __restrict__ shR, int fK, double dt, double eps,
                            cpx<T>* tab) {
  __shared__ double sb[256], sc[256], sr[256];
  const int D1 = 2 * fK + 1, D = D1 * D1 * (fK + 1);
  double b = 0, c = 0, r = 0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const double w = (i % (fK + 1)) == 0 ? 1.0 : 2.0;
    for (int q = 0; q < 3; ++q) {
      const cpx<double> p0 = pj[q * D + i], p1 = pj1[q * D + i];
      const double fx = (1.0 - theta) * p0.x + theta * p1.x, fy = (1.0 - theta) * p0.y + theta * p1.y;
      const cpx<T> s = shS[q * D + i], x = shR[q * D + i];
      b += w * ((double)s.x * fx + (double)s.y * fy);
      c += w * (fx * fx + fy * fy);
      r += w * ((double)x.x * fx + (double)x.y * fy);
    }
  }
  sb[threadIdx.x] = b;
  sc[threadIdx.x] = c;
  sr[threadIdx.x] = r;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sb[threadIdx.x] += sb[threadIdx.x + s];
      sc[threadIdx.x] += sc[threadIdx.x + s];
      sr[threadIdx.x] += sr[threadIdx.x + s];
    }
    __syncthreads();
  }
  const double B = sb[0], C = 0.5 * dt * sc[0], R = sr[0];
  const double q = sqrt(B * B + 4.0 * C * eps);
  const double amp = (B >= 0.0) ? 2.0 * eps / (B + q) : 2.0 * eps / (B - q);
  const double coef = -fabs(amp) / q * R;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      const cpx<double> p0 = pj[k * D + i], p1 = pj1[k * D + i];
      const double fx = (1.0 - theta) * p0.x + theta * p1.x, fy = (1.0 - theta) * p0.y + theta * p1.y;
      tab[k * D + i] = mk<T>((T)(coef * fx), (T)(coef * fy));
    }
  }
}

// convert between the working precision and FP64 (state transfers)
template <typename T>
__global__ void k_to_double(const cpx<T>* __restrict__ in, cpx<double>* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cpx<T> v = in[i];
    out[i] = mk<double>((double)v.x, (double)v.y);
  }
}
template <typename T>
__global__ void k_from_double(const cpx<double>* __restrict__ in, cpx<T>* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cpx<double> v = in[i];
    out[i] = mk<T>((T)v.x, (T)v.y);
  }
}
template <typename T>
__global__ void k_real_to_double(const T* __restrict__ in, double* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
template <typename T>
__global__ void k_real_from_double(const double* __restrict__ in, T* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}

}  // namespace ns
