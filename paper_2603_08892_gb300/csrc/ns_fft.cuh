// ns_fft.cuh -- complex arithmetic and the shared-memory mixed-radix FFT used by every pass.
//
// The transforms are the discrete Fourier transforms of supplementary Eq. (dft_def) along
// one direction at a time: forward X_k = sum_j x_j exp(-2 pi i jk/n), inverse with
// exp(+2 pi i jk/n), both unnormalised (the 1/N^3 factor is applied once, in the spectral
// stage).  Lines of a batch live in shared memory; each stage is a Stockham autosort
// radix-R step (R in {2, 3, 4, 8}) whose R inputs and outputs are held in registers, so a
// stage costs one shared-memory read and one write per element and the result ends in
// natural order.  Twiddles come from one table tw[k] = exp(-2 pi i k / N) computed in FP64
// (sincospi) and rounded to the working precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ns {

template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return mk(s * a.x, s * a.y); }
template <typename T>
__device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk(a.x, -a.y); }
// Complex product in one fixed rounding order (the a.y products rounded, then one fused
// multiply-add per part), the same bits wherever it is compiled: used where two kernels must
// form the same value (the shifted fields carried from a step's last pass and the same fields
// formed again from the state).
__device__ __forceinline__ cpx<float> cmul_fixed(cpx<float> a, cpx<float> b) {
  return mk<float>(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ cpx<double> cmul_fixed(cpx<double> a, cpx<double> b) {
  return mk<double>(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
}
// multiply by s*i (s = +1 or -1)
template <typename T>
__device__ __forceinline__ cpx<T> mul_si(cpx<T> a, T s) { return mk(-s * a.y, s * a.x); }
// a * conj(b)
template <typename T>
__device__ __forceinline__ cpx<T> mul_conj(cpx<T> a, cpx<T> b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Packed single-precision pairs: on sm_100 and later one instruction adds (or fuses a
// multiply-add into) both halves of a complex value, each half rounded exactly as the scalar
// operation.  The FP32 butterflies below use them for their pure additions (NS_PACKED_F32=0
// keeps the scalar forms).
#ifndef NS_PACKED_F32
#define NS_PACKED_F32 1
#endif
__device__ __forceinline__ float2 as_f2(cpx<float> a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ cpx<float> as_c(float2 a) { return mk<float>(a.x, a.y); }
__device__ __forceinline__ cpx<float> padd(cpx<float> a, cpx<float> b) {
  return as_c(__fadd2_rn(as_f2(a), as_f2(b)));
}
// a - b as fma(b, -1, a): one rounding, the same value as the subtraction
__device__ __forceinline__ cpx<float> psub(cpx<float> a, cpx<float> b) {
  return as_c(__ffma2_rn(as_f2(b), make_float2(-1.f, -1.f), as_f2(a)));
}
// r b, r real
__device__ __forceinline__ cpx<float> pmul(float r, cpx<float> b) {
  return as_c(__fmul2_rn(make_float2(r, r), as_f2(b)));
}
// a w as two packed operations: a.x (w.x, w.y) + a.y (-w.y, w.x) (NS_PACKED_CMUL)
#ifndef NS_PACKED_CMUL
#define NS_PACKED_CMUL 0
#endif
__device__ __forceinline__ cpx<float> pcmul(cpx<float> a, cpx<float> w) {
  return as_c(__ffma2_rn(make_float2(a.y, a.y), make_float2(-w.y, w.x),
                         __fmul2_rn(make_float2(a.x, a.x), as_f2(w))));
}
template <typename T>
__device__ __forceinline__ cpx<T> tw_mul(cpx<T> a, cpx<T> w) { return a * w; }
#if NS_PACKED_CMUL
template <>
__device__ __forceinline__ cpx<float> tw_mul<float>(cpx<float> a, cpx<float> w) { return pcmul(a, w); }
#endif
// a + r b, r real (one rounding per half)
__device__ __forceinline__ cpx<float> pfma(float r, cpx<float> b, cpx<float> a) {
  return as_c(__ffma2_rn(make_float2(r, r), as_f2(b), as_f2(a)));
}

// read-only cached load of a complex value
__device__ __forceinline__ cpx<float> ldg(const cpx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cpx<double> ldg(const cpx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mk<double>(v.x, v.y);
}

// Radix plan of a length-n transform: n = prod radix[s].
struct FFTPlan {
  int n;          // transform length
  int nst;        // number of stages
  int tw_stride;  // (table length N) / n
  int radix[16];
};

// ----------------------------------------------------------------------------------------
// Small DFTs in registers.  s = -1: forward (exp(-2 pi i ...)), s = +1: inverse.
// ----------------------------------------------------------------------------------------
template <typename T, int R>
struct DFT;

template <typename T>
struct DFT<T, 2> {
  static __device__ __forceinline__ void run(cpx<T>* v, T) {
    cpx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

template <typename T>
struct DFT<T, 3> {
  // y_m = sum_t v_t w^{mt}, w = exp(s 2 pi i / 3) = -1/2 + s i sqrt(3)/2
  static __device__ __forceinline__ void run(cpx<T>* v, T s) {
    const T h = T(0.86602540378443864676);  // sqrt(3)/2
    cpx<T> a = v[0], b = v[1], c = v[2];
    cpx<T> bp = b + c, bm = b - c;
    cpx<T> m = a - T(0.5) * bp;
    cpx<T> r = mul_si(h * bm, s);
    v[0] = a + bp;
    v[1] = m + r;
    v[2] = m - r;
  }
};

template <typename T>
struct DFT<T, 4> {
  static __device__ __forceinline__ void run(cpx<T>* v, T s) {
    cpx<T> a = v[0], b = v[1], c = v[2], d = v[3];
    cpx<T> p0 = a + c, p1 = a - c, q0 = b + d, q1 = mul_si(b - d, s);
    v[0] = p0 + q0;
    v[2] = p0 - q0;
    v[1] = p1 + q1;
    v[3] = p1 - q1;
  }
};

template <typename T>
struct DFT<T, 8> {
  // split into even / odd 4-point DFTs and combine with w8^k, w8 = exp(s 2 pi i / 8)
  static __device__ __forceinline__ void run(cpx<T>* v, T s) {
    const T r2 = T(0.70710678118654752440);  // 1/sqrt(2)
    cpx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cpx<T> o[4] = {v[1], v[3], v[5], v[7]};
    DFT<T, 4>::run(e, s);
    DFT<T, 4>::run(o, s);
    // w8^1 = (1 + s i)/sqrt2, w8^2 = s i, w8^3 = (-1 + s i)/sqrt2
    cpx<T> o1 = r2 * (o[1] + mul_si(o[1], s));
    cpx<T> o2 = mul_si(o[2], s);
    cpx<T> o3 = r2 * (mul_si(o[3], s) - o[3]);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
  }
};

#if NS_PACKED_F32
// FP32 forms of the 2-, 4- and 8-point DFTs above with the additions packed; the products by
// s i stay scalar (a swap of the halves, folded into the additions that use them).
template <>
struct DFT<float, 2> {
  static __device__ __forceinline__ void run(cpx<float>* v, float) {
    const cpx<float> a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
  }
};

template <>
struct DFT<float, 4> {
  static __device__ __forceinline__ void run(cpx<float>* v, float s) {
    const cpx<float> a = v[0], b = v[1], c = v[2], d = v[3];
    const cpx<float> p0 = padd(a, c), p1 = psub(a, c), q0 = padd(b, d), t = psub(b, d);
    v[0] = padd(p0, q0);
    v[2] = psub(p0, q0);
    v[1] = mk<float>(p1.x - s * t.y, p1.y + s * t.x);  // p1 + s i t
    v[3] = mk<float>(p1.x + s * t.y, p1.y - s * t.x);  // p1 - s i t
  }
};

template <>
struct DFT<float, 8> {
  static __device__ __forceinline__ void run(cpx<float>* v, float s) {
    const float r2 = 0.70710678118654752440f;
    cpx<float> e[4] = {v[0], v[2], v[4], v[6]};
    cpx<float> o[4] = {v[1], v[3], v[5], v[7]};
    DFT<float, 4>::run(e, s);
    DFT<float, 4>::run(o, s);
    // w8^1 o1 = r2 (o1 + s i o1), w8^3 o3 = r2 (s i o3 - o3), w8^2 o2 = s i o2
    const cpx<float> t1 = mk<float>(o[1].x - s * o[1].y, o[1].y + s * o[1].x);
    const cpx<float> t3 = mk<float>(-s * o[3].y - o[3].x, s * o[3].x - o[3].y);
    v[0] = padd(e[0], o[0]);
    v[4] = psub(e[0], o[0]);
    v[1] = pfma(r2, t1, e[1]);
    v[5] = pfma(-r2, t1, e[1]);
    v[3] = pfma(r2, t3, e[3]);
    v[7] = pfma(-r2, t3, e[3]);
    v[2] = mk<float>(e[2].x - s * o[2].y, e[2].y + s * o[2].x);
    v[6] = mk<float>(e[2].x + s * o[2].y, e[2].y - s * o[2].x);
  }
};
#endif

// Butterflies held per thread per stage (R * KB <= 16 values in registers).
template <int R>
struct StageKB {
  static constexpr int value = (R == 2) ? 8 : (R == 3) ? 5 : (R == 4) ? 4 : 2;
};

// One Stockham radix-R stage over a batch of nl lines of length n in shared memory.
// Element e of line l is buf[l * ls + e * es].  line_fast: consecutive threads take
// consecutive lines (use when es > 1) rather than consecutive butterflies of one line.
// Requires nl * n / R <= StageKB<R> * blockDim.x (checked; *err set otherwise).
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(cpx<T>* buf, int n, int nl, int es, int ls,
                                               bool line_fast, int Ns,
                                               const cpx<T>* __restrict__ tw, int tw_stride,
                                               T s, int* err) {
  constexpr int KB = StageKB<R>::value;
  const int nb = n / R;
  const int total = nb * nl;
  if (total > KB * (int)blockDim.x) {
    if (threadIdx.x == 0 && err) atomicOr(err, 1);
    return;
  }
  cpx<T> v[KB][R];
  const int tstep = (n / (Ns * R)) * tw_stride;
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    const int b = threadIdx.x + c * blockDim.x;
    if (b < total) {
      int line, j;
      if (line_fast) {
        line = b % nl;
        j = b / nl;
      } else {
        j = b % nb;
        line = b / nb;
      }
      const cpx<T>* src = buf + line * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) v[c][r] = src[(j + r * nb) * es];
      if (Ns > 1) {
        const int p = j % Ns;
        const int base = p * tstep;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cpx<T> w = ldg(&tw[r * base]);
          w.y *= -s;  // table holds exp(-..); s = +1 (inverse) needs the conjugate
          v[c][r] = v[c][r] * w;
        }
      }
      DFT<T, R>::run(v[c], s);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    const int b = threadIdx.x + c * blockDim.x;
    if (b < total) {
      int line, j;
      if (line_fast) {
        line = b % nl;
        j = b / nl;
      } else {
        j = b % nb;
        line = b / nb;
      }
      const int p = j % Ns, q = j / Ns;
      cpx<T>* dst = buf + line * ls;
      const int o = q * Ns * R + p;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[(o + r * Ns) * es] = v[c][r];
    }
  }
  __syncthreads();
}

// Full transform of a batch of lines (forward if s = -1, inverse if s = +1).
template <typename T>
__device__ __forceinline__ void fft_lines(cpx<T>* buf, const FFTPlan& pl, int nl, int es, int ls,
                                          bool line_fast, const cpx<T>* __restrict__ tw, T s,
                                          int* err) {
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.radix[st];
    switch (R) {
      case 2:
        stockham_stage<T, 2>(buf, pl.n, nl, es, ls, line_fast, Ns, tw, pl.tw_stride, s, err);
        break;
      case 3:
        stockham_stage<T, 3>(buf, pl.n, nl, es, ls, line_fast, Ns, tw, pl.tw_stride, s, err);
        break;
      case 4:
        stockham_stage<T, 4>(buf, pl.n, nl, es, ls, line_fast, Ns, tw, pl.tw_stride, s, err);
        break;
      default:
        stockham_stage<T, 8>(buf, pl.n, nl, es, ls, line_fast, Ns, tw, pl.tw_stride, s, err);
        break;
    }
    Ns *= R;
  }
}

}  // namespace ns
