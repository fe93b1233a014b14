// ns_fft2.cuh -- compile-time mixed-radix FFT for the grid sizes the library specialises.
//
// Same transform as ns_fft.cuh (supplementary Eq. dft_def per direction, unnormalised), but
// the length, the radix plan (16, 16, ..., then 8/4/2, then 3s), the batch width and the
// thread count are template parameters, so every index is resolved at compile time.  A
// length-n transform of NL lines is a chain of Stockham stages:
//   stage 0        reads its inputs through an accessor (global memory or shared memory,
//                  with any pointwise factor applied on the fly) and writes a shared work tile;
//   middle stages  work tile -> work tile in place (all reads before a barrier, then writes);
//   last stage     reads the work tile and writes through an output accessor (global rows,
//                  or a shared tile).
// For n = 16^2 = 256 that is the four-step algorithm with a single shared-memory transpose.
#pragma once

#include "ns_fft.cuh"

namespace ns {

struct CPlan {
  int nst;
  int r[8];
};

// Largest radix of the register butterflies (16 or 8).  8 halves the values a thread holds
// and doubles the threads that share a tile (more warps to hide latency), at the cost of one
// more shared-memory pass for n = 256; every kernel can pick its own cap (template MR).
#ifndef NS_MAX_RADIX
#define NS_MAX_RADIX 8
#endif

__host__ __device__ constexpr CPlan cplan(int n, int mr = NS_MAX_RADIX) {
  CPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}};
  int m = n, a2 = 0, a3 = 0;
  while (m % 2 == 0) { m /= 2; ++a2; }
  while (m % 3 == 0) { m /= 3; ++a3; }
  if (mr >= 16)
    while (a2 >= 4) { p.r[p.nst++] = 16; a2 -= 4; }
  while (a2 >= 3) { p.r[p.nst++] = 8; a2 -= 3; }
  if (a2 == 2) p.r[p.nst++] = 4;
  else if (a2 == 1) p.r[p.nst++] = 2;
  for (int i = 0; i < a3; ++i) p.r[p.nst++] = 3;
  return p;
}

// 16-point DFT as 4 x 4 (n = n1 + 4 n2, k = 4 k1 + k2), internal twiddles W16^(n1 k2)
template <typename T>
struct DFT<T, 16> {
  static __device__ __forceinline__ void run(cpx<T>* v, T s) {
    const T c8 = T(0.92387953251128675613), s8 = T(0.38268343236508977173);
    const T r2 = T(0.70710678118654752440);
    cpx<T> a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      cpx<T> q[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
      DFT<T, 4>::run(q, s);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[n1][k2] = q[k2];
    }
    // twiddles W16^m = cos(2 pi m/16) + s i sin(2 pi m/16)
    a[1][1] = a[1][1] * mk<T>(c8, s * s8);
    a[1][2] = a[1][2] * mk<T>(r2, s * r2);
    a[1][3] = a[1][3] * mk<T>(s8, s * c8);
    a[2][1] = a[2][1] * mk<T>(r2, s * r2);
    a[2][2] = mul_si(a[2][2], s);
    a[2][3] = a[2][3] * mk<T>(-r2, s * r2);
    a[3][1] = a[3][1] * mk<T>(s8, s * c8);
    a[3][2] = a[3][2] * mk<T>(-r2, s * r2);
    a[3][3] = a[3][3] * mk<T>(-c8, -s * s8);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      cpx<T> q[4] = {a[0][k2], a[1][k2], a[2][k2], a[3][k2]};
      DFT<T, 4>::run(q, s);
#pragma unroll
      for (int k1 = 0; k1 < 4; ++k1) v[4 * k1 + k2] = q[k1];
    }
  }
};

#if NS_PACKED_F32
// FP32 form with packed additions (the 4-point DFTs above); the s i twiddle of a[2][2] is
// folded into the additions of its column
template <>
struct DFT<float, 16> {
  static __device__ __forceinline__ void run(cpx<float>* v, float s) {
    const float c8 = 0.92387953251128675613f, s8 = 0.38268343236508977173f;
    const float r2 = 0.70710678118654752440f;
    cpx<float> a[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
      cpx<float> q[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
      DFT<float, 4>::run(q, s);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) a[n1][k2] = q[k2];
    }
    a[1][1] = a[1][1] * mk<float>(c8, s * s8);
    a[1][2] = pmul(r2, mk<float>(a[1][2].x - s * a[1][2].y, a[1][2].y + s * a[1][2].x));
    a[1][3] = a[1][3] * mk<float>(s8, s * c8);
    a[2][1] = pmul(r2, mk<float>(a[2][1].x - s * a[2][1].y, a[2][1].y + s * a[2][1].x));
    a[2][3] = pmul(r2, mk<float>(-a[2][3].x - s * a[2][3].y, s * a[2][3].x - a[2][3].y));
    a[3][1] = a[3][1] * mk<float>(s8, s * c8);
    a[3][2] = pmul(r2, mk<float>(-a[3][2].x - s * a[3][2].y, s * a[3][2].x - a[3][2].y));
    a[3][3] = a[3][3] * mk<float>(-c8, -s * s8);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      const cpx<float> x0 = a[0][k2], x1 = a[1][k2], x3 = a[3][k2];
      cpx<float> p0, p1;
      if (k2 == 2) {  // x2 = s i a[2][2]
        const cpx<float> y = a[2][2];
        p0 = mk<float>(x0.x - s * y.y, x0.y + s * y.x);
        p1 = mk<float>(x0.x + s * y.y, x0.y - s * y.x);
      } else {
        p0 = padd(x0, a[2][k2]);
        p1 = psub(x0, a[2][k2]);
      }
      const cpx<float> q0 = padd(x1, x3), t = psub(x1, x3);
      v[k2] = padd(p0, q0);
      v[8 + k2] = psub(p0, q0);
      v[4 + k2] = mk<float>(p1.x - s * t.y, p1.y + s * t.x);
      v[12 + k2] = mk<float>(p1.x + s * t.y, p1.y - s * t.x);
    }
  }
};
#endif

// Line-fast tiles [e][line] of W lines.  When a row is narrower than the 32 banks of shared
// memory, rows 8 apart share banks (the radix-8 first stage writes rows 8 j + r); NS_LF_PAD=1
// inserts one empty row after every 8 (element row e at row lf_row(e) of lf_rows(n)).  Off by
// default: on GB300 at 256^3 the index arithmetic cost more than the conflicts it removed.
#ifndef NS_LF_PAD
#define NS_LF_PAD 0
#endif
template <typename T, int W>
__host__ __device__ constexpr bool lf_padded() { return NS_LF_PAD && W * (int)sizeof(cpx<T>) < 128; }
template <typename T, int W>
__host__ __device__ constexpr int lf_rows(int n) { return lf_padded<T, W>() ? n + (n - 1) / 8 : n; }
template <typename T, int W>
__host__ __device__ __forceinline__ int lf_row(int e) { return lf_padded<T, W>() ? e + (e >> 3) : e; }
template <typename T, int W>
__host__ __device__ __forceinline__ int lf_idx(int e, int line) { return lf_row<T, W>(e) * W + line; }

#ifndef NS_NLF_STRIDE_OLD
#define NS_NLF_STRIDE_OLD 0
#endif
// Shared work tile of NL lines of length n.  LF (line-fast) layout [e][line] as above;
// otherwise [line][e] with one pad element per 16 to spread the stride-R writes of a stage.
template <typename T, int n, int NL, bool LF>
struct WorkTile {
  cpx<T>* p;
  // line stride: one pad element per 16 spreads the stride-R writes within a line; choosing
  // LS = n/16 (mod 16) makes the lines a warp covers in a radix-16 first stage (32 / (n/16)
  // lines of n/16 consecutive elements) tile the 32 banks evenly
  static constexpr int LS = NS_NLF_STRIDE_OLD ? n + n / 16 + 1 : n + n / 16 + (16 - n % 16) % 16;
  static __host__ __device__ constexpr int elems() { return LF ? lf_rows<T, NL>(n) * NL : NL * LS; }
  __device__ __forceinline__ int idx(int line, int e) const {
    return LF ? lf_idx<T, NL>(e, line) : line * LS + e + (e >> 4);
  }
  __device__ __forceinline__ cpx<T> get(int line, int e) const { return p[idx(line, e)]; }
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const { p[idx(line, e)] = v; }
};

// Twiddles w[r] = W^(r base) (conjugated when cs = -1), r = 1 .. R-1, of one butterfly.  Only
// the powers r = 1, 2, 4, 8 are read from the (shared-memory) table; the others are their
// products, which moves work from the shared-memory pipe to the FMA pipe.
#ifndef NS_TW_PRODUCTS
#define NS_TW_PRODUCTS 1
#endif
// Shared-memory twiddle tables hold entry i at tw_pad(i): one pad per 16 entries, so the
// strided reads r * base of a stage's butterflies fall in distinct banks.
#ifndef NS_TW_PAD
#define NS_TW_PAD 1
#endif
__host__ __device__ constexpr int tw_pad(int i) { return NS_TW_PAD ? i + (i >> 4) : i; }
__host__ __device__ constexpr int tw_elems(int n) { return NS_TW_PAD ? n + n / 16 + 1 : n; }
template <typename T, int R>
__device__ __forceinline__ void stage_twiddles(cpx<T>* w, const cpx<T>* __restrict__ tw, int base, T cs) {
  auto ld = [&](int r) {
    cpx<T> v = tw[tw_pad(r * base)];
    v.y *= cs;
    return v;
  };
  if constexpr (R == 2) {
    w[1] = ld(1);
  } else if constexpr (R == 3) {
    w[1] = ld(1);
    w[2] = ld(2);
  } else if constexpr (R == 4) {
    w[1] = ld(1);
    w[2] = ld(2);
    w[3] = tw_mul(w[1], w[2]);
  } else if constexpr ((R == 8 || R == 16) && NS_TW_PRODUCTS) {
    w[1] = ld(1);
    w[2] = ld(2);
    w[4] = ld(4);
    w[3] = tw_mul(w[1], w[2]);
    w[5] = tw_mul(w[1], w[4]);
    w[6] = tw_mul(w[2], w[4]);
    w[7] = tw_mul(w[3], w[4]);
    if constexpr (R == 16) {
      w[8] = ld(8);
#pragma unroll
      for (int r = 9; r < 16; ++r) w[r] = tw_mul(w[r - 8], w[8]);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = ld(r);
  }
}

// One Stockham stage: butterfly j of a line reads elements j + r n/R, applies the
// twiddles W_{NS R}^{p r} (p = j mod NS), a radix-R DFT, and writes q NS R + p + r NS.
// HOLD: every input is read (and a barrier passed) before any output is written.
// Threads with threadIdx.x >= NT take no butterflies but pass the barriers.
// tid: the thread's index in the block (threadIdx.x; a caller may pass a value the compiler
// cannot prove loop-invariant, to keep the stage's index arithmetic out of its registers
// across unrelated code).
template <typename T, int n, int R, int NS, int TWS, int NL, int NT, bool LF, int DIR, bool HOLD,
          class Src, class Dst>
__device__ __forceinline__ void cstage(const Src& src, const Dst& dst, const cpx<T>* __restrict__ tw,
                                       int tid = threadIdx.x) {
  constexpr int NB = n / R;
  constexpr int TOT = NB * NL;
  constexpr int KB = (TOT + NT - 1) / NT;
  constexpr int TSTEP = (n / (NS * R)) * TWS;
  const T s = T(DIR);
  auto map = [](int b, int& line, int& j) {
    if (LF) {
      line = b % NL;
      j = b / NL;
    } else {
      j = b % NB;
      line = b / NB;
    }
  };
  auto compute = [&](cpx<T>* v, int line, int j) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src.get(line, j + r * NB);
    if (NS > 1) {
      const int base = (j % NS) * TSTEP;
      cpx<T> w[R];
      stage_twiddles<T, R>(w, tw, base, -s);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = tw_mul(v[r], w[r]);
    }
    DFT<T, R>::run(v, s);
  };
  auto emit = [&](const cpx<T>* v, int line, int j) {
    const int p = j % NS, q = j / NS;
    const int o = q * NS * R + p;
#pragma unroll
    for (int r = 0; r < R; ++r) dst.put(line, o + r * NS, v[r]);
  };
  if (HOLD) {
    cpx<T> v[KB][R];
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      const int b = tid + c * NT;
      if (tid < NT && (TOT % NT == 0 || b < TOT)) {
        int line, j;
        map(b, line, j);
        compute(v[c], line, j);
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      const int b = tid + c * NT;
      if (tid < NT && (TOT % NT == 0 || b < TOT)) {
        int line, j;
        map(b, line, j);
        emit(v[c], line, j);
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      const int b = tid + c * NT;
      if (tid < NT && (TOT % NT == 0 || b < TOT)) {
        int line, j;
        map(b, line, j);
        cpx<T> v[R];
        compute(v, line, j);
        emit(v, line, j);
      }
    }
  }
}

template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, int S, int NS,
          bool HOLD0 = false, int MR = NS_MAX_RADIX>
struct CStages {
  static constexpr CPlan P = cplan(n, MR);
  template <class Src, class Dst>
  static __device__ __forceinline__ void run(const Src& src, const Dst& dst, cpx<T>* work,
                                             const cpx<T>* __restrict__ tw) {
    constexpr int R = P.r[S];
    constexpr bool first = S == 0;
    constexpr bool last = S == P.nst - 1;
    const WorkTile<T, n, NL, LF> W{work};
    if constexpr (first && last) {
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, true>(src, dst, tw);
    } else if constexpr (first) {
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, HOLD0>(src, W, tw);
      __syncthreads();
      CStages<T, n, TWS, NL, NT, LF, DIR, S + 1, NS * R, false, MR>::run(src, dst, work, tw);
    } else if constexpr (last) {
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, false>(W, dst, tw);
    } else {
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, true>(W, W, tw);
      __syncthreads();
      CStages<T, n, TWS, NL, NT, LF, DIR, S + 1, NS * R, false, MR>::run(src, dst, work, tw);
    }
  }
};

// Transform of NL lines of length n: src -> dst through the shared work tile `work`
// (WorkTile<T, n, NL, LF>::elems() values).  DIR = -1 forward, +1 inverse.  TWS = table
// length / n.  The caller places a barrier after it before dst is read by other threads.
template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, int MR = NS_MAX_RADIX,
          class Src, class Dst>
__device__ __forceinline__ void cfft(const Src& src, const Dst& dst, cpx<T>* work,
                                     const cpx<T>* __restrict__ tw) {
  CStages<T, n, TWS, NL, NT, LF, DIR, 0, 1, false, MR>::run(src, dst, work, tw);
}

// Same, for a source that reads the work tile itself: stage 0 reads every input before it
// writes the work tile.
template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, int MR = NS_MAX_RADIX,
          class Src, class Dst>
__device__ __forceinline__ void cfft_src_in_work(const Src& src, const Dst& dst, cpx<T>* work,
                                                 const cpx<T>* __restrict__ tw) {
  CStages<T, n, TWS, NL, NT, LF, DIR, 0, 1, true, MR>::run(src, dst, work, tw);
}

// In place: stage 0 reads src (ALIAS: src is the tile itself) and writes the tile B; every
// later stage runs in place on B with its inputs held in registers across a barrier.  The
// last stage writes through dst (an accessor over the same tile, e.g. applying a pointwise
// factor); the result is left in natural order.  No separate work tile is needed.
template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, bool ALIAS, int S, int NS,
          int MR = NS_MAX_RADIX>
struct CStagesIP {
  static constexpr CPlan P = cplan(n, MR);
  template <class Src, class Tile, class Dst>
  static __device__ __forceinline__ void run(const Src& src, const Tile& B, const Dst& dst,
                                             const cpx<T>* __restrict__ tw, int tid = threadIdx.x) {
    constexpr int R = P.r[S];
    constexpr bool last = S + 1 == P.nst;
    if constexpr (S == 0 && last)
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, ALIAS>(src, dst, tw, tid);
    else if constexpr (S == 0)
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, ALIAS>(src, B, tw, tid);
    else if constexpr (last)
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, true>(B, dst, tw, tid);
    else
      cstage<T, n, R, NS, TWS, NL, NT, LF, DIR, true>(B, B, tw, tid);
    if constexpr (!last) {
      __syncthreads();
      CStagesIP<T, n, TWS, NL, NT, LF, DIR, ALIAS, S + 1, NS * R, MR>::run(src, B, dst, tw, tid);
    }
  }
};

template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, bool ALIAS,
          int MR = NS_MAX_RADIX, class Src>
__device__ __forceinline__ void cfft_ip(const Src& src, cpx<T>* tile, const cpx<T>* __restrict__ tw) {
  const WorkTile<T, n, NL, LF> B{tile};
  CStagesIP<T, n, TWS, NL, NT, LF, DIR, ALIAS, 0, 1, MR>::run(src, B, B, tw);
}

// Same, the last stage writing through dst (which must address the same tile)
template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, bool ALIAS,
          int MR = NS_MAX_RADIX, class Src, class Dst>
__device__ __forceinline__ void cfft_ip_to(const Src& src, cpx<T>* tile, const Dst& dst,
                                           const cpx<T>* __restrict__ tw) {
  CStagesIP<T, n, TWS, NL, NT, LF, DIR, ALIAS, 0, 1, MR>::run(src, WorkTile<T, n, NL, LF>{tile}, dst, tw);
}

// In-place transform of NL lines over any tile accessor B (get / put of (line, e)); the last
// stage writes through dst.  tid as in cstage.
template <typename T, int n, int TWS, int NL, int NT, bool LF, int DIR, bool ALIAS,
          int MR = NS_MAX_RADIX, class Src, class Tile, class Dst>
__device__ __forceinline__ void cfft_ip_tid(const Src& src, const Tile& B, const Dst& dst,
                                            const cpx<T>* __restrict__ tw, int tid) {
  CStagesIP<T, n, TWS, NL, NT, LF, DIR, ALIAS, 0, 1, MR>::run(src, B, dst, tw, tid);
}

// copy of the twiddle table into shared memory (all threads of the block participate)
template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* dst, const cpx<T>* __restrict__ tw, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[tw_pad(i)] = ldg(&tw[i]);
  __syncthreads();
}

}  // namespace ns
