// ns_kernels2.cuh -- the hot kernels specialised on the grid size N (compile-time FFTs).
//
// Same passes, layouts and arithmetic as the generic kernels of ns_kernels.cuh (see there
// for the data layout): k2_pencil = z transforms + spectral stage of Sec. 4 / 6.1,
// k2_yinv / k2_xrow / k2_yfwd = slab pass (y transforms, x rows with u x omega), and
// k2_slabpipe = the slab pass as one persistent pipelined launch.  What changes is how the
// transforms run: tiles are staged with cp.async, the first FFT stage reads the staged tile
// or global memory and the last one writes global memory or applies the spectral factors,
// every index is a compile-time expression, and the butterflies are radix 8 or 16 in
// registers (per kernel, K2Cfg).
#pragma once

#include "ns_fft2.cuh"
#include "ns_kernels.cuh"

namespace ns {

__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int pick_div(int m, int target, int cap) {
  int t = cmin(cmax(target, 1), cap);
  for (int d = t; d >= 1; --d)
    if (m % d == 0) return d;
  return 1;
}
__host__ __device__ constexpr int round_warps(int t) { return cmin(cmax((t + 31) / 32 * 32, 64), 512); }
__host__ __device__ constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }
// thread count: >= t, >= 64, a multiple of the warp size and of w (each thread keeps one line)
__host__ __device__ constexpr int round_lines(int t, int w) {
  const int l = 32 / cgcd(32, w) * w;
  const int v = cmax(t, 64);
  return (v + l - 1) / l * l;
}

// Global-memory access policy.  MemNC: data written by earlier launches (read-only path).
// MemCG: data written by other blocks of the same launch (persistent kernel): loads and
// stores go to L2 (.cg) so a block never sees a stale line in its own L1.
struct MemNC {
  template <typename T>
  static __device__ __forceinline__ cpx<T> ld(const cpx<T>* p) { return ldg(p); }
  template <typename T>
  static __device__ __forceinline__ cpx<T> ldw(const cpx<T>* p) { return *p; }
  template <typename T>
  static __device__ __forceinline__ void st(cpx<T>* p, cpx<T> v) { *p = v; }
  // two consecutive FP32 modes (16-byte aligned)
  static __device__ __forceinline__ float4 ld2(const cpx<float>* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ void st2(cpx<float>* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
};
struct MemCG {
  static __device__ __forceinline__ float4 ld2(const cpx<float>* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
  static __device__ __forceinline__ void st2(cpx<float>* p, float4 v) { __stcg(reinterpret_cast<float4*>(p), v); }
  static __device__ __forceinline__ cpx<float> ld(const cpx<float>* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk<float>(v.x, v.y);
  }
  static __device__ __forceinline__ cpx<double> ld(const cpx<double>* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk<double>(v.x, v.y);
  }
  template <typename T>
  static __device__ __forceinline__ cpx<T> ldw(const cpx<T>* p) { return ld(p); }
  static __device__ __forceinline__ void st(cpx<float>* p, cpx<float> v) {
    __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
  }
  static __device__ __forceinline__ void st(cpx<double>* p, cpx<double> v) {
    __stcg(reinterpret_cast<double2*>(p), make_double2(v.x, v.y));
  }
};

// Asynchronous 16-byte global -> shared copies (cp.async.cg: through L2 only, so data written
// by other blocks of a persistent launch is never read from a stale L1 line).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most P of this thread's committed groups are still in flight
template <int P>
__device__ __forceinline__ void cp_async_wait_pending() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(P) : "memory");
}
// Stage a column tile [e][line] (W lines, n elements) of a [z|kz][ky][kx] field from global
// memory; W * sizeof(cpx<T>) is a multiple of 16 bytes and x0 a multiple of W.
// PLANE: the tile of a fixed plane p of a [p][e][kx] field (element e = ky or y) instead.
template <typename T, int N, int W, int NT, bool PLANE = false>
__device__ __forceinline__ void stage_col_tile(cpx<T>* dst, const cpx<T>* src, int iy, int x0) {
  constexpr int PER = 16 / (int)sizeof(cpx<T>);  // complex values per 16-byte chunk
  constexpr int CH = W / PER;                     // chunks per row
  static_assert(W % PER == 0, "tile rows must be whole 16-byte chunks");
  if (threadIdx.x >= NT) return;
  for (int i = threadIdx.x; i < N * CH; i += NT) {
    const int e = i / CH, xc = (i % CH) * PER;
    const size_t row = PLANE ? (size_t)iy * N + e : (size_t)e * N + iy;
    cp_async16(&dst[lf_idx<T, W>(e, xc)], &src[row * (N / 2) + x0 + xc]);
  }
}

// Radix cap of each kernel's transforms (pencil z, inverse y, forward y, x rows); 0 = the
// measured default: in FP32 radix 16 for both y passes and the x rows (one shared-memory pass
// fewer; the inverse y, bound by shared memory, 0.268 against 0.287 ms per step at 256^3 with
// radix 8), radix 8 for the pencil (more threads per tile); 8 in FP64.
#ifndef NS_RADIX_Z
#define NS_RADIX_Z 0
#endif
#ifndef NS_RADIX_YI
#define NS_RADIX_YI 0
#endif
#ifndef NS_RADIX_YF
#define NS_RADIX_YF 0
#endif
#ifndef NS_RADIX_X
#define NS_RADIX_X 0
#endif
__host__ __device__ constexpr int radix_cap(int set, int f32_default, bool f32) {
  return set > 0 ? set : (f32 ? f32_default : NS_MAX_RADIX);
}
// NS_SLAB_RADIX_RULE=1: the FP32 slab passes of N <= 128 take radix 8 where the radix-16 plan
// keeps a radix-2 stage that the radix-8 plan avoids (N = 32: 16.2 -> 8.4; N = 96: 16.2.3 ->
// 8.4.3).  Measured on GB300: 96^3 step 0.110 against 0.123 ms, 32^3 0.058 against 0.060, the
// 64-member ensemble +4 %; at 512 (16.16.2 -> 8.8.8) it was 14 % slower, so larger N keep 16.
#ifndef NS_SLAB_RADIX_RULE
#define NS_SLAB_RADIX_RULE 1
#endif
__host__ __device__ constexpr bool plan_has_radix2(int n, int mr) {
  const CPlan p = cplan(n, mr);
  for (int i = 0; i < p.nst; ++i)
    if (p.r[i] == 2) return true;
  return false;
}
__host__ __device__ constexpr int slab_radix(int n) {
  return NS_SLAB_RADIX_RULE && n <= 128 && plan_has_radix2(n, 16) && !plan_has_radix2(n, 8) ? 8 : 16;
}

// Unroll factor of the pencil's loops over the transforms of the components: 1 keeps one copy
// of the transform code per loop (measured 6 % faster than full unrolling at 256^3 FP32: the
// pencil is sensitive to instruction-cache misses)
#ifndef NS_PENCIL_UNROLL
#define NS_PENCIL_UNROLL 1
#endif
constexpr int kPencilUnroll = NS_PENCIL_UNROLL;
// modes per thread whose state loads the fused spectral pass keeps in flight together
#ifndef NS_PENCIL_CHK
#define NS_PENCIL_CHK 4
#endif  // (pragma arguments are not macro-expanded)
// NS_PENCIL_STAGE_STATE=1: the one-input pencil also stages the 3 state tiles with cp.async at
// the start of a tile (6 tiles of shared memory, 2 blocks per SM instead of 3)
#ifndef NS_PENCIL_STAGE_STATE
#define NS_PENCIL_STAGE_STATE 0
#endif

// The alternative width of a tile (lines per tile): twice the default where that divides
// the half length m within the cap, else half (down to minw), else the default.
__host__ __device__ constexpr int alt_width(int w, int m, int cap, int minw) {
  return (m % (2 * w) == 0 && 2 * w <= cap) ? 2 * w : ((w / 2 >= minw && m % (w / 2) == 0) ? w / 2 : w);
}

// Tile shapes of size N.  V selects compiled alternatives for the autotuner, one bit per
// kernel family: bit 0 the pencil width TX, bit 1 the inverse-y width TYI, bit 2 the x-row
// count RX, bit 3 the forward-y width TY, bit 4 the pencil's register budget (64: one more
// resident block) (V = 0: the defaults).
template <typename T, int N, int V = 0>
struct K2Cfg {
  static constexpr int M = N / 2;
  static constexpr int CS = (int)sizeof(cpx<T>);
  static constexpr int MINW = 32 / CS;  // 32-byte global segments
  static constexpr bool F32 = sizeof(T) == 4;
  static constexpr int RZ = radix_cap(NS_RADIX_Z, NS_MAX_RADIX, F32);
  static constexpr int RYI = radix_cap(NS_RADIX_YI, slab_radix(N), F32);
  static constexpr int RYF = radix_cap(NS_RADIX_YF, slab_radix(N), F32);
  static constexpr int RXR = radix_cap(NS_RADIX_X, slab_radix(N), F32);
  // pencil: TX columns of N (NS_PZ_LINES / NS_YF_LINES override the pencil / forward-y width)
#ifndef NS_PZ_LINES
#define NS_PZ_LINES 0
#endif
#ifndef NS_YF_LINES
#define NS_YF_LINES 0
#endif
  static constexpr int TX0 = (NS_PZ_LINES > 0 && M % NS_PZ_LINES == 0 && NS_PZ_LINES % MINW == 0)
                                 ? NS_PZ_LINES
                                 : pick_div(M, cmax(16384 / (N * CS), MINW), 16);
  static constexpr int TX = (V & 1) ? alt_width(TX0, M, 16, MINW) : TX0;
  static constexpr int NTP = round_lines(TX * N / RZ, TX);
  // blocks per SM the register budget must allow (NS_PENCIL_REGS registers per thread;
  // 80 measured best at 256^3 FP32 on GB300 against 96 and 128)
#ifndef NS_PENCIL_REGS
#define NS_PENCIL_REGS 80
#endif
  // (variant bit 16: the pencil held to 64 registers, one more resident block)
  static constexpr int MINB_P = cmax(1, cmin(8, 65536 / (NTP * ((V & 16) ? 64 : NS_PENCIL_REGS))));
  // forward y pass: TY columns of N in a tile of about 32 KB (measured at 256^3 FP32: 16
  // columns, 0.133 ms per step against 0.141 for 8)
  static constexpr int TY0 = (NS_YF_LINES > 0 && M % NS_YF_LINES == 0 && NS_YF_LINES % MINW == 0)
                                 ? NS_YF_LINES
                                 : pick_div(M, cmax(32768 / (N * CS), MINW), 16);
  static constexpr int TY = (V & 8) ? alt_width(TY0, M, 32, MINW) : TY0;
  static constexpr int NTY = round_warps(TY * N / RYF);
  // inverse y pass: 4 shared tiles (3 input slots and a work tile); the width is the one
  // measured best when the tile held 6 (the 5 inputs and the work tile) within 110 KB
#ifndef NS_YI_LINES
#define NS_YI_LINES 0
#endif
  static constexpr int TYI0 = (NS_YI_LINES > 0 && M % NS_YI_LINES == 0 && NS_YI_LINES % MINW == 0)
                                  ? NS_YI_LINES
                                  : pick_div(M, cmax(110000 / (6 * N * CS), MINW), 16);
  static constexpr int TYI = (V & 2) ? alt_width(TYI0, M, 16, MINW) : TYI0;
  static constexpr int NTYI = round_warps(TYI * N / RYI);
  // x rows: RX rows of M, processed three fields at a time (NS_XR_ROWS overrides RX)
#ifndef NS_XR_ROWS
#define NS_XR_ROWS 0
#endif
  static constexpr int RX0 = NS_XR_ROWS > 0 ? NS_XR_ROWS : cmin(cmax(8192 / (M * CS), 1), 16);
  static constexpr int RX = (V & 4) ? (2 * RX0 <= 16 ? 2 * RX0 : cmax(RX0 / 2, 1)) : RX0;
  static constexpr int NTX = round_warps(3 * RX * M / RXR);
  // elements of the x-row tile: 3 RX complex lines of length N (two real rows per line), and
  // the blocks per SM its shared memory allows (the register budget is held to that many)
  static constexpr int XELEMS = WorkTile<T, N, 3 * RX, false>::elems();
  static constexpr int MINB_X = cmax(1, cmin(8, (227 * 1024) / ((XELEMS + tw_elems(N)) * CS + 1024)));
  static __host__ __device__ constexpr int pencil_tiles(int nF) { return nF > 1 ? 5 : 4; }
};

// ---- accessors ------------------------------------------------------------------------
template <typename T, int N, int W, class MP>
struct ColIn {  // global [z|kz][ky][kx] column tile (element e = z index), read-only
  const cpx<T>* p;
  int iy, x0;
  __device__ __forceinline__ cpx<T> get(int line, int e) const {
    return MP::ld(&p[((size_t)e * N + iy) * (N / 2) + x0 + line]);
  }
};
template <typename T, int N, int W, class MP>
struct ColOut {
  cpx<T>* p;
  int iy, x0;
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const {
    MP::st(&p[((size_t)e * N + iy) * (N / 2) + x0 + line], v);
  }
};
template <typename T, int W>
struct SmTile {  // shared [e][line]
  cpx<T>* p;
  __device__ __forceinline__ cpx<T> get(int line, int e) const { return p[lf_idx<T, W>(e, line)]; }
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const { p[lf_idx<T, W>(e, line)] = v; }
};
template <class MP, typename T>
__device__ __forceinline__ cpx<T> phase3p(const cpx<T>* tab, int N, int ix, int iy, int iz) {
  return cmul_fixed(cmul_fixed(MP::ld(&tab[ix]), MP::ld(&tab[N + iy])), MP::ld(&tab[2 * N + iz]));
}
// pencil output: shift, optional i kz factor, from a shared component tile
template <typename T, int N, int W, class MP>
struct PencilOutSrc {
  const cpx<T>* s;
  const cpx<T>* sh;
  int iy, x0;
  bool deriv;
  __device__ __forceinline__ cpx<T> get(int line, int e) const {
    cpx<T> v = s[lf_idx<T, W>(e, line)];
    if (sh) v = cmul_fixed(v, phase3p<MP>(sh, N, x0 + line, iy, e));
    if (deriv) v = mul_si(v, (T)kof(e, N));
    return v;
  }
};

// 1 / k^2 of the projection: FP32 uses the fast division intrinsic (within 2 ulp, far below
// the FP32 path's per-step error), FP64 the correctly rounded division.
template <typename T>
__device__ __forceinline__ T recip_k2(int k2);
template <>
__device__ __forceinline__ float recip_k2<float>(int k2) { return __fdividef(1.0f, (float)k2); }
template <>
__device__ __forceinline__ double recip_k2<double>(int k2) { return 1.0 / (double)k2; }

// ---- spectral stage at one mode (Sec. 4.1, 4.2, 6.1) ----------------------------------
// nv: de-shifted, weighted transform of u x omega at the mode: N(0) = 0, truncation T,
// Leray projection P, then the forcing term O (added on the modes of the forcing table).
template <typename T>
__device__ __forceinline__ void project_point(const PencilArgs<T>& a, int kx, int ky, int kz,
                                              cpx<T> nv[3]) {
  const int k2 = kx * kx + ky * ky + kz * kz;
  const bool keep = trunc_keep(a.trunc, kx, ky, kz, a.N, a.K2max, a.Kimax) && (k2 != 0);
  if (keep) {
    const cpx<T> v0 = nv[0], v1 = nv[1], v2 = nv[2];
    const T fx = (T)kx, fy = (T)ky, fz = (T)kz;
    const T ik2 = recip_k2<T>(k2);
    const cpx<T> kd = mk<T>(fx * v0.x + fy * v1.x + fz * v2.x, fx * v0.y + fy * v1.y + fz * v2.y);
    nv[0] = v0 - (fx * ik2) * kd;
    nv[1] = v1 - (fy * ik2) * kd;
    nv[2] = v2 - (fz * ik2) * kd;
  } else {
    nv[0] = nv[1] = nv[2] = mk<T>(0, 0);
  }
  if (a.force && kx <= a.fK && abs(ky) <= a.fK && abs(kz) <= a.fK) {
    const int D1 = 2 * a.fK + 1, D = D1 * D1 * (a.fK + 1);
    const int fi = ((kz + a.fK) * D1 + (ky + a.fK)) * (a.fK + 1) + kx;
#pragma unroll
    for (int c = 0; c < 3; ++c) nv[c] = nv[c] + a.force[c * D + fi];
  }
}

// RK stage combine of component c at one mode (modes of PencilMode).  s0: the value read
// from src (INIT), acc (RK4_4) or state (all other modes); s1: acc for RK4_2 / RK4_3.
// Performs the mode's global writes and returns S_next.
// mode: the pencil's stage (a.mode, or a compile-time constant in the specialised kernels)
template <typename T, class MP>
__device__ __forceinline__ cpx<T> stage_combine(const PencilArgs<T>& a, int c, size_t g, cpx<T> n,
                                                cpx<T> s0, cpx<T> s1, T E1, T Eh, int mode) {
  const T dt = a.dt, hdt = T(0.5) * a.dt;
  (void)c;
  switch (mode) {
    case MODE_INIT:
      return s0;
    case MODE_RK2_1:
      return Eh * (s0 + hdt * n);
    case MODE_RK2_2: {
      const cpx<T> s = E1 * s0 + (dt * Eh) * n;
      MP::st(&a.state[g], s);
      return s;
    }
    case MODE_RK4_1:
      MP::st(&a.acc[g], E1 * s0 + (dt / T(6) * E1) * n);
      return Eh * (s0 + hdt * n);
    case MODE_RK4_2:
      MP::st(&a.acc[g], s1 + (dt / T(3) * Eh) * n);
      return Eh * s0 + hdt * n;
    case MODE_RK4_3:
      MP::st(&a.acc[g], s1 + (dt / T(3) * Eh) * n);
      return E1 * s0 + (dt * Eh) * n;
    case MODE_RK4_4: {
      const cpx<T> s = s0 + (dt / T(6)) * n;
      MP::st(&a.state[g], s);
      return s;
    }
    case MODE_ROG_1:
      MP::st(&a.state[g], E1 * s0 + (hdt * Eh) * n);
      return E1 * (s0 + dt * n);
    case MODE_ROG_2: {
      const cpx<T> s = s0 + (hdt * Eh) * n;
      MP::st(&a.state[g], s);
      return s;
    }
    case MODE_NL:
      MP::st(&a.acc[g], n);
      return mk<T>(0, 0);
    default:  // MODE_PROJECT
      MP::st(&a.state[g], n);
      return mk<T>(0, 0);
  }
}

// S_next of component c at the modes of the forcing table (the forcing amplitude of the
// next stage needs Re<S_next, f>)
template <typename T, class MP>
__device__ __forceinline__ void shell_record(const PencilArgs<T>& a, int c, int kx, int ky, int kz,
                                             cpx<T> sn) {
  if (a.shell && kx <= a.fK && abs(ky) <= a.fK && abs(kz) <= a.fK) {
    const int D1 = 2 * a.fK + 1, D = D1 * D1 * (a.fK + 1);
    const int fi = ((kz + a.fK) * D1 + (ky + a.fK)) * (a.fK + 1) + kx;
    MP::st(&a.shell[c * D + fi], sn);
  }
}

// ---- pencil pass --------------------------------------------------------------------
// One tile: TX consecutive kx at one ky, all kz.  Shared memory: 3 component tiles (a 4th
// when there are two inputs or two outputs) and the twiddle table.  Every thread works on
// one fixed kx (NT is a multiple of TX), so the kx and ky factors of the phase and
// integrating-factor tables are loaded once per thread.
template <typename T, int N>
__host__ __device__ constexpr int pencil_tiles(int nF, int nOut) { return (nF > 1 || nOut > 1) ? 4 : 3; }

// True when every mode of a pencil tile (kx in [x0, x0 + TX), this ky, every kz) lies outside
// the truncation and none is in the forcing table: the truncated nonlinear term and the
// forcing vanish there, so the tile's forward transforms are skipped (Sec. 2, truncation).
template <typename T, int TX>
__device__ __forceinline__ bool pencil_tile_truncated(const PencilArgs<T>& a, int x0, int ky) {
  bool out;  // the no-double-alias mask lies inside the sphere: the spherical test is safe
  if (a.trunc == 1)
    out = x0 > a.Kimax || abs(ky) > a.Kimax;
  else
    out = (long long)x0 * x0 + (long long)ky * ky > (long long)a.K2max;
  const bool forced = (a.force != nullptr || a.shell != nullptr) && x0 <= a.fK && abs(ky) <= a.fK;
  return out && !forced;
}

// Zero columns of the outputs of a tile whose S_next vanishes (the inverse transforms of zero)
template <typename T, int N, int TX, int NT, class MP>
__device__ __forceinline__ void pencil_zero_outputs(const PencilArgs<T>& a, int nOut, int iy, int x0) {
  constexpr int M = N / 2;
  const size_t fstride = (size_t)N * N * M;
  if (threadIdx.x >= NT) return;
  for (int o = 0; o < nOut; ++o)
    for (int f = 0; f < 5; ++f)
      for (int i = threadIdx.x; i < N * TX; i += NT) {
        const int iz = i / TX, line = i % TX;
        MP::st(&a.out[o][f * fstride + ((size_t)iz * N + iy) * M + x0 + line], mk<T>(0, 0));
      }
}

// Last-stage output of a forward z transform of one input component: de-shift by
// e^{-i k.delta} (the kx, ky factor cxy is the thread's own: the thread's line is fixed) and
// the weight w.
template <typename T, int W, class MP>
struct DeshiftOut {
  cpx<T>* p;
  cpx<T> cxy;
  const cpx<T>* dz;  // z factors of the shift table, or null (no shift)
  T w;
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const {
    if (dz) v = mul_conj(v, cxy * MP::ld(&dz[e]));
    p[lf_idx<T, W>(e, line)] = w * v;
  }
};

// Energy and dissipation sums of the state a final-stage pencil tile writes (Sec. 3.4: E =
// 1/2 sum w |S|^2, eps = nu sum w k^2 |S|^2, w = 1 at kx = 0 and 2 elsewhere): each thread's
// sums (in T, a few modes each) are reduced across the block in FP64 and stored as the
// tile's pair; a fixed-order sum over the tiles follows.  Every thread of the block calls it.
template <typename T>
__device__ __forceinline__ void tile_energy_store(double* epart, T e, T d) {
  __shared__ double red[2][32];
  double a = (double)e, b = (double)d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    red[0][w] = a;
    red[1][w] = b;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x + 31) >> 5;
    a = l < nw ? red[0][l] : 0.0;
    b = l < nw ? red[1][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (l == 0) {
      epart[2 * blockIdx.x] = a;
      epart[2 * blockIdx.x + 1] = b;
    }
  }
}

// Spectral stage of a pencil tile with one input: the three components of F are staged,
// transformed in place (the last stage de-shifting and weighting), then one pass per mode
// applies N(0) = 0, truncation, projection and forcing and the RK stage combine of all three
// components, leaving S_next (shifted for the output when there is one output) in the tiles.
// MC: the stage mode fixed at compile time (-1: a.mode at run time)
template <typename T, int N, class MP, bool EP, int MC = -1, int V = 0>
__device__ __forceinline__ void pencil_spectral_one(const PencilArgs<T>& a, cpx<T>* buf, cpx<T>* tws,
                                                    int iy, int x0, int nOut, bool tz, T& eacc,
                                                    T& dacc) {
  const int mode = MC >= 0 ? MC : a.mode;
  using C = K2Cfg<T, N, V>;
  constexpr int M = N / 2, TX = C::TX, NT = C::NTP, tile = lf_rows<T, C::TX>(N) * TX;
  constexpr int PER = (tile + NT - 1) / NT;
  constexpr int DZ = NT / TX;
  const size_t fstride = (size_t)N * N * M;
  const int ky = kof(iy, N);
  const bool act = threadIdx.x < NT;
  const int line = threadIdx.x % TX, kx = x0 + line;
  const int iz0 = threadIdx.x / TX;
  const bool rd0 = mode != MODE_NL && mode != MODE_PROJECT;
  const cpx<T>* base0 = mode == MODE_RK4_4 ? a.acc : a.state;
  if (!tz)
    for (int c = 0; c < 3; ++c) stage_col_tile<T, N, TX, NT>(buf + c * tile, a.F[0] + c * fstride, iy, x0);
  cp_async_commit();
  if (NS_PENCIL_STAGE_STATE && rd0)  // the state tiles arrive during the forward transforms
    for (int c = 0; c < 3; ++c) stage_col_tile<T, N, TX, NT>(buf + (3 + c) * tile, base0 + c * fstride, iy, x0);
  cp_async_commit();
  load_twiddles(tws, a.tw, N);
  if (!tz) {
    cp_async_wait_pending<1>();
    __syncthreads();
    const cpx<T>* dz = a.dsh[0] ? a.dsh[0] + 2 * N : nullptr;
    cpx<T> d0 = mk<T>(1, 0);
    if (dz) d0 = MP::ld(&a.dsh[0][kx]) * MP::ld(&a.dsh[0][N + iy]);
#pragma unroll (kPencilUnroll)
    for (int c = 0; c < 3; ++c) {
      cpx<T>* t = buf + c * tile;
      cfft_ip_to<T, N, 1, TX, NT, true, -1, true, C::RZ>(SmTile<T, TX>{t}, t,
                                                         DeshiftOut<T, TX, MP>{t, d0, dz, a.wF[0]}, tws);
    }
    __syncthreads();
  }

  const bool pre = nOut == 1 && a.osh[0] != nullptr;
  cpx<T> oxy = mk<T>(1, 0);
  if (pre) oxy = cmul_fixed(MP::ld(&a.osh[0][kx]), MP::ld(&a.osh[0][N + iy]));
  const bool useE = mode != MODE_INIT && mode != MODE_NL && mode != MODE_PROJECT;
  T e1xy = 1, ehxy = 1;
  if (useE) {
    e1xy = a.ifac[kx] * a.ifac[iy];
    ehxy = a.ifac[N + kx] * a.ifac[N + iy];
  }
  if (NS_PENCIL_STAGE_STATE) {
    cp_async_wait_pending<0>();
    __syncthreads();
  }
  if (act) {
    constexpr int CHK = PER < NS_PENCIL_CHK ? PER : NS_PENCIL_CHK;  // modes whose state loads are in flight together
    const bool rd1 = mode == MODE_RK4_2 || mode == MODE_RK4_3;
    const size_t gxy = (size_t)iy * M + kx;
    for (int i0 = 0; i0 < PER; i0 += CHK) {
      cpx<T> s0[3][CHK];  // (the RK4 accumulator, read by two modes only, is loaded on use)
#pragma unroll
      for (int j = 0; j < CHK; ++j) {
        const int iz = iz0 + (i0 + j) * DZ;
        const size_t g = gxy + (size_t)iz * N * M;
        const bool ok = iz < N && i0 + j < PER;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s0[c][j] = mk<T>(0, 0);
          if (ok && rd0)
            s0[c][j] = NS_PENCIL_STAGE_STATE ? buf[(3 + c) * tile + lf_idx<T, TX>(iz, line)]
                                             : MP::ldw(&base0[c * fstride + g]);
        }
      }
#pragma unroll
      for (int j = 0; j < CHK; ++j) {
        const int iz = iz0 + (i0 + j) * DZ, e = lf_idx<T, TX>(iz, line);
        if (iz >= N || i0 + j >= PER) break;
        const size_t g = gxy + (size_t)iz * N * M;
        const int kz = kof(iz, N);
        cpx<T> nv[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
        if (!tz) {
          nv[0] = buf[e];
          nv[1] = buf[tile + e];
          nv[2] = buf[2 * tile + e];
          project_point(a, kx, ky, kz, nv);
        }
        T E1 = 1, Eh = 1;
        if (useE) {
          E1 = e1xy * a.ifac[iz];
          Eh = ehxy * a.ifac[N + iz];
        }
        cpx<T> shz = oxy;
        if (pre) shz = cmul_fixed(oxy, MP::ld(&a.osh[0][2 * N + iz]));
        T m2 = 0;  // |S|^2 of the written state (EP: final stages with a.epart)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const cpx<T> s1 = rd1 ? MP::ldw(&a.acc[c * fstride + g]) : mk<T>(0, 0);
          cpx<T> sn = stage_combine<T, MP>(a, c, c * fstride + g, nv[c], s0[c][j], s1, E1, Eh, mode);
          shell_record<T, MP>(a, c, kx, ky, kz, sn);
          if constexpr (EP) m2 += sn.x * sn.x + sn.y * sn.y;
          if (pre) sn = cmul_fixed(sn, shz);
          buf[c * tile + e] = sn;
        }
        if constexpr (EP) {
          const T wm = (kx == 0 ? T(1) : T(2)) * m2;
          eacc += wm;
          dacc += wm * (T)(kx * kx + ky * ky + kz * kz);
        }
      }
    }
  }
  __syncthreads();
}

// NFC, NOC: the number of inputs and outputs known at compile time (-1: read from the
// arguments).  (1, 1) is every RK2, Rogallo and RK4 stage, (2, 2) the exact scheme's stage;
// fixing them keeps those kernels free of register spills.
template <typename T, int N, class MP, int NFC = -1, int NOC = -1, bool EP = false, int MC = -1,
          int V = 0>
__device__ __forceinline__ void pencil_tile(const PencilArgs<T>& a, int tile_id, cpx<T>* buf) {
  using C = K2Cfg<T, N, V>;
  const int nF = NFC >= 0 ? NFC : a.nF, nOut = NOC >= 0 ? NOC : a.nOut;
  constexpr int M = N / 2, TX = C::TX, NT = C::NTP, tile = lf_rows<T, C::TX>(N) * TX;
  constexpr int PER = (tile + NT - 1) / NT;  // modes per thread (the last may not exist)
  static_assert(NT % TX == 0, "every thread keeps one kx");
  // component tile c is buf + c * tile (pointer arithmetic, not an array: no local memory)
  auto bc = [&](int c) { return buf + c * tile; };
  cpx<T>* b3 = buf + 3 * tile;
  cpx<T>* tws = buf + (NFC == 1 && NS_PENCIL_STAGE_STATE ? 6 : pencil_tiles<T, N>(nF, nOut)) * tile;
  constexpr int ntx = M / TX;
  const int iy = a.iy0 + tile_id / ntx;  // (iy0: first ky row of a rank-range launch)
  const int x0 = (tile_id % ntx) * TX;
  const size_t fstride = (size_t)N * N * M;
  const int ky = kof(iy, N);
  const bool act = threadIdx.x < NT;
  const int line = threadIdx.x % TX, kx = x0 + line;
  const int iz0 = threadIdx.x / TX;  // this thread's modes: iz = iz0 + i * (NT / TX)
  constexpr int DZ = NT / TX;

  const bool pre = nOut == 1 && a.osh[0] != nullptr;  // S_next is shifted in the tiles
  const bool tt = pencil_tile_truncated<T, TX>(a, x0, ky);  // N = 0 on the whole tile
  const bool tz = nF > 0 && tt;                               // so its inputs are not transformed
  T eacc = 0, dacc = 0;  // energy sums of the written state (a.epart)
  if constexpr (NFC == 1) {
    pencil_spectral_one<T, N, MP, EP, MC, V>(a, buf, tws, iy, x0, nOut, tz, eacc, dacc);
  } else {
    const int nFe = tz ? 0 : nF;  // inputs that are transformed
    // 1) inputs: all three components staged asynchronously, then transformed in place
    if (nFe > 0) {
      for (int c = 0; c < 3; ++c) stage_col_tile<T, N, TX, NT>(bc(c), a.F[0] + c * fstride, iy, x0);
    }
    load_twiddles(tws, a.tw, N);  // also the barrier after which the staged tiles may be read
    if (nFe > 0) {
      cp_async_wait_all();
      __syncthreads();
      cpx<T> d0 = mk<T>(1, 0), d1 = mk<T>(1, 0);
      if (a.dsh[0]) d0 = MP::ld(&a.dsh[0][kx]) * MP::ld(&a.dsh[0][N + iy]);
      if (nF > 1 && a.dsh[1]) d1 = MP::ld(&a.dsh[1][kx]) * MP::ld(&a.dsh[1][N + iy]);
      for (int c = 0; c < 3; ++c) {
        cfft_ip<T, N, 1, TX, NT, true, -1, true, C::RZ>(SmTile<T, TX>{bc(c)}, bc(c), tws);
        __syncthreads();
        if (nF > 1) {
          stage_col_tile<T, N, TX, NT>(b3, a.F[1] + c * fstride, iy, x0);
          cp_async_wait_all();
          __syncthreads();
          cfft_ip<T, N, 1, TX, NT, true, -1, true, C::RZ>(SmTile<T, TX>{b3}, b3, tws);
          __syncthreads();
        }
        if (act) {
  #pragma unroll 4
          for (int i = 0; i < PER; ++i) {
            const int iz = iz0 + i * DZ, e = lf_idx<T, TX>(iz, line);
            if (iz >= N) break;
            cpx<T> v = bc(c)[e];
            if (a.dsh[0]) v = mul_conj(v, d0 * MP::ld(&a.dsh[0][2 * N + iz]));
            v = a.wF[0] * v;
            if (nF > 1) {
              cpx<T> w = b3[e];
              if (a.dsh[1]) w = mul_conj(w, d1 * MP::ld(&a.dsh[1][2 * N + iz]));
              v = v + a.wF[1] * w;
            }
            bc(c)[e] = v;
          }
        }
        __syncthreads();
      }
      // 2a) N(0) = 0, truncation, projection, forcing (all components of a mode at once)
      if (act) {
        for (int i = 0; i < PER; ++i) {
          const int iz = iz0 + i * DZ, e = lf_idx<T, TX>(iz, line);
          if (iz >= N) break;
          cpx<T> nv[3] = {bc(0)[e], bc(1)[e], bc(2)[e]};
          project_point(a, kx, ky, kof(iz, N), nv);
          bc(0)[e] = nv[0];
          bc(1)[e] = nv[1];
          bc(2)[e] = nv[2];
        }
      }
    }

    // 2b) stage combine per component, the state of the thread's modes loaded together
    cpx<T> oxy = mk<T>(1, 0);
    if (pre) oxy = cmul_fixed(MP::ld(&a.osh[0][kx]), MP::ld(&a.osh[0][N + iy]));
    const bool useE = a.mode != MODE_INIT && a.mode != MODE_NL && a.mode != MODE_PROJECT;
    T e1xy = 1, ehxy = 1;
    if (useE) {
      e1xy = a.ifac[kx] * a.ifac[iy];
      ehxy = a.ifac[N + kx] * a.ifac[N + iy];
    }
    if (act) {
      constexpr int CHK = PER < 8 ? PER : 8;  // modes whose state loads are in flight together
      const bool rd0 = a.mode != MODE_NL && a.mode != MODE_PROJECT;
      const bool rd1 = a.mode == MODE_RK4_2 || a.mode == MODE_RK4_3;
      const cpx<T>* base0 = a.mode == MODE_INIT ? a.src : (a.mode == MODE_RK4_4 ? a.acc : a.state);
      for (int c = 0; c < 3; ++c)
      for (int i0 = 0; i0 < PER; i0 += CHK) {
        const size_t gc = c * fstride + (size_t)iy * M + kx;
        cpx<T> s0[CHK], s1[CHK];
  #pragma unroll
        for (int j = 0; j < CHK; ++j) {
          const int iz = iz0 + (i0 + j) * DZ;
          const size_t g = gc + (size_t)iz * N * M;
          s0[j] = s1[j] = mk<T>(0, 0);
          if (iz < N && i0 + j < PER) {
            if (rd0) s0[j] = MP::ldw(&base0[g]);
            if (rd1) s1[j] = MP::ldw(&a.acc[g]);
          }
        }
  #pragma unroll
        for (int j = 0; j < CHK; ++j) {
          const int iz = iz0 + (i0 + j) * DZ, e = lf_idx<T, TX>(iz, line);
          if (iz >= N || i0 + j >= PER) break;
          const size_t g = gc + (size_t)iz * N * M;
          T E1 = 1, Eh = 1;
          if (useE) {
            E1 = e1xy * a.ifac[iz];
            Eh = ehxy * a.ifac[N + iz];
          }
          const cpx<T> n = nFe > 0 ? bc(c)[e] : mk<T>(0, 0);
          cpx<T> sn = stage_combine<T, MP>(a, c, g, n, s0[j], s1[j], E1, Eh, a.mode);
          shell_record<T, MP>(a, c, kx, ky, kof(iz, N), sn);
          if (a.epart) {
            const int kz = kof(iz, N);
            const T wm = (kx == 0 ? T(1) : T(2)) * (sn.x * sn.x + sn.y * sn.y);
            eacc += wm;
            dacc += wm * (T)(kx * kx + ky * ky + kz * kz);
          }
          if (pre) sn = cmul_fixed(sn, cmul_fixed(oxy, MP::ld(&a.osh[0][2 * N + iz])));
          bc(c)[e] = sn;
        }
      }
    }
    __syncthreads();
  }

  // one-input tiles take the sums only in the EP variant; the others whenever a.epart is set
  if constexpr (NFC == 1) {
    if constexpr (EP) tile_energy_store<T>(a.epart, eacc, dacc);
  } else if (a.epart) {
    tile_energy_store<T>(a.epart, eacc, dacc);
  }
  if (tt) {  // S_next vanishing on the whole tile (a truncated state): zero outputs, no transforms
    bool nz = false;
    if (act)
      for (int i = 0; i < PER; ++i) {
        const int iz = iz0 + i * DZ, e = lf_idx<T, TX>(iz, line);
        if (iz >= N) break;
        for (int c = 0; c < 3; ++c) {
          const cpx<T> v = bc(c)[e];
          nz = nz || v.x != T(0) || v.y != T(0);
        }
      }
    if (!__syncthreads_or(nz)) {
      pencil_zero_outputs<T, N, TX, NT, MP>(a, nOut, iy, x0);
      return;
    }
  }
  if (nOut == 1) {
    // u_z first (its tile then serves as the work tile), then u_x, d_z u_x, u_y, d_z u_y
    const cpx<T>* sh = pre ? nullptr : a.osh[0];
    cfft_src_in_work<T, N, 1, TX, NT, true, 1, C::RZ>(PencilOutSrc<T, N, TX, MP>{bc(2), sh, iy, x0, false},
                                               ColOut<T, N, TX, MP>{a.out[0] + 2 * fstride, iy, x0},
                                               bc(2), tws);
    __syncthreads();
#pragma unroll (kPencilUnroll)
    for (int i = 0; i < 4; ++i) {
      const int f = (i & 1) ? 3 + (i >> 1) : (i >> 1), c = f < 3 ? f : f - 3;  // 0, 3, 1, 4
      cfft<T, N, 1, TX, NT, true, 1, C::RZ>(PencilOutSrc<T, N, TX, MP>{bc(c), sh, iy, x0, f >= 3},
                                     ColOut<T, N, TX, MP>{a.out[0] + f * fstride, iy, x0}, bc(2), tws);
      __syncthreads();
    }
  } else {
    for (int o = 0; o < nOut; ++o) {
      for (int f = 0; f < 5; ++f) {
        const int c = f < 3 ? f : f - 3;
        cfft<T, N, 1, TX, NT, true, 1, C::RZ>(PencilOutSrc<T, N, TX, MP>{bc(c), a.osh[o], iy, x0, f >= 3},
                                       ColOut<T, N, TX, MP>{a.out[o] + f * fstride, iy, x0}, b3, tws);
        __syncthreads();
      }
    }
  }
}

// the two-input variant holds 4 shared tiles (3 blocks per SM at most): it is given the
// registers of 2 resident blocks rather than spill
// EP: the one-input variant that also stores the tile's energy sums (a.epart non-null)
// MC: the stage mode at compile time (the Rogallo stages) or -1 (a.mode); V: tile variant
template <typename T, int N, int NFC, int NOC, bool EP = false, int MC = -1, int V = 0>
__global__ void __launch_bounds__(K2Cfg<T, N, V>::NTP, (NFC == 2 || (NFC == 1 && NS_PENCIL_STAGE_STATE))
                                                            ? cmin(2, K2Cfg<T, N, V>::MINB_P)
                                                            : K2Cfg<T, N, V>::MINB_P)
    k2_pencil(PencilArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pencil_tile<T, N, MemNC, NFC, NOC, EP, MC, V>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smem_raw));
}

// ---- slab pass: y transforms --------------------------------------------------------
// field F of the spectral-in-xy pair (u, omega) formed on the fly from the mixed fields
// staged in shared memory ([slot][e][line], TY lines): slots 0, 1, 2 hold u_x, u_y, u_z,
// then d_z u_x and d_z u_y replace u_x and u_y in slots 0 and 1 once those are transformed.
template <typename T, int N, int F, int TY>
struct YInvSrc {
  const cpx<T>* m;
  int x0;
  __device__ __forceinline__ cpx<T> get(int line, int e) const {
    constexpr int fs = lf_rows<T, TY>(N) * TY;
    const int i = lf_idx<T, TY>(e, line);
    const T kx = (T)(x0 + line), ky = (T)kof(e, N);
    if (F == 0) return m[i];
    if (F == 1) return m[i + fs];
    if (F == 2) return m[i + 2 * fs];
    if (F == 3) return mul_si(m[i + 2 * fs], ky) - m[i + fs];       // i ky u_z - d_z u_y
    if (F == 4) return m[i] - mul_si(m[i + 2 * fs], kx);            // d_z u_x - i kx u_z
    return mul_si(m[i + fs], kx) - mul_si(m[i], ky);                // i kx u_y - i ky u_x
  }
};
template <typename T, int N, class MP>
struct ScrCol {  // one field [plane][y|ky][kx], column tile of a plane (scratch or Ft)
  cpx<T>* p;
  int zg, x0;
  __device__ __forceinline__ cpx<T> get(int line, int e) const {
    return MP::ldw(&p[((size_t)zg * N + e) * (N / 2) + x0 + line]);
  }
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const {
    MP::st(&p[((size_t)zg * N + e) * (N / 2) + x0 + line], v);
  }
};

// One output field of the y-inverse.  IP: the field's only input is slot SLOT, which the
// transform then uses as its work tile (its inputs are read before the tile is written);
// otherwise the transform goes through the work tile W.
template <typename T, int N, int F, class MP, int TY, int NT, bool IP = false>
__device__ __forceinline__ void yinv_field(const SlabArgs<T>& a, cpx<T>* in, cpx<T>* W, int zg,
                                           int x0, size_t sstride, const cpx<T>* tws) {
  using C = K2Cfg<T, N>;
  const YInvSrc<T, N, F, TY> src{in, x0};
  const ScrCol<T, N, MP> dst{a.scr + F * sstride, zg, x0};
  if constexpr (IP)
    cfft_src_in_work<T, N, 1, TY, NT, true, 1, C::RYI>(src, dst, in + F * (lf_rows<T, TY>(N) * TY), tws);
  else
    cfft<T, N, 1, TY, NT, true, 1, C::RYI>(src, dst, W, tws);
  __syncthreads();
}

// One tile: TYI consecutive kx of plane zg, in 4 shared tiles (3 input slots and a work tile).
// u_x, u_y, u_z are staged first; omega_z (from u_x, u_y) goes through the work tile, u_x and
// u_y are transformed in place, and d_z u_x, d_z u_y are then copied into their slots while the
// next transform runs; omega_y, omega_x and u_z (in place) follow.
// TY_, NT_: tile width and threads (the defaults of the size; the slab pipeline uses 4 columns)
template <typename T, int N, class MP, int TY_ = K2Cfg<T, N>::TYI, int NT_ = K2Cfg<T, N>::NTYI>
__device__ __forceinline__ void yinv_tile(const SlabArgs<T>& a, int tx, int zg, cpx<T>* in) {
  constexpr int M = N / 2, TY = TY_, NT = NT_, tile = lf_rows<T, TY>(N) * TY;
  cpx<T>* W = in + 3 * tile;
  cpx<T>* tws = in + 4 * tile;
  const int x0 = tx * TY, z = a.z0 + zg;
  const size_t sstride = (size_t)a.G * N * M;
  const size_t fs = (size_t)N * N * M;
  for (int f = 0; f < 3; ++f) stage_col_tile<T, N, TY, NT, true>(in + f * tile, a.mixed + f * fs, z, x0);
  cp_async_commit();
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[tw_pad(i)] = ldg(&a.tw[i]);
  cp_async_wait_pending<0>();
  __syncthreads();
  yinv_field<T, N, 5, MP, TY, NT>(a, in, W, zg, x0, sstride, tws);        // omega_z
  yinv_field<T, N, 0, MP, TY, NT, true>(a, in, W, zg, x0, sstride, tws);  // u_x in slot 0
  stage_col_tile<T, N, TY, NT, true>(in, a.mixed + 3 * fs, z, x0);        // d_z u_x -> slot 0
  cp_async_commit();
  yinv_field<T, N, 1, MP, TY, NT, true>(a, in, W, zg, x0, sstride, tws);  // u_y in slot 1
  stage_col_tile<T, N, TY, NT, true>(in + tile, a.mixed + 4 * fs, z, x0); // d_z u_y -> slot 1
  cp_async_commit();
  cp_async_wait_pending<1>();
  __syncthreads();
  yinv_field<T, N, 4, MP, TY, NT>(a, in, W, zg, x0, sstride, tws);        // omega_y
  cp_async_wait_pending<0>();
  __syncthreads();
  yinv_field<T, N, 3, MP, TY, NT>(a, in, W, zg, x0, sstride, tws);        // omega_x
  yinv_field<T, N, 2, MP, TY, NT, true>(a, in, W, zg, x0, sstride, tws);  // u_z in slot 2
}

template <typename T, int N, int V = 0>
__global__ void __launch_bounds__(K2Cfg<T, N, V>::NTYI) k2_yinv(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  yinv_tile<T, N, MemNC, K2Cfg<T, N, V>::TYI, K2Cfg<T, N, V>::NTYI>(a, blockIdx.x, blockIdx.y,
                                                                  reinterpret_cast<cpx<T>*>(smem_raw));
}

#ifndef NS_FT_SKIP
#define NS_FT_SKIP 1
#endif
// Ft output of the forward y transforms: a mode is stored unless every pencil tile of
// a.skip_tx columns that holds it lies outside the truncation and the forcing block (the
// criterion of pencil_tile_truncated with x0 the tile's first column): the pencil passes
// neither load nor transform such tiles.
template <typename T, int N, class MP>
struct FtColOut {
  cpx<T>* p;
  int z, x0;
  const SlabArgs<T>* a;
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const {
    if (a->skip_tx > 0) {
      const int kx = x0 + line, px = kx - kx % a->skip_tx, ky = kof(e, N);
      const bool out = a->trunc == 1 ? (px > a->Kimax || abs(ky) > a->Kimax) : px * px + ky * ky > a->K2max;
      const bool forced = a->fK >= 0 && px <= a->fK && abs(ky) <= a->fK;
      if (out && !forced) return;
    }
    MP::st(&p[((size_t)z * N + e) * (N / 2) + x0 + line], v);
  }
};

template <typename T, int N, class MP, int V = 0>
__device__ __forceinline__ void yfwd_tile(const SlabArgs<T>& a, int tx, int zg, cpx<T>* W) {
  using C = K2Cfg<T, N, V>;
  const int x0 = tx * C::TY, z = a.z0 + zg;
  const size_t sstride = (size_t)a.G * N * (N / 2);
  const size_t fstride = (size_t)N * N * (N / 2);
  cpx<T>* tws = W + lf_rows<T, C::TY>(N) * C::TY;
  load_twiddles(tws, a.tw, N);
  for (int f = 0; f < 3; ++f) {
    cfft<T, N, 1, C::TY, C::NTY, true, -1, C::RYF>(ScrCol<T, N, MP>{a.scr + f * sstride, zg, x0},
                                                   FtColOut<T, N, MP>{a.Ft + f * fstride, z, x0, &a}, W, tws);
    __syncthreads();
  }
}

template <typename T, int N, int V = 0>
__global__ void __launch_bounds__(K2Cfg<T, N, V>::NTY, 2) k2_yfwd(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  yfwd_tile<T, N, MemNC, V>(a, blockIdx.x, blockIdx.y, reinterpret_cast<cpx<T>*>(smem_raw));
}

// ---- slab pass: x rows --------------------------------------------------------------
#ifndef NS_XROW_PAIRS
#define NS_XROW_PAIRS 1
#endif
// One tile: RX consecutive rows (plane, y) of the group.  Each row holds the half spectra
// (kx < N/2, the Nyquist mode zero) of 6 real fields, and two real rows share one complex line
// of length N: the line of fields a and b is z = a + i b, whose full spectrum is
// Z[k] = A[k] + i B[k] and Z[N - k] = conj(A[k]) + i conj(B[k]) (A[0], B[0] real).  Inverse
// lines per row: (u_x, u_y), (u_z, w_x), (w_y, w_z); the products come back as lines (f_0, f_1)
// of every row and (f_2 of row q, f_2 of row q + RXh), whose forward transforms P split into
// F_a[k] = (P[k] + conj(P[N - k])) / 2 and F_b[k] = (P[k] - conj(P[N - k])) / (2 i).  All
// transforms are unnormalised, as the r2c / c2r pair they replace.
template <typename T, int N, class MP, int V = 0>
__device__ __forceinline__ void xrow_tile(const SlabArgs<T>& a, int tile_id, cpx<T>* buf) {
  using C = K2Cfg<T, N, V>;
  constexpr int M = N / 2, RX = C::RX, NT = C::NTX, RXh = (RX + 1) / 2;
  constexpr int NLI = 3 * RX, NLF = RX + RXh;  // inverse and forward lines
  const WorkTile<T, N, NLI, false> L{buf};     // line p RX + r: pair p of row r
  cpx<T>* tws = buf + C::XELEMS;
  const bool act = threadIdx.x < NT;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[tw_pad(i)] = ldg(&a.tw[i]);
  const int rows_total = a.G * N;
  const int r0 = tile_id * RX;
  const int nr = min(RX, rows_total - r0);
  const size_t sstride = (size_t)a.G * N * M;

  // FP32 with NT a multiple of M / 2: every thread keeps one pair of modes (k, k + 1) and
  // walks lines, so the loads and stores are 16 bytes wide and its indices loop-invariant
  constexpr int H = M / 2;
  constexpr bool PAIR = NS_XROW_PAIRS && sizeof(T) == 4 && NT % H == 0;
  constexpr int GP = PAIR ? NT / H : 1;  // lines in flight per pass of the block
  const int kp2 = 2 * (threadIdx.x % H), g0 = threadIdx.x / H;
  if constexpr (PAIR) {
    // 1) item (line = p RX + row, k pair): modes k, k + 1 of fields 2p and 2p + 1 give Z[k],
    //    Z[k + 1], Z[N - k], Z[N - k - 1] of the line (k = 0: Z[0] from the real parts and
    //    Z[M] = 0); all loads first, rows past the end of the group are zero
    constexpr int KC = (NLI + GP - 1) / GP;
    float4 xa[KC], xb[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int line = g0 + c * GP, p = line / RX, row = line % RX;
      xa[c] = xb[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act && (NLI % GP == 0 || line < NLI) && row < nr) {
        const cpx<float>* src = reinterpret_cast<const cpx<float>*>(a.scr) + 2 * p * sstride + (size_t)(r0 + row) * M + kp2;
        xa[c] = MP::ld2(src);
        xb[c] = MP::ld2(src + sstride);
      }
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const int line = g0 + c * GP;
      if (act && (NLI % GP == 0 || line < NLI)) {
        const float4 A = xa[c], B = xb[c];
        if (kp2 == 0) {
          L.put(line, 0, mk<T>(A.x, B.x));
          L.put(line, M, mk<T>(0, 0));
        } else {
          L.put(line, kp2, mk<T>(A.x - B.y, A.y + B.x));
          L.put(line, N - kp2, mk<T>(A.x + B.y, B.x - A.y));
        }
        L.put(line, kp2 + 1, mk<T>(A.z - B.w, A.w + B.z));
        L.put(line, N - kp2 - 1, mk<T>(A.z + B.w, B.z - A.w));
      }
    }
  } else {
  // 1) item (p, row, k) reads mode k of fields 2p and 2p + 1 and writes Z[k] and Z[N - k] of
  //    line p RX + row (k = 0: Z[0] from the real parts and Z[M] = 0).  Every load is issued
  //    before any store; rows past the end of the group are zero.
  constexpr int NI = 3 * RX * M, KI = (NI + NT - 1) / NT;
  cpx<T> xa[KI], xb[KI];
#pragma unroll
  for (int c = 0; c < KI; ++c) {
    const int i = threadIdx.x + c * NT;
    xa[c] = xb[c] = mk<T>(0, 0);
    if (act && (NI % NT == 0 || i < NI)) {
      const int p = i / (RX * M), row = (i / M) % RX, k = i % M;
      if (row < nr) {
        const cpx<T>* src = a.scr + 2 * p * sstride + (size_t)(r0 + row) * M + k;
        xa[c] = MP::ld(src);
        xb[c] = MP::ld(src + sstride);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < KI; ++c) {
    const int i = threadIdx.x + c * NT;
    if (act && (NI % NT == 0 || i < NI)) {
      const int p = i / (RX * M), row = (i / M) % RX, k = i % M;
      const int line = p * RX + row;
      const cpx<T> A = xa[c], B = xb[c];
      if (k == 0) {
        L.put(line, 0, mk<T>(A.x, B.x));
        L.put(line, M, mk<T>(0, 0));
      } else {
        L.put(line, k, mk<T>(A.x - B.y, A.y + B.x));      // A + i B
        L.put(line, N - k, mk<T>(A.x + B.y, B.x - A.y));  // conj(A) + i conj(B)
      }
    }
  }
  }
  __syncthreads();
  // 2) the 3 RX inverse transforms in one in-place call
  cfft_ip<T, N, 1, NLI, NT, false, 1, true, C::RXR>(L, buf, tws);
  __syncthreads();

  // 3) u x omega: item (q, x) takes rows q and q + RXh (when RX is odd the last q has one) at
  //    point x, writes (f_0, f_1) over each row's first line and (f_2(q), f_2(q + RXh)) over
  //    line RX + q (row q's second line): every line it writes is one it has read
  T m[3] = {T(0), T(0), T(0)};  // max |u_i| over the rows (CFL), padding rows are zero
  for (int i = threadIdx.x; act && i < RXh * N; i += NT) {
    const int q = i / N, x = i % N;
    T f2[2] = {T(0), T(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = q + h * RXh;
      if (row < RX) {
        const cpx<T> z0 = L.get(row, x), z1 = L.get(RX + row, x), z2 = L.get(2 * RX + row, x);
        const T ux = z0.x, uy = z0.y, uz = z1.x, wx = z1.y, wy = z2.x, wz = z2.y;
        m[0] = fmax(m[0], fabs(ux));
        m[1] = fmax(m[1], fabs(uy));
        m[2] = fmax(m[2], fabs(uz));
        L.put(row, x, mk<T>(uy * wz - uz * wy, uz * wx - ux * wz));
        f2[h] = ux * wy - uy * wx;
      }
    }
    L.put(RX + q, x, mk<T>(f2[0], f2[1]));
  }
  __syncthreads();
  // lines NLF .. 3 RX - 1 are free now
  if (a.umax) block_max3<T>(m[0], m[1], m[2], reinterpret_cast<T*>(buf + NLF * L.LS), a.umax);
  // 4) the NLF forward transforms of the products
  cfft_ip<T, N, 1, NLF, NT, false, -1, true, C::RXR>(WorkTile<T, N, NLF, false>{buf}, buf, tws);
  __syncthreads();

  // 5) split and store: item (line, k), k < M (pairs of modes in the FP32 layout above)
  if constexpr (PAIR) {
#pragma unroll
    for (int c = 0; c < (NLF + GP - 1) / GP; ++c) {
      const int line = g0 + c * GP;
      if (!act || (NLF % GP != 0 && line >= NLF)) break;
      const cpx<T> P0 = L.get(line, kp2), Q0 = L.get(line, kp2 == 0 ? 0 : N - kp2);
      const cpx<T> P1 = L.get(line, kp2 + 1), Q1 = L.get(line, N - kp2 - 1);
      const float4 Fa = make_float4(0.5f * (P0.x + Q0.x), 0.5f * (P0.y - Q0.y), 0.5f * (P1.x + Q1.x), 0.5f * (P1.y - Q1.y));
      const float4 Fb = make_float4(0.5f * (P0.y + Q0.y), 0.5f * (Q0.x - P0.x), 0.5f * (P1.y + Q1.y), 0.5f * (Q1.x - P1.x));
      const bool own = line < RX;
      const int ra = own ? line : line - RX, rb = own ? line : line - RX + RXh;
      const int fa = own ? 0 : 2, fb = own ? 1 : 2;
      cpx<float>* scr = reinterpret_cast<cpx<float>*>(a.scr);
      if (ra < nr) MP::st2(&scr[fa * sstride + (size_t)(r0 + ra) * M + kp2], Fa);
      if (rb < nr) MP::st2(&scr[fb * sstride + (size_t)(r0 + rb) * M + kp2], Fb);
    }
    return;
  }
  constexpr int NO = NLF * M;
  for (int i = threadIdx.x; act && i < NO; i += NT) {
    const int line = i / M, k = i % M;
    const cpx<T> P = L.get(line, k), Q = L.get(line, k == 0 ? 0 : N - k);
    const cpx<T> Fa = mk<T>(T(0.5) * (P.x + Q.x), T(0.5) * (P.y - Q.y));
    const cpx<T> Fb = mk<T>(T(0.5) * (P.y + Q.y), T(0.5) * (Q.x - P.x));
    const bool own = line < RX;  // (f_0, f_1) of row `line`, else f_2 of rows q, q + RXh
    const int ra = own ? line : line - RX, rb = own ? line : line - RX + RXh;
    const int fa = own ? 0 : 2, fb = own ? 1 : 2;
    if (ra < nr) MP::st(&a.scr[fa * sstride + (size_t)(r0 + ra) * M + k], Fa);
    if (rb < nr) MP::st(&a.scr[fb * sstride + (size_t)(r0 + rb) * M + k], Fb);
  }
}

template <typename T, int N, int V = 0>
__global__ void __launch_bounds__(K2Cfg<T, N, V>::NTX, K2Cfg<T, N, V>::MINB_X) k2_xrow(SlabArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xrow_tile<T, N, MemNC, V>(a, blockIdx.x, reinterpret_cast<cpx<T>*>(smem_raw));
}

// ---- slab pipeline: the three slab kernels as one persistent launch -------------------
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Control block of a pipeline launch (zeroed by the host before each launch).
struct PipeCtl {
  unsigned long long* next;  // ticket counter
  int* done;                 // [3][N]: finished y-inverse, x-row and y-forward tiles per plane
  int* abort;                // set when a wait gives up: every block leaves its loop
  long long spin_limit;      // polls before a wait gives up (then bit PIPE_ERR_TIMEOUT in err)
  int ring, lag;             // scratch planes in the ring; slots between the three stages
  int stall;                 // test hook: added to every awaited count (waits cannot succeed)
};
constexpr int PIPE_ERR_TIMEOUT = 0x100;
#ifndef NS_PIPE_MINB
#define NS_PIPE_MINB 3  // resident blocks per SM the register allocation must allow
#endif

// Work items of plane z: y-inverse tiles of 4 columns, x-row tiles of RX rows, y-forward
// tiles; tickets in slot order, slot s = [y-inverse(s), x rows(s - lag), y-forward(s - 2 lag)].
template <typename T, int N>
struct PipeCfg {
  using C = K2Cfg<T, N>;
  static constexpr int M = N / 2;
  static constexpr int TYP = 4;
  static constexpr int NTYP = round_warps(TYP * N / C::RYI);
  static constexpr int nYI = M / TYP, nX = N / C::RX, nYF = M / C::TY;
  static constexpr int per_slot = nYI + nX + nYF;
  static constexpr int NT = cmax(cmax(NTYP, C::NTX), C::NTY);
  static constexpr bool ok = N % C::RX == 0 && M % TYP == 0 && TYP % C::MINW == 0;
  static constexpr size_t smem = sizeof(cpx<T>) *
      cmax(cmax(4 * lf_rows<T, TYP>(N) * TYP, lf_rows<T, C::TY>(N) * C::TY), C::XELEMS) +
      sizeof(cpx<T>) * tw_elems(N);
};

// One slab pass over all N planes with the scratch as a ring of `ring` planes: every item
// waits (bounded) for the items it reads: x rows(z) for y-inverse(z), y-forward(z) for
// x rows(z), y-inverse(z) for y-forward(z - ring) (the ring slot it overwrites).  Each waits on
// an earlier ticket, held by a running block, so the pipeline progresses whatever the number
// of resident blocks.  Data written in the launch is read through L2 (MemCG).
// the y-pass tile bodies as separate functions (the union of the three bodies in one
// allocation spilled); the x-row body stays inline
template <typename T, int N>
__device__ __noinline__ void pipe_yinv(const SlabArgs<T>& b, int tile, int zs, cpx<T>* smem) {
  yinv_tile<T, N, MemCG, PipeCfg<T, N>::TYP, PipeCfg<T, N>::NTYP>(b, tile, zs, smem);
}
template <typename T, int N>
__device__ __noinline__ void pipe_yfwd(const SlabArgs<T>& b, int tile, int zs, cpx<T>* smem) {
  yfwd_tile<T, N, MemCG>(b, tile, zs, smem);
}

template <typename T, int N>
__global__ void __launch_bounds__(PipeCfg<T, N>::NT, NS_PIPE_MINB)
    k2_slabpipe(SlabArgs<T> a, PipeCtl c) {
  using P = PipeCfg<T, N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* smem = reinterpret_cast<cpx<T>*>(smem_raw);
  __shared__ long long s_t;
  __shared__ int s_go;
  const long long total = (long long)(N + 2 * c.lag) * P::per_slot;
  for (;;) {
    if (threadIdx.x == 0) s_t = (long long)atomicAdd(c.next, 1ull);
    __syncthreads();
    const long long tk = s_t;
    __syncthreads();
    if (tk >= total) break;
    const int slot = (int)(tk / P::per_slot), r = (int)(tk % P::per_slot);
    int type, z, tile;
    if (r < P::nYI) {
      type = 0; z = slot; tile = r;
    } else if (r < P::nYI + P::nX) {
      type = 1; z = slot - c.lag; tile = r - P::nYI;
    } else {
      type = 2; z = slot - 2 * c.lag; tile = r - P::nYI - P::nX;
    }
    if (z < 0 || z >= N) continue;
    const int wtype = type == 0 ? 2 : type - 1;
    const int wz = type == 0 ? z - c.ring : z;
    const int wcnt = (type == 0 ? P::nYF : type == 1 ? P::nYI : P::nX) + c.stall;
    if (threadIdx.x == 0) {
      int ok = 1;
      if (wz >= 0) {
        long long it = 0;
        while (ld_acquire(&c.done[wtype * N + wz]) < wcnt) {
          if (*(volatile int*)c.abort || ++it > c.spin_limit) {
            ok = 0;
            atomicOr(a.err, PIPE_ERR_TIMEOUT);
            atomicExch(c.abort, 1);
            break;
          }
          __nanosleep(64);
        }
      }
      s_go = ok;
    }
    __syncthreads();
    if (!s_go) break;
    const int zs = z % c.ring;
    SlabArgs<T> b = a;
    b.z0 = z - zs;
    if (type == 0)
      pipe_yinv<T, N>(b, tile, zs, smem);
    else if (type == 1)
      xrow_tile<T, N, MemCG>(b, zs * P::nX + tile, smem);  // inline: it needs every register
    else
      pipe_yfwd<T, N>(b, tile, zs, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&c.done[type * N + z], 1);
    }
  }
}

}  // namespace ns

#include "ns_slabcl.cuh"

namespace ns {

// ---- registry entry of one size ------------------------------------------------------
template <typename T>
struct K2Entry {
  int N = 0;
  void (*pencil)(PencilArgs<T>) = nullptr;   // any number of inputs / outputs
  void (*pencil1)(PencilArgs<T>) = nullptr;  // one input, one output
  void (*pencil1e)(PencilArgs<T>) = nullptr; // same, also storing the tile's energy sums
  void (*pencil1re)(PencilArgs<T>) = nullptr; // the energy-sum variant of the ROG_2 stage
  void (*pencil1r[2])(PencilArgs<T>) = {nullptr, nullptr};  // one in, one out: ROG_1, ROG_2
  void (*pencil2)(PencilArgs<T>) = nullptr;  // two inputs, two outputs
  void (*yinv)(SlabArgs<T>) = nullptr;
  void (*yfwd)(SlabArgs<T>) = nullptr;
  void (*xrow)(SlabArgs<T>) = nullptr;
  void (*slabpipe)(SlabArgs<T>, PipeCtl) = nullptr;  // null when the size has no pipeline
  int NTPIPE = 0;
  size_t smPIPE = 0;
  // the slab pass in thread-block clusters of CLS CTAs (null when the size has none), two
  // thread counts: variant v has NTCL[v] threads
  void (*slabcl[2])(CUtensorMap, cpx<T>*, const cpx<T>*, ClArgs) = {nullptr, nullptr};
  int CLS = 0, NTCL[2] = {0, 0}, CLKC = 0, CLPL = 1;
  size_t smCL = 0;
  int TX = 0, NTP = 0, TY = 0, NTY = 0, TYI = 0, NTYI = 0, RX = 0, NTX = 0;
  size_t smP1 = 0, smP4 = 0, smP5 = 0, smY = 0, smYI = 0, smX = 0;
  // the autotuner's compiled alternatives (K2Cfg variant 15: every family's other width);
  // has_alt false when the size has none
  struct Alt {
    void (*pencil1r[2])(PencilArgs<T>) = {nullptr, nullptr};
    void (*yinv)(SlabArgs<T>) = nullptr;
    void (*yfwd)(SlabArgs<T>) = nullptr;
    void (*xrow)(SlabArgs<T>) = nullptr;
    int TX = 0, NTP = 0, TY = 0, NTY = 0, TYI = 0, NTYI = 0, RX = 0, NTX = 0;
    size_t smP1 = 0, smY = 0, smYI = 0, smX = 0;
  } alt;
  void (*pencil1r64[2])(PencilArgs<T>) = {nullptr, nullptr};  // variant 16 (64 registers)
  bool has_alt = false;
};

// sizes with compiled alternatives: the FP32 grids of 128^3 and larger
template <typename T, int N>
__host__ __device__ constexpr bool k2_has_alt() { return sizeof(T) == 4 && N >= 128; }

template <typename T, int N>
K2Entry<T> make_k2_entry() {
  using C = K2Cfg<T, N>;
  K2Entry<T> e;
  e.N = N;
  e.pencil = k2_pencil<T, N, -1, -1>;
#ifndef NS_PENCIL_VARIANTS
#define NS_PENCIL_VARIANTS 1
#endif
  // NS_PENCIL_VARIANTS=0 routes every pencil pass through the generic kernel (comparisons)
  e.pencil1 = NS_PENCIL_VARIANTS ? k2_pencil<T, N, 1, 1> : e.pencil;
  e.pencil1e = NS_PENCIL_VARIANTS ? k2_pencil<T, N, 1, 1, true> : e.pencil;
#ifndef NS_PENCIL_MODE_VARIANTS
#define NS_PENCIL_MODE_VARIANTS 1
#endif
  e.pencil1r[0] = NS_PENCIL_MODE_VARIANTS ? k2_pencil<T, N, 1, 1, false, MODE_ROG_1> : e.pencil1;
  e.pencil1r[1] = NS_PENCIL_MODE_VARIANTS ? k2_pencil<T, N, 1, 1, false, MODE_ROG_2> : e.pencil1;
  e.pencil1re = NS_PENCIL_VARIANTS && NS_PENCIL_MODE_VARIANTS ? k2_pencil<T, N, 1, 1, true, MODE_ROG_2> : e.pencil1e;
  e.pencil2 = NS_PENCIL_VARIANTS ? k2_pencil<T, N, 2, 2> : e.pencil;
  e.yinv = k2_yinv<T, N>;
  e.yfwd = k2_yfwd<T, N>;
  e.xrow = k2_xrow<T, N>;
  if constexpr (ClCfg<T, N>::ok) {
    e.slabcl[0] = k2_slabcl<T, N, 384>;
    e.slabcl[1] = k2_slabcl<T, N, 768>;
    e.NTCL[0] = 384;
    e.NTCL[1] = 768;
    e.CLS = ClCfg<T, N>::CS;
    e.CLKC = ClCfg<T, N>::KC;
    e.CLPL = ClCfg<T, N>::PL;
    e.smCL = ClCfg<T, N>::smem;
  }
  if constexpr (PipeCfg<T, N>::ok) {
    e.slabpipe = k2_slabpipe<T, N>;
    e.NTPIPE = PipeCfg<T, N>::NT;
    e.smPIPE = PipeCfg<T, N>::smem;
  }
  e.TX = C::TX; e.NTP = C::NTP; e.TY = C::TY; e.NTY = C::NTY; e.RX = C::RX; e.NTX = C::NTX;
  e.TYI = C::TYI; e.NTYI = C::NTYI;
  e.smYI = (4 * (size_t)lf_rows<T, C::TYI>(N) * C::TYI + tw_elems(N)) * sizeof(cpx<T>);
  e.smP4 = (3 * (size_t)lf_rows<T, C::TX>(N) * C::TX + tw_elems(N)) * sizeof(cpx<T>);  // 3 tiles + twiddles
  e.smP1 = NS_PENCIL_STAGE_STATE ? (6 * (size_t)lf_rows<T, C::TX>(N) * C::TX + tw_elems(N)) * sizeof(cpx<T>) : e.smP4;
  e.smP5 = (4 * (size_t)lf_rows<T, C::TX>(N) * C::TX + tw_elems(N)) * sizeof(cpx<T>);  // 4 tiles + twiddles
  e.smY = ((size_t)lf_rows<T, C::TY>(N) * C::TY + tw_elems(N)) * sizeof(cpx<T>);
  e.smX = ((size_t)C::XELEMS + tw_elems(N)) * sizeof(cpx<T>);
  if constexpr (k2_has_alt<T, N>()) {
    using A = K2Cfg<T, N, 15>;
    e.has_alt = true;
    e.alt.pencil1r[0] = k2_pencil<T, N, 1, 1, false, MODE_ROG_1, 15>;
    e.alt.pencil1r[1] = k2_pencil<T, N, 1, 1, false, MODE_ROG_2, 15>;
    e.alt.yinv = k2_yinv<T, N, 15>;
    e.alt.yfwd = k2_yfwd<T, N, 15>;
    e.alt.xrow = k2_xrow<T, N, 15>;
    e.alt.TX = A::TX; e.alt.NTP = A::NTP; e.alt.TY = A::TY; e.alt.NTY = A::NTY;
    e.alt.TYI = A::TYI; e.alt.NTYI = A::NTYI; e.alt.RX = A::RX; e.alt.NTX = A::NTX;
    e.alt.smYI = (4 * (size_t)lf_rows<T, A::TYI>(N) * A::TYI + tw_elems(N)) * sizeof(cpx<T>);
    e.alt.smP1 = (3 * (size_t)lf_rows<T, A::TX>(N) * A::TX + tw_elems(N)) * sizeof(cpx<T>);
    e.alt.smY = ((size_t)lf_rows<T, A::TY>(N) * A::TY + tw_elems(N)) * sizeof(cpx<T>);
    e.alt.smX = ((size_t)A::XELEMS + tw_elems(N)) * sizeof(cpx<T>);
    e.pencil1r64[0] = k2_pencil<T, N, 1, 1, false, MODE_ROG_1, 16>;
    e.pencil1r64[1] = k2_pencil<T, N, 1, 1, false, MODE_ROG_2, 16>;
  }
  return e;
}

}  // namespace ns
