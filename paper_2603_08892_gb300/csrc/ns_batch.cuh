// ns_batch.cuh -- ensembles of independent simulations of uneven N in one persistent launch.
//
// No counterpart in the paper (its runs are single fields on CPU clusters); the members
// each run the RK2 phase-shift random (or approx) scheme of Sec. 4.2 exactly as a single
// context does, with the same kernels' tile bodies.
//
// Work list.  Every member m advances through the same sequence of passes:
//   prologue:  TAB (shift tables of step 0), INIT (pencil tiles: shifted state -> mixed)
//   per step:  TAB, YINV, XROW, YFWD, P1 (ROG_1), YINV, XROW, YFWD, P2 (ROG_2)
// A pass consists of tiles ("items"), taken gran tiles per ticket (the work-list granularity:
// the ticket, the wait and the completion fence are paid once per gran tiles).  Tickets are
// numbered step-major, then pass, then member, then tile group, and the CTAs of one persistent
// launch take them in that order from an atomic ticket counter.  Before running an item of member m, a CTA waits until done[m]
// (the member's count of finished items) covers every item of the member's earlier passes;
// an item only ever waits for items with smaller tickets, which running CTAs already hold,
// so the schedule cannot deadlock.  Each wait is bounded (spin_limit polls); on expiry the
// kernel records NS_ERR_TIMEOUT in a device flag, raises an abort flag that every other
// waiter also polls, and returns.  Data produced by other CTAs of the launch is read with
// L2-coherent loads (.cg), never through L1 or the read-only path.
//
// Grid schedule (gran = 0).  The same items without a work list: every pass of each size class
// is one ordinary grid launch (blockIdx.x the tile, blockIdx.y the member within the class)
// with the block shape and shared memory of that size alone, the classes one after another on
// the batch's stream (measured 2 % faster than one stream per class).  Stream order separates
// the passes, so nothing waits on the device.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ns_internal.h"
#include "ns_kernels2.cuh"

using namespace ns;

// (a named namespace: the grid schedule's kernels are compiled in translation units of their
// own and reached through launch_class_any)
namespace nsb {

constexpr int kPasses = 9;  // per step
enum { P_TAB = 0, P_Y1, P_X1, P_F1, P_P1, P_Y2, P_X2, P_F2, P_P2 };
constexpr int kSizes[] = {16, 32, 48, 64, 96, 128};
constexpr int kNumSizes = 6;
constexpr int kMaxMembers = 1024;
enum { BERR_TIMEOUT = 4 };

template <typename T>
struct BatchMem {
  int N, sz;
  PencilArgs<T> pa;  // pointers and stage constants; mode/inputs/outputs set per item
  SlabArgs<T> sa;
  cpx<T>* tab;            // [3][3N]: alpha_s, beta_s, alpha_{s+1}
  const double* shifts;   // [nsteps + 1][3] alpha of each step of this call
  double dx;
  int items[kPasses];     // items (tiles) of each pass
  int cum[kPasses + 1];   // items of the member before pass p within a step
  int pro_init;           // INIT items
};

struct BatchCtl {
  unsigned long long* next;
  int* done;
  int* err;
  int* abort;
  int nmem, nsteps;
  long long pro_total, step_total, total;
  long long pro_off[3];
  long long pass_off[kPasses + 1];
  const int* mem_off;      // [kPasses][nmem + 1]
  const int* pro_mem_off;  // [2][nmem + 1]
  long long spin_limit;
  long long stall;  // added to every per-step requirement (test hook)
  int gran;         // tiles per ticket
};

template <typename T>
struct BCfg {
  template <int N>
  static constexpr int nt() {
    using C = K2Cfg<T, N>;
    return cmax(cmax(C::NTP, C::NTYI), cmax(C::NTY, C::NTX));
  }
  template <int N>
  static constexpr size_t sm() {
    using C = K2Cfg<T, N>;
    const size_t cs = sizeof(cpx<T>);
    const size_t tw = (size_t)tw_elems(N);
    const size_t p = (3 * (size_t)lf_rows<T, C::TX>(N) * C::TX + tw) * cs;
    const size_t yi = (4 * (size_t)lf_rows<T, C::TYI>(N) * C::TYI + tw) * cs;  // 3 input slots + work
    const size_t yf = ((size_t)lf_rows<T, C::TY>(N) * C::TY + tw) * cs, x = ((size_t)C::XELEMS + tw) * cs;
    const size_t a = p > yi ? p : yi, b = yf > x ? yf : x;
    return a > b ? a : b;
  }
  static constexpr int NT = cmax(cmax(cmax(nt<16>(), nt<32>()), cmax(nt<48>(), nt<64>())),
                                 cmax(nt<96>(), nt<128>()));
  static constexpr size_t SM_a = sm<16>() > sm<32>() ? sm<16>() : sm<32>();
  static constexpr size_t SM_b = sm<48>() > sm<64>() ? sm<48>() : sm<64>();
  static constexpr size_t SM_c = sm<96>() > sm<128>() ? sm<96>() : sm<128>();
  static constexpr size_t SM_ab = SM_a > SM_b ? SM_a : SM_b;
  static constexpr size_t SM = SM_ab > SM_c ? SM_ab : SM_c;
};


// last index i with off[i] <= r  (off ascending, off[0] = 0, off[n] = total)
__device__ __forceinline__ int upper_member(const int* off, int n, int r) {
  int lo = 0, hi = n;  // answer in [0, n)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&off[mid]) <= r) lo = mid; else hi = mid;
  }
  return lo;
}

// shift tables exp(i k delta) (Sec. 4.2, Eq. shift_operator_3d) in FP64 of the member's step
// (slots alpha_s, beta_s = alpha_s + dx / 2, alpha_{s+1})
template <typename T, int N>
__device__ __forceinline__ void batch_tab(const BatchMem<T>& bm, int step, int nsteps) {
  for (int i = threadIdx.x; i < 9 * N; i += blockDim.x) {
    const int slot = i / (3 * N), rem = i % (3 * N), d = rem / N, k = rem % N;
    const int s = slot == 2 ? step + 1 : step;
    double delta = s <= nsteps ? bm.shifts[3 * s + d] : 0.0;
    if (slot == 1) delta += 0.5 * bm.dx;
    double sn, cs;
    sincos((double)kof(k, N) * delta, &sn, &cs);
    MemCG::st(&bm.tab[i], mk<T>((T)cs, (T)sn));
  }
}

// arguments of a pencil pass: INIT (pass < 0), P1 (ROG_1) or P2 (ROG_2)
template <typename T>
__device__ __forceinline__ PencilArgs<T> batch_pencil_args(const BatchMem<T>& bm, int pass, int step, int nsteps) {
  PencilArgs<T> a = bm.pa;
  const int NN = bm.N;
  const cpx<T>* ta = bm.tab;
  const cpx<T>* tb = bm.tab + 3 * NN;
  const cpx<T>* tc = bm.tab + 6 * NN;
  if (pass < 0) {
    a.mode = MODE_INIT;
    a.nF = 0;
    a.src = a.state;
    a.nOut = 1;
    a.osh[0] = ta;
  } else if (pass == P_P1) {
    a.mode = MODE_ROG_1;
    a.nF = 1;
    a.dsh[0] = ta;
    a.nOut = 1;
    a.osh[0] = tb;
  } else {
    a.mode = MODE_ROG_2;
    a.nF = 1;
    a.dsh[0] = tb;
    a.nOut = step + 1 < nsteps ? 1 : 0;
    a.osh[0] = tc;
  }
  return a;
}

template <typename T, int N>
__device__ __noinline__ void run_item(const BatchMem<T>& bm, int pass, int step, int nsteps,
                                      int tile, cpx<T>* smem) {
  using C = K2Cfg<T, N>;
  constexpr int M = N / 2;
  if (pass == P_TAB) {
    batch_tab<T, N>(bm, step, nsteps);
    return;
  }
  if (pass == P_Y1 || pass == P_Y2) {
    constexpr int ntx = M / C::TYI;
    yinv_tile<T, N, MemCG>(bm.sa, tile % ntx, tile / ntx, smem);
    return;
  }
  if (pass == P_X1 || pass == P_X2) {
    xrow_tile<T, N, MemCG>(bm.sa, tile, smem);
    return;
  }
  if (pass == P_F1 || pass == P_F2) {
    constexpr int ntx = M / C::TY;
    yfwd_tile<T, N, MemCG>(bm.sa, tile % ntx, tile / ntx, smem);
    return;
  }
  // pencil passes: INIT (pass < 0), P1, P2
  pencil_tile<T, N, MemCG>(batch_pencil_args(bm, pass, step, nsteps), tile, smem);
}

template <typename T>
__global__ void __launch_bounds__(BCfg<T>::NT) k_batch(BatchCtl c, const BatchMem<T>* __restrict__ mems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* smem = reinterpret_cast<cpx<T>*>(smem_raw);
  __shared__ long long s_ticket;
  __shared__ int s_go;
  for (;;) {
    if (threadIdx.x == 0) s_ticket = (long long)atomicAdd(c.next, 1ull);
    __syncthreads();
    const long long tk = s_ticket;
    if (tk >= c.total) break;
    int pass, m, tile, step, ntile;  // tiles [tile, tile + ntile) of the member's pass
    long long need;
    if (tk < c.pro_total) {
      const int pp = tk < c.pro_off[1] ? 0 : 1;
      const int r = (int)(tk - c.pro_off[pp]);
      const int* off = c.pro_mem_off + pp * (c.nmem + 1);
      m = upper_member(off, c.nmem, r);
      const int items = pp == 0 ? 1 : mems[m].pro_init;
      tile = (r - __ldg(&off[m])) * c.gran;
      ntile = min(c.gran, items - tile);
      pass = pp == 0 ? P_TAB : -1;
      step = 0;
      need = pp == 0 ? 0 : 1;
    } else {
      const long long t2 = tk - c.pro_total;
      step = (int)(t2 / c.step_total);
      const long long r = t2 % c.step_total;
      int p = 0;
      while (p < kPasses - 1 && r >= c.pass_off[p + 1]) ++p;
      const int r2 = (int)(r - c.pass_off[p]);
      const int* off = c.mem_off + p * (c.nmem + 1);
      m = upper_member(off, c.nmem, r2);
      const BatchMem<T>& b0 = mems[m];
      tile = (r2 - __ldg(&off[m])) * c.gran;
      ntile = min(c.gran, b0.items[p] - tile);
      pass = p;
      need = 1 + (long long)b0.pro_init + (long long)step * b0.cum[kPasses] + b0.cum[p] + c.stall;
    }
    if (threadIdx.x == 0) {
      int ok = 1;
      if (need > 0) {
        long long it = 0;
        while (ld_acquire(&c.done[m]) < need) {
          if (*(volatile int*)c.abort || ++it > c.spin_limit) {
            ok = 0;
            atomicOr(c.err, BERR_TIMEOUT);
            atomicExch(c.abort, 1);
            break;
          }
          __nanosleep(100);
        }
      }
      s_go = ok;
    }
    __syncthreads();
    if (!s_go) break;
    const BatchMem<T>& bm = mems[m];
    for (int q = 0; q < ntile; ++q) {
      if (q > 0) __syncthreads();  // the previous tile is done with the shared memory
      switch (bm.sz) {
        case 0: run_item<T, 16>(bm, pass, step, c.nsteps, tile + q, smem); break;
        case 1: run_item<T, 32>(bm, pass, step, c.nsteps, tile + q, smem); break;
        case 2: run_item<T, 48>(bm, pass, step, c.nsteps, tile + q, smem); break;
        case 3: run_item<T, 64>(bm, pass, step, c.nsteps, tile + q, smem); break;
        case 4: run_item<T, 96>(bm, pass, step, c.nsteps, tile + q, smem); break;
        default: run_item<T, 128>(bm, pass, step, c.nsteps, tile + q, smem); break;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&c.done[m], ntile);
    }
  }
}

#ifdef NS_BATCH_GRID_DEFS
// The grid schedule's kernels, one per kind of pass: tile blockIdx.x of member
// cls[blockIdx.y] (a member of size N), each with only its own tile body and the block shape
// of the single-context kernel of that body (the same arithmetic as the persistent kernel's
// items, so every schedule gives the same bits).
template <typename T, int N>
__global__ void __launch_bounds__(128) k_bgrid_tab(const BatchMem<T>* __restrict__ mems, const int* __restrict__ cls,
                                                   int step, int nsteps) {
  batch_tab<T, N>(mems[__ldg(&cls[blockIdx.y])], step, nsteps);
}
template <typename T, int N>
__global__ void __launch_bounds__(K2Cfg<T, N>::NTP) k_bgrid_pencil(const BatchMem<T>* __restrict__ mems,
                                                                  const int* __restrict__ cls, int pass, int step,
                                                                  int nsteps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const BatchMem<T>& bm = mems[__ldg(&cls[blockIdx.y])];
  pencil_tile<T, N, MemNC>(batch_pencil_args(bm, pass, step, nsteps), (int)blockIdx.x,
                           reinterpret_cast<cpx<T>*>(smem_raw));
}
template <typename T, int N>
__global__ void __launch_bounds__(K2Cfg<T, N>::NTYI) k_bgrid_yinv(const BatchMem<T>* __restrict__ mems,
                                                                 const int* __restrict__ cls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ntx = (N / 2) / K2Cfg<T, N>::TYI;
  yinv_tile<T, N, MemNC>(mems[__ldg(&cls[blockIdx.y])].sa, (int)blockIdx.x % ntx, (int)blockIdx.x / ntx,
                         reinterpret_cast<cpx<T>*>(smem_raw));
}
template <typename T, int N>
__global__ void __launch_bounds__(K2Cfg<T, N>::NTX, K2Cfg<T, N>::MINB_X) k_bgrid_xrow(
    const BatchMem<T>* __restrict__ mems, const int* __restrict__ cls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xrow_tile<T, N, MemNC>(mems[__ldg(&cls[blockIdx.y])].sa, (int)blockIdx.x, reinterpret_cast<cpx<T>*>(smem_raw));
}
template <typename T, int N>
__global__ void __launch_bounds__(K2Cfg<T, N>::NTY, 2) k_bgrid_yfwd(const BatchMem<T>* __restrict__ mems,
                                                                   const int* __restrict__ cls) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int ntx = (N / 2) / K2Cfg<T, N>::TY;
  yfwd_tile<T, N, MemNC>(mems[__ldg(&cls[blockIdx.y])].sa, (int)blockIdx.x % ntx, (int)blockIdx.x / ntx,
                         reinterpret_cast<cpx<T>*>(smem_raw));
}

#endif  // NS_BATCH_GRID_DEFS

template <typename T, int N>
void member_items(int* items, int* pro_init) {
  using C = K2Cfg<T, N>;
  constexpr int M = N / 2;
  const int pen = (M / C::TX) * N, yi = (M / C::TYI) * N, yf = (M / C::TY) * N;
  const int xr = (N * N + C::RX - 1) / C::RX;
  const int v[kPasses] = {1, yi, xr, yf, pen, yi, xr, yf, pen};
  for (int p = 0; p < kPasses; ++p) items[p] = v[p];
  *pro_init = pen;
}

inline int size_index(int N) {
  for (int i = 0; i < kNumSizes; ++i)
    if (kSizes[i] == N) return i;
  return -1;
}

template <typename T>
void items_for(int N, int* items, int* pro) {
  switch (N) {
    case 16: member_items<T, 16>(items, pro); break;
    case 32: member_items<T, 32>(items, pro); break;
    case 48: member_items<T, 48>(items, pro); break;
    case 64: member_items<T, 64>(items, pro); break;
    case 96: member_items<T, 96>(items, pro); break;
    default: member_items<T, 128>(items, pro); break;
  }
}

// every pass of nsteps steps (and the prologue) of the nc members cls[0 .. nc) of the size
// class sz (kSizes[sz]) on stream cs, as grid launches; returns the first launch error.
// Defined in the grid schedule's translation units (ns_batch_grid_f32.cu, ns_batch_grid_f64.cu).
template <typename T>
cudaError_t launch_class_any(int sz, const BatchMem<T>* dm, const int* cls, int nc, int nsteps, cudaStream_t cs);

#ifdef NS_BATCH_GRID_DEFS
// every pass of nsteps steps (and the prologue) of the nc members cls[0 .. nc) of size N on
// stream cs; returns the first launch error
template <typename T, int N>
cudaError_t launch_class(const BatchMem<T>* dm, const int* cls, int nc, int nsteps, cudaStream_t cs) {
  using C = K2Cfg<T, N>;
  constexpr int M = N / 2;
  const size_t cz = sizeof(cpx<T>), tw = (size_t)tw_elems(N);
  const size_t smP = (3 * (size_t)lf_rows<T, C::TX>(N) * C::TX + tw) * cz;
  const size_t smYI = (4 * (size_t)lf_rows<T, C::TYI>(N) * C::TYI + tw) * cz;
  const size_t smY = ((size_t)lf_rows<T, C::TY>(N) * C::TY + tw) * cz;
  const size_t smX = ((size_t)C::XELEMS + tw) * cz;
  static bool attr = false;  // (per template instance: the opt-in sizes set before the first launch)
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_bgrid_pencil<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smP);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bgrid_yinv<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smYI);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bgrid_yfwd<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smY);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_bgrid_xrow<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smX);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int pen = (M / C::TX) * N, yi = (M / C::TYI) * N, yf = (M / C::TY) * N;
  const int xr = (N * N + C::RX - 1) / C::RX;
  k_bgrid_tab<T, N><<<dim3(1, nc), 128, 0, cs>>>(dm, cls, 0, nsteps);
  k_bgrid_pencil<T, N><<<dim3(pen, nc), C::NTP, smP, cs>>>(dm, cls, -1, 0, nsteps);
  for (int s = 0; s < nsteps; ++s) {
    k_bgrid_tab<T, N><<<dim3(1, nc), 128, 0, cs>>>(dm, cls, s, nsteps);
    for (int h = 0; h < 2; ++h) {  // the two stages: slab pass, then the pencil pass P1 / P2
      k_bgrid_yinv<T, N><<<dim3(yi, nc), C::NTYI, smYI, cs>>>(dm, cls);
      k_bgrid_xrow<T, N><<<dim3(xr, nc), C::NTX, smX, cs>>>(dm, cls);
      k_bgrid_yfwd<T, N><<<dim3(yf, nc), C::NTY, smY, cs>>>(dm, cls);
      k_bgrid_pencil<T, N><<<dim3(pen, nc), C::NTP, smP, cs>>>(dm, cls, h == 0 ? P_P1 : P_P2, s, nsteps);
    }
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_class_any(int sz, const BatchMem<T>* dm, const int* cls, int nc, int nsteps, cudaStream_t cs) {
  switch (sz) {
    case 0: return launch_class<T, 16>(dm, cls, nc, nsteps, cs);
    case 1: return launch_class<T, 32>(dm, cls, nc, nsteps, cs);
    case 2: return launch_class<T, 48>(dm, cls, nc, nsteps, cs);
    case 3: return launch_class<T, 64>(dm, cls, nc, nsteps, cs);
    case 4: return launch_class<T, 96>(dm, cls, nc, nsteps, cs);
    default: return launch_class<T, 128>(dm, cls, nc, nsteps, cs);
  }
}

#endif  // NS_BATCH_GRID_DEFS

inline uint64_t smix(uint64_t s, uint64_t n) {
  uint64_t z = s + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct ns_batch {
  int count = 0, precision = NS_FP32, scheme = NS_RK2_PS_RANDOM;
  std::vector<ns_ctx*> mem;
  cudaStream_t st = nullptr;
  std::string err;
  // device work-list state
  void* d_mems = nullptr;
  int* d_off = nullptr;
  double* d_shifts = nullptr;
  size_t shifts_cap = 0;
  unsigned long long* d_next = nullptr;
  int* d_done = nullptr;
  int* d_flags = nullptr;  // err, abort
  void* d_tab = nullptr;
  size_t tab_bytes = 0;
  bool own_stream = false;
  cudaGraphExec_t gexec = nullptr;
  int g_nsteps = -1, g_grid = -1, g_stall = -1;
  long long g_spin = -1;
  long long spin_limit = 2000000;
  int stall = 0;
  int grid = 0;
  int g_gran = -1;
  // work-list granularity (tiles per ticket) and CTAs per SM (0: as many as fit), chosen by
  // the tuner at the first step (or forced by ns_batch_set_schedule / NS_BATCH_SCHEDULE)
  int gran = 1, per_sm_req = 0;
  bool tuned = false;
  // grid schedule (gran 0): member indices grouped by size class
  int* d_cls = nullptr;
};

namespace nsb {

template <typename T>
int batch_step_t(ns_batch* b, const double* dt, int nsteps) {
  const int n = b->count;
  std::vector<BatchMem<T>> hm(n);
  std::vector<int> off_pass(kPasses * (n + 1)), off_pro(2 * (n + 1));
  // shifts of every member for steps 0..nsteps of this call: [m][nsteps+1][3]
  const size_t per = (size_t)(nsteps + 1) * 3;
  std::vector<double> sh((size_t)n * per);
  if ((size_t)n * per > b->shifts_cap) {
    cudaFree(b->d_shifts);
    b->d_shifts = nullptr;
    if (cudaMalloc(&b->d_shifts, (size_t)n * per * sizeof(double)) != cudaSuccess) return NS_ERR_OOM;
    b->shifts_cap = (size_t)n * per;
  }
  for (int m = 0; m < n; ++m) {
    NsCtxBuffers cb;
    int rc = ns_ctx_buffers(b->mem[m], dt[m], &cb);
    if (rc != NS_OK) return rc;
    BatchMem<T>& bm = hm[m];
    memset(&bm, 0, sizeof(bm));
    bm.N = cb.N;
    bm.sz = size_index(cb.N);
    bm.dx = 2.0 * M_PI / cb.N;
    const int N = cb.N, M = N / 2;
    PencilArgs<T>& a = bm.pa;
    a.N = N; a.M = M; a.tw = (const cpx<T>*)cb.tw; a.dt = (T)dt[m]; a.ifac = (const T*)cb.ifac;
    a.state = (cpx<T>*)cb.state; a.acc = nullptr; a.trunc = cb.truncation; a.K2max = cb.K2max;
    a.Kimax = cb.Kimax; a.err = (int*)cb.err; a.wF[0] = (T)(1.0 / ((double)N * N * N));
    a.F[0] = (const cpx<T>*)cb.Ft; a.out[0] = (cpx<T>*)cb.mixed;
    SlabArgs<T>& s = bm.sa;
    s.N = N; s.M = M; s.z0 = 0; s.G = N; s.tw = (const cpx<T>*)cb.tw; s.mixed = (const cpx<T>*)cb.mixed;
    s.scr = (cpx<T>*)cb.scr; s.Ft = (cpx<T>*)cb.Ft; s.xmode = XMODE_NONLINEAR; s.err = (int*)cb.err;
    if (cb.G < N) return NS_ERR_INTERNAL;
    items_for<T>(N, bm.items, &bm.pro_init);
    bm.cum[0] = 0;
    for (int p = 0; p < kPasses; ++p) bm.cum[p + 1] = bm.cum[p] + bm.items[p];
    for (int s2 = 0; s2 <= nsteps; ++s2)
      for (int i = 0; i < 3; ++i) {
        double d = 0.0;
        if (b->scheme == NS_RK2_PS_RANDOM)
          d = bm.dx * ((double)(smix(cb.seed, (uint64_t)(3 * (cb.step + s2) + i)) >> 11) *
                       (1.0 / 9007199254740992.0));
        sh[(size_t)m * per + 3 * s2 + i] = d;
      }
    bm.shifts = b->d_shifts + (size_t)m * per;
  }
  // shift tables: one [3][3N] slot per member
  size_t tab_elems = 0;
  for (int m = 0; m < n; ++m) {
    hm[m].tab = nullptr;
    tab_elems += 9 * (size_t)hm[m].N;
  }
  if (tab_elems * sizeof(cpx<T>) > b->tab_bytes) {
    cudaFree(b->d_tab);
    b->d_tab = nullptr;
    if (cudaMalloc(&b->d_tab, tab_elems * sizeof(cpx<T>)) != cudaSuccess) return NS_ERR_OOM;
    b->tab_bytes = tab_elems * sizeof(cpx<T>);
  }
  {
    size_t o = 0;
    for (int m = 0; m < n; ++m) {
      hm[m].tab = (cpx<T>*)b->d_tab + o;
      o += 9 * (size_t)hm[m].N;
    }
  }
  // offsets: pass-major, member, tile
  BatchCtl c;
  memset(&c, 0, sizeof(c));
  c.nmem = n;
  c.nsteps = nsteps;
  long long acc = 0;
  c.pro_off[0] = 0;
  const int gran = b->gran > 0 ? b->gran : 1;
  auto tickets = [&](int items) { return (items + gran - 1) / gran; };
  for (int pp = 0; pp < 2; ++pp) {
    int o = 0;
    for (int m = 0; m < n; ++m) {
      off_pro[pp * (n + 1) + m] = o;
      o += pp == 0 ? 1 : tickets(hm[m].pro_init);
    }
    off_pro[pp * (n + 1) + n] = o;
    acc += o;
    c.pro_off[pp + 1] = acc;
  }
  c.pro_total = acc;
  long long sacc = 0;
  for (int p = 0; p < kPasses; ++p) {
    c.pass_off[p] = sacc;
    int o = 0;
    for (int m = 0; m < n; ++m) {
      off_pass[p * (n + 1) + m] = o;
      o += tickets(hm[m].items[p]);
    }
    off_pass[p * (n + 1) + n] = o;
    sacc += o;
  }
  c.pass_off[kPasses] = sacc;
  c.step_total = sacc;
  c.total = c.pro_total + (long long)nsteps * c.step_total;
  c.spin_limit = b->spin_limit;
  c.stall = b->stall ? (1ll << 40) : 0;
  c.gran = gran;

  cudaStream_t st = b->st;
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess) {
      b->err = cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  if (!chk(cudaMemcpyAsync(b->d_shifts, sh.data(), sh.size() * sizeof(double), cudaMemcpyHostToDevice, st)) ||
      !chk(cudaMemcpyAsync(b->d_mems, hm.data(), n * sizeof(BatchMem<T>), cudaMemcpyHostToDevice, st)) ||
      !chk(cudaMemcpyAsync(b->d_off, off_pass.data(), off_pass.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
      !chk(cudaMemcpyAsync(b->d_off + kPasses * (kMaxMembers + 1), off_pro.data(), off_pro.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st))) {
    return NS_ERR_CUDA;
  }
  if (b->gran == 0) {  // grid schedule
    std::vector<int> cls;
    int start[kNumSizes + 1];
    for (int z = 0; z < kNumSizes; ++z) {
      start[z] = (int)cls.size();
      for (int m = 0; m < n; ++m)
        if (hm[m].sz == z) cls.push_back(m);
    }
    start[kNumSizes] = (int)cls.size();
    if (!b->d_cls && !chk(cudaMalloc(&b->d_cls, kMaxMembers * sizeof(int)))) return NS_ERR_OOM;
    if (!chk(cudaMemcpyAsync(b->d_cls, cls.data(), cls.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
        !chk(cudaMemsetAsync(b->d_flags, 0, 2 * sizeof(int), st)))
      return NS_ERR_CUDA;
    const BatchMem<T>* dmg = (const BatchMem<T>*)b->d_mems;
    for (int z = kNumSizes - 1; z >= 0; --z) {  // the largest class first
      const int nc = start[z + 1] - start[z];
      if (nc > 0 && !chk(launch_class_any<T>(z, dmg, b->d_cls + start[z], nc, nsteps, st))) return NS_ERR_CUDA;
    }
    b->grid = 0;
    int flags[2] = {0, 0};
    if (!chk(cudaMemcpyAsync(flags, b->d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !chk(cudaStreamSynchronize(st)))
      return NS_ERR_CUDA;
    for (int m = 0; m < n; ++m) ns_ctx_advance(b->mem[m], dt[m], nsteps);
    return NS_OK;
  }
  c.next = b->d_next;
  c.done = b->d_done;
  c.err = b->d_flags;
  c.abort = b->d_flags + 1;
  c.mem_off = b->d_off;
  c.pro_mem_off = b->d_off + kPasses * (kMaxMembers + 1);
  const size_t smem = BCfg<T>::SM;
  if (!chk(cudaFuncSetAttribute(k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return NS_ERR_CUDA;
  int per_sm = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<T>, BCfg<T>::NT, smem);
  if (per_sm < 1) per_sm = 1;
  if (b->per_sm_req > 0 && b->per_sm_req < per_sm) per_sm = b->per_sm_req;
  const int grid = nsm * per_sm;
  b->grid = grid;
  // the launch and its counter resets are captured in a CUDA graph once per work-list
  // shape (nsteps); per-call data lives in device buffers the kernel reads at run time
  const BatchMem<T>* dm = (const BatchMem<T>*)b->d_mems;
  bool ok = true;
  if (b->gexec == nullptr || b->g_nsteps != nsteps || b->g_grid != grid ||
      b->g_spin != b->spin_limit || b->g_stall != b->stall || b->g_gran != gran) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    cudaGraph_t g;
    ok = chk(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    if (ok) {
      cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), st);
      cudaMemsetAsync(b->d_done, 0, n * sizeof(int), st);
      cudaMemsetAsync(b->d_flags, 0, 2 * sizeof(int), st);
      k_batch<T><<<grid, BCfg<T>::NT, smem, st>>>(c, dm);
      ok = chk(cudaStreamEndCapture(st, &g));
    }
    if (ok) {
      ok = chk(cudaGraphInstantiate(&b->gexec, g, 0));
      cudaGraphDestroy(g);
    }
    b->g_nsteps = nsteps;
    b->g_grid = grid;
    b->g_spin = b->spin_limit;
    b->g_stall = b->stall;
    b->g_gran = gran;
  }
  if (ok) ok = chk(cudaGraphLaunch(b->gexec, st));
  int flags[2] = {0, 0};
  if (ok) ok = chk(cudaMemcpyAsync(flags, b->d_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (ok) ok = chk(cudaStreamSynchronize(st));
  if (!ok) return NS_ERR_CUDA;
  if (flags[0] & BERR_TIMEOUT) {
    b->err = "a bounded wait of the persistent kernel expired";
    return NS_ERR_TIMEOUT;
  }
  for (int m = 0; m < n; ++m) ns_ctx_advance(b->mem[m], dt[m], nsteps);
  return NS_OK;
}

}  // namespace

