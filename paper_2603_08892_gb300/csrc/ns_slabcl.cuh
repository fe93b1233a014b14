// ns_slabcl.cuh -- the slab pass of one z-plane in a thread-block cluster, on chip.
//
// Same arithmetic as k2_yinv + k2_xrow + k2_yfwd (the slab pass of Sec. 3.1's pseudo-spectral
// product, with u x omega formed in registers between the x transforms), but the plane's
// intermediate fields never leave the cluster: CS CTAs (one per SM) share one plane.
//
//   phase A  CTA r owns the KC = M/CS columns kx0 = r KC ...: the 5 mixed fields of its columns
//            arrive by TMA (5 boxes of N x KC), the 6 spectral-in-xy fields (u, omega = i k x u)
//            are formed and transformed in y (inverse), and stay in the CTA's shared memory A
//            as [y][6][KC];
//   phase B  CTA r owns the RC = N/CS rows y0 = r RC ...: it gathers the 6 fields of its rows
//            from the A of every CTA of the cluster (distributed shared memory), packs two
//            real rows per complex line, runs the inverse x transforms, forms u x omega, runs
//            the forward x transforms and stores the 3 products of each (row, kx) straight
//            into the A of the CTA owning that kx ([y][3][KC], the first half of A);
//   phase C  CTA r transforms its 3 product columns in y (forward) and writes them to Ft.
//
// Three cluster barriers per plane order the exchanges: after phase A (every A complete),
// between the gathers and the product stores (nobody reads A any more), and after the
// stores (every product has arrived).  Each cluster walks the planes z = c, c + ncl, ...;
// the next plane's TMA load is issued as soon as the x-line tile (its landing area) is free,
// so it overlaps phase C.  HBM traffic per plane: the 5 mixed fields read once, the 3
// products written once (the 8C model of the pass).  The TMA wait is bounded: on timeout
// the kernel records CL_ERR_TIMEOUT and keeps going through every barrier (no CTA leaves the
// cluster's barrier sequence early), so the launch always ends.
//
// Included by ns_kernels2.cuh (it uses its tiles, accessors and block_max3).
#pragma once

#include <cuda.h>

namespace ns {

constexpr int CL_ERR_TIMEOUT = 0x200;

// Cluster size, tile widths and shared memory of the cluster slab pass of size N (ok = false:
// the size has no cluster pass; the plane does not fit the distributed shared memory).
template <typename T, int N, int NT_ = 384>
struct ClCfg {
  static constexpr int M = N / 2;
  static constexpr int CS_ = (N == 256 && sizeof(T) == 4) ? 16 : (N == 128 ? 8 : 0);
  static constexpr int CS = CS_ > 0 ? CS_ : 1;
  static constexpr int KC = M / CS;   // kx columns per CTA (y passes)
  static constexpr int RC = N / CS;   // y rows per CTA (x rows)
  static constexpr int NLA = 6 * KC;  // lines of the y-inverse
  static constexpr int NLB = 3 * RC;  // x lines, inverse
  static constexpr int RCh = RC / 2;
  static constexpr int NLF = RC + RCh;  // x lines, forward
  static constexpr int NLC = 3 * KC;    // lines of the y-forward
  static constexpr int PL = 2;          // planes per cluster (straight-line code)
  static constexpr int R = sizeof(T) == 4 ? 16 : 8;  // radix cap of the butterflies
  static constexpr int NT = NT_;  // threads: 384 (2 butterflies each) or 768 (1 each)
  static constexpr int EA = N * NLA;                   // A: [y][6][KC]
  static constexpr int FS = N * KC;                    // one staged field [ky][KC]
  static constexpr int EB = WorkTile<T, N, NLB, false>::elems() > 5 * FS ? WorkTile<T, N, NLB, false>::elems() : 5 * FS;
  static constexpr int ETW = tw_elems(N) + 1;          // (+1: 16-byte alignment of the mbarrier)
  static constexpr size_t smem = (size_t)(EA + EB + ETW) * sizeof(cpx<T>) + 32;  // + mbarrier, zero word
  static constexpr bool ok = CS_ > 0 && M % CS == 0 && N % CS == 0 && RC % 2 == 0 && N % PL == 0 &&
                             (KC * sizeof(cpx<T>)) % 16 == 0 && (FS * sizeof(cpx<T>)) % 128 == 0 &&
                             (EA * sizeof(cpx<T>)) % 128 == 0 && smem <= 227 * 1024;
};

// ---- cluster, distributed shared memory, mbarrier and TMA primitives (inline PTX) ----------
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// the address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cl_map(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// two complex FP32 values (or one FP64) from / to a shared-memory address of the cluster
__device__ __forceinline__ void cl_ld16(unsigned a, cpx<float>* v) {
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v[0].x), "=f"(v[0].y), "=f"(v[1].x), "=f"(v[1].y) : "r"(a) : "memory");
}
__device__ __forceinline__ void cl_ld16(unsigned a, cpx<double>* v) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v[0].x), "=d"(v[0].y) : "r"(a) : "memory");
}
__device__ __forceinline__ void cl_st16(unsigned a, const cpx<float>* v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};"
               :: "r"(a), "f"(v[0].x), "f"(v[0].y), "f"(v[1].x), "f"(v[1].y) : "memory");
}
__device__ __forceinline__ void cl_st16(unsigned a, const cpx<double>* v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" :: "r"(a), "d"(v[0].x), "d"(v[0].y) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(a), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 3D tiled TMA load of one box into this CTA's shared memory, completing on mbarrier `bar`
__device__ __forceinline__ void tma_load3(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2,
                                          unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      :: "r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Tile of the x lines (WorkTile layout): see xrow_tile for the packing of two real rows per line.
// Output of the last forward-y stage: line = f KC + col of plane z, straight to Ft.
template <typename T, int N, int KC>
struct ClFtOut {
  cpx<T>* Ft;
  int z, kx0;
  __device__ __forceinline__ void put(int line, int e, cpx<T> v) const {
    const int f = line / KC, col = line % KC;
    Ft[(((size_t)f * N + z) * N + e) * (N / 2) + kx0 + col] = v;
  }
};

// The thread index as a fresh value for each phase of a plane: threadIdx.x plus a shared
// word that holds 0, read with a volatile load, so that neither the compiler nor the
// assembler can treat the result as invariant.  The phases' index arithmetic (transforms,
// gathers, stores) all derives from it; from threadIdx.x it would be shared between phases
// and across planes and kept in registers throughout (register spills).
__device__ __forceinline__ int cl_tid(const int* zero) {
  return (int)threadIdx.x + *reinterpret_cast<const volatile int*>(zero);
}

struct ClArgs {
  int* err;    // device flag (CL_ERR_TIMEOUT)
  void* umax;  // or null: max |u_i| of the rows (as SlabArgs::umax)
  long long spin_limit;  // polls of the TMA wait before it gives up
};

// Shared memory of a CTA: A [y][6][KC] (then the products [y][3][KC]), B the x-line tile
// (first the 5 staged mixed fields [f][ky][KC]), the twiddles, the mbarrier of the TMA loads.
template <typename T, int N, int NT>
struct ClSmem {
  cpx<T>* A;
  cpx<T>* B;
  cpx<T>* tws;
  unsigned bar;
  int* zero;  // a shared word holding 0 (see cl_tid)
  __device__ __forceinline__ ClSmem() {
    using C = ClCfg<T, N, NT>;
    extern __shared__ __align__(128) unsigned char cl_smem[];
    A = reinterpret_cast<cpx<T>*>(cl_smem);
    B = A + C::EA;
    tws = B + C::EB;
    unsigned long long* mb = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(tws + tw_elems(N)) + 15) & ~uintptr_t(15));
    bar = smem_addr(mb);
    zero = reinterpret_cast<int*>(mb + 1);
  }
};

// the 5 mixed-field boxes of plane z (this CTA's columns) into B, completing on the mbarrier
template <typename T, int N, int NT>
__device__ __forceinline__ void cl_issue(const ClSmem<T, N, NT>& sm, const CUtensorMap* map, int kx0, int z) {
  using C = ClCfg<T, N, NT>;
  mbar_expect_tx(sm.bar, 5u * C::FS * (unsigned)sizeof(cpx<T>));
  const unsigned aB = smem_addr(sm.B);
  for (int f = 0; f < 5; ++f)
    tma_load3(aB + f * C::FS * (unsigned)sizeof(cpx<T>), map, 2 * kx0, 0, f * N + z, sm.bar);
}

// One plane z.  Not inlined into the plane loop: every phase's index arithmetic is the same
// for every plane, and inlined the compiler hoists all of it out of the loop and keeps it in
// registers across every phase (spills); as a call, the plane is allocated like straight-line
// code.  The next plane's load is issued by thread 0 when next >= 0.
template <typename T, int N, int NT>
__device__ __forceinline__ void cl_plane(const CUtensorMap* map, cpx<T>* __restrict__ Ft, int z, int next,
                                      unsigned parity, T* mx, ClArgs a) {
  using C = ClCfg<T, N, NT>;
  constexpr int M = N / 2, KC = C::KC, RC = C::RC, RCh = C::RCh, FS = C::FS;
  const ClSmem<T, N, NT> sm;
  cpx<T>* A = sm.A;
  cpx<T>* B = sm.B;
  const cpx<T>* tws = sm.tws;
  const unsigned rank = cl_rank();
  const int kx0 = (int)rank * KC, y0 = (int)rank * RC;
  const unsigned aA = smem_addr(A);
  const bool act = threadIdx.x < NT;
  const WorkTile<T, N, C::NLB, false> L{B};

  // ---- phase A: staged mixed fields -> 6 spectral-in-xy fields -> inverse y, in A ---------
  {
    long long it = 0;  // every thread waits for the landed boxes (bounded)
    while (!mbar_try_wait(sm.bar, parity)) {
      if (++it > a.spin_limit) {
        atomicOr(a.err, CL_ERR_TIMEOUT);
        break;
      }
    }
  }
  for (int i = cl_tid(sm.zero); act && i < N * KC; i += NT) {
    const int ky = i / KC, col = i % KC;
    const T fkx = (T)(kx0 + col), fky = (T)kof(ky, N);
    const cpx<T> m0 = B[i], m1 = B[FS + i], m2 = B[2 * FS + i], m3 = B[3 * FS + i], m4 = B[4 * FS + i];
    cpx<T>* o = A + ky * C::NLA + col;
    o[0] = m0;                                      // u_x
    o[KC] = m1;                                     // u_y
    o[2 * KC] = m2;                                 // u_z
    o[3 * KC] = mul_si(m2, fky) - m4;               // omega_x = i ky u_z - d_z u_y
    o[4 * KC] = m3 - mul_si(m2, fkx);               // omega_y = d_z u_x - i kx u_z
    o[5 * KC] = mul_si(m1, fkx) - mul_si(m0, fky);  // omega_z = i kx u_y - i ky u_x
  }
  __syncthreads();
  cfft_ip_tid<T, N, 1, C::NLA, NT, true, 1, true, C::R>(SmTile<T, C::NLA>{A}, WorkTile<T, N, C::NLA, true>{A},
                                                      WorkTile<T, N, C::NLA, true>{A}, tws, cl_tid(sm.zero));
  __syncthreads();
  cl_arrive();  // (1) every A of the cluster is complete
  cl_wait();

  // ---- phase B: gather the rows, x transforms, u x omega, products to their owners ---------
  // item (p, row, kp): fields 2p, 2p+1 at (y0 + row, k = VEC kp ...) from the owner of k;
  // line p RC + row gets Z[k] = A + iB and Z[N - k] = conj(A) + i conj(B)
  constexpr int VEC = 16 / (int)sizeof(cpx<T>);  // complex values per 16-byte access
  {
    // every remote load of the thread is issued before the first write (one round trip)
    constexpr int NI = 3 * RC * (M / VEC), KI = (NI + NT - 1) / NT;
    const int t0 = cl_tid(sm.zero);
    cpx<T> va[KI][2], vb[KI][2];
#pragma unroll
    for (int c = 0; c < KI; ++c) {
      const int i = t0 + c * NT;
      if (act && (NI % NT == 0 || i < NI)) {
        const int kp = i % (M / VEC), row = (i / (M / VEC)) % RC, p = i / (RC * (M / VEC));
        const int k = kp * VEC, s = k / KC, col = k % KC;
        const unsigned off = (unsigned)(((y0 + row) * C::NLA + 2 * p * KC + col) * sizeof(cpx<T>));
        cl_ld16(cl_map(aA + off, (unsigned)s), va[c]);
        cl_ld16(cl_map(aA + off + KC * (unsigned)sizeof(cpx<T>), (unsigned)s), vb[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < KI; ++c) {
      const int i = t0 + c * NT;
      if (act && (NI % NT == 0 || i < NI)) {
        const int kp = i % (M / VEC), row = (i / (M / VEC)) % RC, p = i / (RC * (M / VEC));
        const int k = kp * VEC, line = p * RC + row;
#pragma unroll
        for (int h = 0; h < VEC; ++h) {
          const int kk = k + h;
          const cpx<T> Av = va[c][h], Bv = vb[c][h];
          if (kk == 0) {
            L.put(line, 0, mk<T>(Av.x, Bv.x));
            L.put(line, M, mk<T>(0, 0));
          } else {
            L.put(line, kk, mk<T>(Av.x - Bv.y, Av.y + Bv.x));
            L.put(line, N - kk, mk<T>(Av.x + Bv.y, Bv.x - Av.y));
          }
        }
      }
    }
  }
  __syncthreads();
  cl_arrive();  // (2) this CTA has finished reading the cluster's A
  cfft_ip_tid<T, N, 1, C::NLB, NT, false, 1, true, C::R>(L, L, L, tws, cl_tid(sm.zero));
  __syncthreads();
  T m0 = mx[0], m1 = mx[1], m2 = mx[2];
  for (int i = cl_tid(sm.zero); act && i < RCh * N; i += NT) {
    const int q = i / N, x = i % N;
    T f2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = q + h * RCh;
      const cpx<T> z0 = L.get(row, x), z1 = L.get(RC + row, x), z2 = L.get(2 * RC + row, x);
      const T ux = z0.x, uy = z0.y, uz = z1.x, wx = z1.y, wy = z2.x, wz = z2.y;
      m0 = fmax(m0, fabs(ux));
      m1 = fmax(m1, fabs(uy));
      m2 = fmax(m2, fabs(uz));
      L.put(row, x, mk<T>(uy * wz - uz * wy, uz * wx - ux * wz));
      f2[h] = ux * wy - uy * wx;
    }
    L.put(RC + q, x, mk<T>(f2[0], f2[1]));
  }
  mx[0] = m0;
  mx[1] = m1;
  mx[2] = m2;
  __syncthreads();
  {
    const WorkTile<T, N, C::NLF, false> LF{B};
    cfft_ip_tid<T, N, 1, C::NLF, NT, false, -1, true, C::R>(LF, LF, LF, tws, cl_tid(sm.zero));
  }
  __syncthreads();
  cl_wait();  // (2) nobody reads A any more: the products may land there
  // item (line, kp): split the line's spectrum P into the two real rows' spectra and store
  // (F_k, F_k+1, ...) of each into [y][3][KC] of the CTA owning k
  for (int i = cl_tid(sm.zero); act && i < C::NLF * (M / VEC); i += NT) {
    const int kp = i % (M / VEC), line = i / (M / VEC);
    const int k = kp * VEC, s = k / KC, col = k % KC;
    cpx<T> Fa[2], Fb[2];
#pragma unroll
    for (int h = 0; h < VEC; ++h) {
      const int kk = k + h;
      const cpx<T> P = L.get(line, kk), Q = L.get(line, kk == 0 ? 0 : N - kk);
      Fa[h] = mk<T>(T(0.5) * (P.x + Q.x), T(0.5) * (P.y - Q.y));
      Fb[h] = mk<T>(T(0.5) * (P.y + Q.y), T(0.5) * (Q.x - P.x));
    }
    const bool own = line < RC;
    const int ra = own ? line : line - RC, rb = own ? line : line - RC + RCh;
    const int fa = own ? 0 : 2, fb = own ? 1 : 2;
    const unsigned oa = (unsigned)((((y0 + ra) * 3 + fa) * KC + col) * sizeof(cpx<T>));
    const unsigned ob = (unsigned)((((y0 + rb) * 3 + fb) * KC + col) * sizeof(cpx<T>));
    cl_st16(cl_map(aA + oa, (unsigned)s), Fa);
    cl_st16(cl_map(aA + ob, (unsigned)s), Fb);
  }
  fence_proxy_async();  // B is about to be written by the next TMA load
  __syncthreads();
  cl_arrive();  // (3) this CTA's products are stored
  if (threadIdx.x == 0 && next >= 0) cl_issue<T, N, NT>(sm, map, kx0, next);
  cl_wait();  // (3) every product of this CTA's columns has arrived

  // ---- phase C: forward y of the 3 product columns, straight to Ft ------------------------
  cfft_ip_tid<T, N, 1, C::NLC, NT, true, -1, true, C::R>(SmTile<T, C::NLC>{A}, WorkTile<T, N, C::NLC, true>{A},
                                                      ClFtOut<T, N, KC>{Ft, z, kx0}, tws, cl_tid(sm.zero));
  __syncthreads();
}

// planes z0 + P ... z0 + PL - 1 as straight-line code (compile-time recursion, no loop)
template <typename T, int N, int NT, int P, int PL>
struct cl_planes {
  static __device__ __forceinline__ void run(const CUtensorMap* map, cpx<T>* Ft, int z0, T* mx, ClArgs a) {
    cl_plane<T, N, NT>(map, Ft, z0 + P, P + 1 < PL ? z0 + P + 1 : -1, (unsigned)(P & 1), mx, a);
    if constexpr (P + 1 < PL) cl_planes<T, N, NT, P + 1, PL>::run(map, Ft, z0, mx, a);
  }
};

// grid: CS x N / PL clusters, cluster (CS, 1, 1), NT threads, ClCfg::smem bytes.  Cluster c
// takes the planes c PL ... c PL + PL - 1 in straight-line code (the plane loop is unrolled:
// as a run-time loop the compiler kept every phase's plane-invariant index arithmetic live
// across the whole loop and spilled), each plane's load issued during the previous plane's
// phase C.  map_mixed: 3D map over mixed [5][N][N][M] in scalars of T, dims {2M, N (ky),
// 5N (f N + z)}, box {2KC, N, 1} (the box's inner extent 2KC sizeof(T) and its x coordinate
// 2 kx0 sizeof(T) are multiples of 16 bytes).  Ft: [3][N][N][M] complex, written directly.
template <typename T, int N, int NT>
__global__ void __launch_bounds__(NT, 1)
    k2_slabcl(const __grid_constant__ CUtensorMap map_mixed, cpx<T>* __restrict__ Ft,
              const cpx<T>* __restrict__ tw, ClArgs a) {
  using C = ClCfg<T, N, NT>;
  constexpr int PL = C::PL;
  const ClSmem<T, N, NT> sm;
  const int z0 = (int)(blockIdx.x / C::CS) * PL;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sm.tws[tw_pad(i)] = ldg(&tw[i]);
  if (threadIdx.x == 0) {
    mbar_init(sm.bar, 1);
    *sm.zero = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) cl_issue<T, N, NT>(sm, &map_mixed, (int)cl_rank() * C::KC, z0);
  T mx[3] = {T(0), T(0), T(0)};
  cl_planes<T, N, NT, 0, PL>::run(&map_mixed, Ft, z0, mx, a);
  if (a.umax) block_max3<T>(mx[0], mx[1], mx[2], reinterpret_cast<T*>(sm.B), a.umax);
}

}  // namespace ns
