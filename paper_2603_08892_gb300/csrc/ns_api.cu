// ns_api.cu -- host runtime and C ABI of libns (declared in include/ns.h).
//
// The host side owns the device buffers, factorises the transform lengths, sizes the
// tiles, draws the random shifts and forcing patterns (counter-based, reproducible) and
// sequences the kernels of ns_kernels.cuh into the schemes of Sec. 4 and 6.1 of the paper:
//   RK2            INIT | X P(RK2_1) X P(RK2_2)                       41 C bytes / step
//   RK4 (Lawson)   INIT | X P(RK4_1) X P(RK4_2) X P(RK4_3) X P(RK4_4)  94 C
//   PS exact       INIT(2 shifts) | 2X P(RK2_1, avg) 2X P(RK2_2, avg)  73 C
//   PS approx/rand INIT(alpha_0) | X P(ROG_1, beta_n) X P(ROG_2, alpha_{n+1})  44 C
// where X is the slab pass and P the pencil pass of one evaluation, and C = N^3 * sizeof(T)
// is the size of one half-spectrum complex field.
#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ns.h"
#include "ns_internal.h"
#include "ns_kernels.cuh"
#include "ns_kernels2.cuh"

using namespace ns;

// size-specialised kernels (ns_k2_*.cu)
namespace ns {
bool k2_lookup_f32a(int N, K2Entry<float>* e);
bool k2_lookup_f32b(int N, K2Entry<float>* e);
bool k2_lookup_f32c(int N, K2Entry<float>* e);
bool k2_lookup_f32d(int N, K2Entry<float>* e);
bool k2_lookup_f64a(int N, K2Entry<double>* e);
bool k2_lookup_f64b(int N, K2Entry<double>* e);
bool k2_lookup_f64c(int N, K2Entry<double>* e);
}  // namespace ns


namespace {

thread_local std::string g_init_error;

struct NsError {
  int code;
  std::string msg;
};

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      throw NsError{e_ == cudaErrorMemoryAllocation ? NS_ERR_OOM : NS_ERR_CUDA,          \
                    std::string(#call) + ": " + cudaGetErrorString(e_)};                 \
    }                                                                                    \
  } while (0)

#define LAUNCH_CHECK() CUDA_TRY(cudaGetLastError())

bool is_2a3b(int n) {
  if (n <= 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

FFTPlan make_plan(int n, int Ntab) {
  FFTPlan p;
  memset(&p, 0, sizeof(p));
  p.n = n;
  p.tw_stride = Ntab / n;
  int m = n, a2 = 0, a3 = 0;
  while (m % 2 == 0) { m /= 2; ++a2; }
  while (m % 3 == 0) { m /= 3; ++a3; }
  while (a2 >= 3) { p.radix[p.nst++] = 8; a2 -= 3; }
  if (a2 == 2) p.radix[p.nst++] = 4;
  if (a2 == 1) p.radix[p.nst++] = 2;
  for (int i = 0; i < a3; ++i) p.radix[p.nst++] = 3;
  return p;
}

int largest_divisor_le(int m, int cap) {
  for (int d = cap < m ? cap : m; d >= 1; --d)
    if (m % d == 0) return d;
  return 1;
}

// block size for a batch of nl lines of length n (every stage holds <= 15 values / thread)
int fft_block(int nl, int n) {
  const int need = (nl * n + 14) / 15;
  int bd = 128;
  while (bd < need) bd *= 2;
  return bd;
}

// splitmix64 (Steele, Lea & Flood 2014): n-th output of the generator seeded with s
// Tile shapes and launch sizes of the generic (run-time radix) kernels for a grid of N
// points, elements of cs bytes; shared by the contexts and the allocation-free entry point.
struct GenericShapes {
  int TX, bdP;        // pencil: TX columns, threads
  size_t smP;         // pencil shared memory (4 tiles)
  int TY, bdY;        // y passes: TY columns, threads
  size_t smYi, smYf;  // inverse (6 tiles) / forward (3 tiles) shared memory
  int RX, bdX;        // x rows: RX rows, threads
  size_t smX;         // x-row shared memory (6 fields)
};
GenericShapes generic_shapes(int N, size_t cs) {
  const int M = N / 2;
  const size_t smax = 200 * 1024;
  GenericShapes g;
  g.TX = largest_divisor_le(M, 16);
  while (g.TX > 1 && (4 * N * g.TX * cs > smax || fft_block(g.TX, N) > 512)) g.TX = largest_divisor_le(M, g.TX - 1);
  g.bdP = fft_block(g.TX, N) < 256 ? 256 : fft_block(g.TX, N);
  g.smP = 4 * (size_t)N * g.TX * cs;
  g.TY = largest_divisor_le(M, 16);
  while (g.TY > 1 && (6 * N * g.TY * cs > smax || fft_block(g.TY, N) > 512)) g.TY = largest_divisor_le(M, g.TY - 1);
  g.bdY = fft_block(g.TY, N) < 256 ? 256 : fft_block(g.TY, N);
  g.smYi = 6 * (size_t)N * g.TY * cs;
  g.smYf = 3 * (size_t)N * g.TY * cs;
  g.RX = 16;
  while (g.RX > 1 && (6 * (size_t)g.RX * M * cs > 100 * 1024 || fft_block(g.RX, M) > 512)) g.RX /= 2;
  g.bdX = fft_block(g.RX, M) < 256 ? 256 : fft_block(g.RX, M);
  g.smX = 6 * (size_t)g.RX * M * cs;
  return g;
}
// true when every generic kernel's shared memory fits the device's opt-in limit
bool generic_shapes_fit(const GenericShapes& g, int optin) {
  return (long long)g.smP <= optin && (long long)g.smYi <= optin && (long long)g.smYf <= optin &&
         (long long)g.smX <= optin;
}

// Integer bounds of the strict truncation test (Sec. 3.2: modes with |k| >= kmax zeroed):
// K2max = the largest integer below kmax^2 (spherical: keep k^2 <= K2max), Kimax = the largest
// integer below kmax (cubic: keep max|k_i| <= Kimax), both computed in FP64.
void trunc_bounds(double kmax, int* K2max, int* Kimax) {
  const double q = kmax * kmax;
  double m = std::floor(q);
  if (m == q) m -= 1;
  *K2max = (int)m;
  double r = std::floor(kmax);
  if (r == kmax) r -= 1;
  *Kimax = (int)r;
}

uint64_t splitmix64(uint64_t s, uint64_t n) {
  uint64_t z = s + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t s, uint64_t n) {
  return (double)(splitmix64(s, n) >> 11) * (1.0 / 9007199254740992.0);
}

// cuTensorMapEncodeTiled of the driver, looked up through the runtime (no link to libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

bool k2_find(int N, K2Entry<float>* e) {
  if (std::getenv("NS_GENERIC_KERNELS")) return false;
  return k2_lookup_f32a(N, e) || k2_lookup_f32b(N, e) || k2_lookup_f32c(N, e) || k2_lookup_f32d(N, e);
}
bool k2_find(int N, K2Entry<double>* e) {
  if (std::getenv("NS_GENERIC_KERNELS")) return false;
  return k2_lookup_f64a(N, e) || k2_lookup_f64b(N, e) || k2_lookup_f64c(N, e);
}

struct SolverBase {
  virtual ~SolverBase() {}
  virtual void set_velocity(const double* u) = 0;
  virtual void get_velocity(double* u) = 0;
  virtual void get_state(double* s) = 0;
  virtual void set_state(const double* s) = 0;
  virtual void step(double dt, int nsteps) = 0;
  virtual void nonlinear(const double* in, const double* delta, double* out) = 0;
  virtual void energy(double* E, double* eps) = 0;
  virtual void spectrum(int kind, double* out, int nbins) = 0;
  virtual void step_cfl(double cfl, double dt_max, int nsteps) = 0;
  virtual void step_diag(double dt, int nsteps, double* E, double* eps) = 0;
  virtual void invalidate_carry() = 0;  // the next step recomputes its first input
  virtual void raw_state(std::vector<unsigned char>& out) = 0;         // native-precision bytes
  virtual void set_raw_state(const unsigned char* in, size_t n) = 0;
  virtual void forcing_params(int* kind, double* v, uint64_t* seed) = 0;  // v: kmin, kmax, eps, tcorr
  virtual void energy_flux(const double* delta, int nshift, double* flux, double* cumd, int nbins) = 0;
  virtual void set_forcing(int kind, double kfmin, double kfmax, double eps, double tcorr,
                           uint64_t seed) = 0;
  virtual void* state_ptr() = 0;
  virtual void buffers(double dt, NsCtxBuffers* b) = 0;
  virtual void vjp(const double* u0, int nsteps, double dt, int ckpt, int loss, double* L,
                   double* grad) = 0;
  virtual void vjp_state(const double* u0, int nsteps, double dt, int ckpt, const double* gT,
                         double* grad) = 0;
  virtual void tape_forward(const void* u0, int nsteps, double dt, int ckpt, void* uT) = 0;
  virtual void rank_copy(int which, int axis, int lo, int hi, bool to_dev, double* host) = 0;
  virtual void rank_pencil(int kind, const double* delta, int lo, int hi) = 0;
  virtual void rank_slab(int lo, int hi) = 0;
  virtual void tape_backward(const void* gT, int loss, void* grad) = 0;
  virtual void profile(int on) = 0;
  virtual void profile_read(int k, double* ms, int64_t* n, int64_t* launches) = 0;
};

}  // namespace

struct ns_ctx {
  ns_params p;
  double K2maxd;
  int K2max, Kimax;
  double t = 0.0;
  int64_t step = 0;
  bool have_state = false;
  std::vector<double> override_shifts;  // [n][3], consumed from the front
  size_t override_pos = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  SolverBase* solver = nullptr;
  std::string err;
};

namespace {

template <typename T>
struct Solver : SolverBase {
  ns_ctx* c;
  int N, M;
  size_t F1;  // complex elements of one half-spectrum field: N*N*M
  cudaStream_t st;
  // device buffers
  cpx<T>* state = nullptr;
  cpx<T>* acc = nullptr;
  cpx<T>* mixed[2] = {nullptr, nullptr};
  cpx<T>* Ft[2] = {nullptr, nullptr};
  cpx<T>* scr = nullptr;
  cpx<T>* tw = nullptr;
  T* ifac = nullptr;
  cpx<T>* shtab = nullptr;
  size_t shtab_cap = 0;  // number of shift vectors
  double* d_shifts = nullptr;
  double* red = nullptr;
  int red_blocks = 0;
  int* d_err = nullptr;
  double cur_dt = -1.0;
  // slab pass on two internal streams (plane groups alternate, double-buffered scratch) so
  // the kernels of one group overlap those of the next; chosen by the autotuner
  int slab_streams = 1;
  // slab pass as one persistent pipeline launch (k2_slabpipe) with a ring of pipe_ring
  // scratch planes; chosen by the autotuner where the size has the kernel
  bool pipe = false;
  int pipe_ring = 0, pipe_lag = 0, pipe_grid = 0, pipe_stall = 0;
  long long pipe_spin = 1ll << 26;
  unsigned char* d_pipe = nullptr;  // [3][N] done counters, ticket, abort flag
  // slab pass in thread-block clusters, the plane kept on chip (k2_slabcl); chosen by the
  // autotuner where the size has the kernel and the device can hold its clusters
  bool clus = false;
  int cl_var = 1;                  // thread-count variant of the cluster kernel
  // compiled tile alternatives chosen by the autotuner (K2Cfg variant bits: 1 pencil width,
  // 2 inverse-y width, 4 x rows, 8 forward-y width, 16 pencil at 64 registers; 0 = defaults)
  int vsel = 0;
  int cl_ncl = -1;                 // clusters the device holds at once (-1: not yet queried)
  long long cl_spin = 1ll << 20;   // polls of its bounded TMA wait
  std::vector<std::pair<const void*, CUtensorMap>> cl_maps;  // TMA maps of the mixed buffers
  cudaStream_t ss[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  void ensure_streams() {
    if (ss[0]) return;
    for (int i = 0; i < 2; ++i) {
      CUDA_TRY(cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
      CUDA_TRY(cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming));
    }
    CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  }
  // Step whose first evaluation's input the mixed fields (and the forcing record) already
  // hold: the last pencil pass of every ns_step call prepares the next step, so the next call
  // skips its INIT pass.  -1 whenever anything else wrote the state, the mixed fields or the
  // forcing record.
  int64_t carry_step = -1;
  // adaptive time step (ns_step_cfl): dt = min(dt_max, cfl dx / sum_i max|u_i|) per step
  double cfl = 0.0, cfl_dtmax = 0.0;
  unsigned long long* d_umax = nullptr;
  // forcing
  int fkind = NS_FORCE_NONE, fK = 0;
  double fkmin = 0, fkmax = 0, feps = 0, ftcorr = 1, fD = 0;
  uint64_t fseed = 0;
  cpx<double>* fpat = nullptr;
  int fpat_cap = 0;
  cpx<T>* force = nullptr;
  cpx<T>* shell = nullptr;
  // plans and launch shapes
  FFTPlan pz, py, px;
  int TX, bdP;
  size_t smP;
  int TY, bdYi, bdYf;
  size_t smYi, smYf;
  int RX, bdX;
  size_t smX;
  int G, Gmax;
  bool tuned = false;
  int nsm = 148;
  K2Entry<T> k2;     // size-specialised kernels, if this N has them
  bool use2 = false;
  // optional per-kernel timing with CUDA events on the context's stream
  struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> rec;
    double ms[NS_PROF_KINDS] = {0};
    int64_t n[NS_PROF_KINDS] = {0};
    int64_t launches[NS_PROF_KINDS] = {0};
  } prof;

  cudaEvent_t prof_event() {
    if (!prof.pool.empty()) {
      cudaEvent_t e = prof.pool.back();
      prof.pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    return e;
  }
  // brackets one launch (or a pass) of kind k; returns the stop event to record after it
  cudaEvent_t prof_begin(int k, cudaStream_t s = nullptr) {
    prof.launches[k] += 1;
    if (!prof.on || prof.rec.size() >= 65536) return nullptr;
    cudaEvent_t a = prof_event(), b = prof_event();
    CUDA_TRY(cudaEventRecord(a, s ? s : st));
    prof.rec.push_back({k, {a, b}});
    return b;
  }
  void prof_end(cudaEvent_t b, cudaStream_t s = nullptr) {
    if (b) CUDA_TRY(cudaEventRecord(b, s ? s : st));
  }
  void prof_collect() {
    CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& r : prof.rec) {
      float ms = 0;
      CUDA_TRY(cudaEventElapsedTime(&ms, r.second.first, r.second.second));
      prof.ms[r.first] += ms;
      prof.n[r.first] += 1;
      prof.pool.push_back(r.second.first);
      prof.pool.push_back(r.second.second);
    }
    prof.rec.clear();
  }
  void profile(int on) override {
    prof_collect();
    prof.on = on != 0;
    for (int k = 0; k < NS_PROF_KINDS; ++k) prof.ms[k] = 0, prof.n[k] = 0, prof.launches[k] = 0;
  }
  void profile_read(int k, double* ms, int64_t* n, int64_t* launches) override {
    prof_collect();
    if (ms) *ms = prof.ms[k];
    if (n) *n = prof.n[k];
    if (launches) *launches = prof.launches[k];
  }

  explicit Solver(ns_ctx* ctx) : c(ctx) {
    N = c->p.N;
    M = N / 2;
    F1 = (size_t)N * N * M;
    st = c->stream;
    int dev = c->p.device;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    pz = make_plan(N, N);
    py = pz;
    px = make_plan(M, N);
    const size_t cs = sizeof(cpx<T>);
    const GenericShapes gs = generic_shapes(N, cs);
    TX = gs.TX; bdP = gs.bdP; smP = gs.smP;
    TY = gs.TY; bdYi = bdYf = gs.bdY; smYi = gs.smYi; smYf = gs.smYf;
    RX = gs.RX; bdX = gs.bdX; smX = gs.smX;
    // initial plane group: a scratch (6 fields) of 48 MB, small enough for L2
    const size_t plane6 = 6 * (size_t)N * M * cs;
    G = (int)((48ull << 20) / plane6);
    if (G < 1) G = 1;
    if (G > N) G = N;
    // the scratch holds up to Gmax planes (at most 1 GB): the autotuner may pick any group
    // size up to it; on GB300 groups larger than L2 measured faster (fewer launch tails)
    Gmax = (int)((1024ull << 20) / plane6);
    if (Gmax < G) Gmax = G;
    if (Gmax > N) Gmax = N;

    // The attribute belongs to the kernel, not to this context: allow the device maximum so
    // that contexts of different sizes in one process never lower each other's limit.
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (!generic_shapes_fit(gs, optin))
      throw NsError{NS_ERR_INTERNAL, "tile shapes exceed the shared memory of the device"};
    CUDA_TRY(cudaFuncSetAttribute(k_pencil<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    CUDA_TRY(cudaFuncSetAttribute(k_yinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    CUDA_TRY(cudaFuncSetAttribute(k_yfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    CUDA_TRY(cudaFuncSetAttribute(k_xrow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    use2 = k2_find(N, &k2);
    if (const char* e = std::getenv("NS_ZERO_COPY")) zero_copy = std::atoi(e) != 0;
    if (use2) {
      // each kernel may take the opt-in limit less its own static shared memory
      auto allow = [&](auto* f, size_t need) {
        cudaFuncAttributes fa;
        CUDA_TRY(cudaFuncGetAttributes(&fa, f));
        const int dyn = optin - (int)fa.sharedSizeBytes;
        if ((long long)need > (long long)dyn)
          throw NsError{NS_ERR_INTERNAL, "specialised tile shapes exceed the shared memory of the device"};
        CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
      };
      allow(k2.pencil, k2.smP5);
      allow(k2.pencil1, k2.smP1);
      allow(k2.pencil1e, k2.smP1);
      allow(k2.pencil1re, k2.smP1);
      allow(k2.pencil1r[0], k2.smP1);
      allow(k2.pencil1r[1], k2.smP1);
      allow(k2.pencil2, k2.smP5);
      allow(k2.yinv, k2.smYI);
      allow(k2.yfwd, k2.smY);
      allow(k2.xrow, k2.smX);
      if (k2.has_alt) {
        allow(k2.alt.pencil1r[0], k2.alt.smP1);
        allow(k2.alt.pencil1r[1], k2.alt.smP1);
        allow(k2.pencil1r64[0], k2.smP1);
        allow(k2.pencil1r64[1], k2.smP1);
        allow(k2.alt.yinv, k2.alt.smYI);
        allow(k2.alt.yfwd, k2.alt.smY);
        allow(k2.alt.xrow, k2.alt.smX);
      }
      for (int v = 0; v < 2; ++v)
        if (k2.slabcl[v]) {
          allow(k2.slabcl[v], k2.smCL);
          if (k2.CLS > 8)
            CUDA_TRY(cudaFuncSetAttribute(k2.slabcl[v], cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        }
      if (k2.slabpipe)  // (it has a few bytes of static shared memory: its own size, not optin)
        CUDA_TRY(cudaFuncSetAttribute(k2.slabpipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k2.smPIPE));
    }

    const int sch = c->p.scheme;
    const bool two = sch == NS_RK2_PS_EXACT;
    CUDA_TRY(cudaMalloc(&state, 3 * F1 * cs));
    CUDA_TRY(cudaMalloc(&acc, 3 * F1 * cs));
    CUDA_TRY(cudaMalloc(&mixed[0], 5 * F1 * cs));
    CUDA_TRY(cudaMalloc(&Ft[0], 3 * F1 * cs));
    if (two) {
      CUDA_TRY(cudaMalloc(&mixed[1], 5 * F1 * cs));
      CUDA_TRY(cudaMalloc(&Ft[1], 3 * F1 * cs));
    }
    CUDA_TRY(cudaMalloc(&scr, 6 * (size_t)Gmax * N * M * cs));
    CUDA_TRY(cudaMalloc(&tw, N * cs));
    CUDA_TRY(cudaMalloc(&ifac, 2 * N * sizeof(T)));
    red_blocks = 2 * nsm;
    CUDA_TRY(cudaMalloc(&red, (size_t)red_blocks * 1024 * sizeof(double)));
    CUDA_TRY(cudaMalloc(&d_err, sizeof(int)));
    CUDA_TRY(cudaMalloc(&d_umax, 3 * sizeof(unsigned long long)));
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(state, 0, 3 * F1 * cs, st));
    k_twiddle<T><<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    LAUNCH_CHECK();
    CUDA_TRY(cudaStreamSynchronize(st));
  }

  ~Solver() override {
    cudaFree(state); cudaFree(acc); cudaFree(mixed[0]); cudaFree(mixed[1]);
    cudaFree(nlbuf); cudaFree(nltmp); cudaFree(d_umax); cudaFree(d_pipe);
    cudaFree(d_epart);
    if (h_err) cudaFreeHost(h_err);
    if (h_series) cudaFreeHost(h_series);
    cudaFree(Ft[0]); cudaFree(Ft[1]); cudaFree(scr); cudaFree(tw); cudaFree(ifac);
    cudaFree(shtab); cudaFree(d_shifts); cudaFree(red); cudaFree(d_err);
    cudaFree(fpat); cudaFree(force); cudaFree(shell);
    for (int i = 0; i < 2; ++i) {
      if (ss[i]) cudaStreamDestroy(ss[i]);
      if (ev_join[i]) cudaEventDestroy(ev_join[i]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (auto* p : adj) cudaFree(p);
    cudaFree(mixedB); cudaFree(FtB); cudaFree(shS); cudaFree(shR); cudaFree(ftab);
    cudaFree(rank_stg);
    for (auto& r : prof.rec) {
      cudaEventDestroy(r.second.first);
      cudaEventDestroy(r.second.second);
    }
    for (auto e : prof.pool) cudaEventDestroy(e);
  }

  void* state_ptr() override { return state; }

  void buffers(double dt, NsCtxBuffers* b) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    if (dt > 0) set_dt(dt);
    b->N = N; b->precision = c->p.precision; b->scheme = c->p.scheme; b->truncation = c->p.truncation;
    b->K2max = c->K2max; b->Kimax = c->Kimax; b->G = Gmax; b->nu = c->p.nu; b->kmax = c->p.kmax;
    b->state = state; b->mixed = mixed[0]; b->Ft = Ft[0]; b->scr = scr; b->tw = tw; b->ifac = ifac;
    b->err = d_err; b->seed = c->p.seed; b->step = c->step; b->t = c->t;
  }

  // ---- device error flag ------------------------------------------------------------
  // per-step diagnostics (step_diag): the final pencil pass of each step leaves per-tile sums
  // of its written state in d_epart; their fixed-order sum is written by the device, 16 bytes
  // per step, straight into the mapped pinned host array h_series (device address d_series)
  bool diag = false;
  int diag_n = 0;
  size_t series_cap = 0;
  double* d_epart = nullptr;
  double* d_series = nullptr;
  double* h_series = nullptr;
  int* h_err = nullptr;  // pinned copy of the device flag: one stream sync per check
  void sync_check() {
    if (!h_err) CUDA_TRY(cudaMallocHost(&h_err, sizeof(int)));
    CUDA_TRY(cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const int h = *h_err;
    if (h) {
      CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
      CUDA_TRY(cudaStreamSynchronize(st));
      if (h & PIPE_ERR_TIMEOUT)
        throw NsError{NS_ERR_TIMEOUT, "slab pipeline: a bounded wait gave up (the pass was abandoned)"};
      if (h & CL_ERR_TIMEOUT)
        throw NsError{NS_ERR_TIMEOUT, "cluster slab pass: a bounded TMA wait gave up"};
      throw NsError{NS_ERR_INTERNAL, "device-side launch-shape check failed (flag " + std::to_string(h) + ")"};
    }
  }

  // ---- passes -----------------------------------------------------------------------
  SlabArgs<T> slab_args() {
    SlabArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.M = M; a.py = py; a.px = px; a.tw = tw; a.scr = scr;
    a.TY = TY; a.RX = RX; a.err = d_err;
    // Ft modes no pencil tile reads are left unwritten (every pencil instance of this size
    // skips the same truncated tiles; the widest tile decides)
    if (use2 && NS_FT_SKIP) {
      a.skip_tx = std::max(k2.TX, k2.has_alt ? k2.alt.TX : 0);
      a.trunc = c->p.truncation; a.K2max = c->K2max; a.Kimax = c->Kimax;
      a.fK = fkind != NS_FORCE_NONE ? fK : -1;
    }
    return a;
  }

  // clusters of CLS CTAs the device holds at once (0: none fit; the pass is not used)
  int cl_clusters() {
    if (cl_ncl >= 0) return cl_ncl;
    cl_ncl = 0;
    if (!use2 || !k2.slabcl[0]) return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = k2.CLS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(k2.CLS);
    cfg.blockDim = dim3(k2.NTCL[0]);
    cfg.dynamicSmemBytes = k2.smCL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k2.slabcl[0], &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    cl_ncl = n;
    return cl_ncl;
  }
  // TMA map of a mixed buffer [5][N][N][M]: scalars of T, dims {2M, N, 5N}, box {2KC, N, 1}
  CUtensorMap cl_map(const cpx<T>* mix) {
    for (const auto& m : cl_maps)
      if (m.first == mix) return m.second;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) throw NsError{NS_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * M, (cuuint64_t)N, (cuuint64_t)5 * N};
    const cuuint64_t strides[2] = {(cuuint64_t)M * sizeof(cpx<T>), (cuuint64_t)N * M * sizeof(cpx<T>)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * k2.CLKC), (cuuint32_t)N, 1u};
    const cuuint32_t es[3] = {1u, 1u, 1u};
    const CUresult r = enc(&map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                           3, const_cast<cpx<T>*>(mix), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      throw NsError{NS_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    cl_maps.push_back({mix, map});
    return map;
  }
  // the slab pass as one launch of clusters (k2_slabcl): mixed -> Ft, no scratch
  void slab_cluster(const cpx<T>* mix, cpx<T>* out, void* umax) {
    const CUtensorMap map = cl_map(mix);
    ClArgs ca;
    ca.err = d_err;
    ca.umax = umax;
    ca.spin_limit = cl_spin;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = k2.CLS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(k2.CLS * (N / k2.CLPL));  // every cluster takes CLPL planes
    cfg.blockDim = dim3(k2.NTCL[cl_var]);
    cfg.dynamicSmemBytes = k2.smCL;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t e = prof_begin(NS_PROF_SLAB_CLUSTER);
    CUDA_TRY(cudaLaunchKernelEx(&cfg, k2.slabcl[cl_var], map, out, static_cast<const cpx<T>*>(tw), ca));
    prof_end(e);
  }

  // the three slab kernels on the plane group (a.z0, a.G) on stream s
  void slab_group(const SlabArgs<T>& a, cudaStream_t s) {
    cudaEvent_t e = prof_begin(NS_PROF_YINV, s);
    if (use2)
      if (vsel & 2)
        k2.alt.yinv<<<dim3(M / k2.alt.TYI, a.G), k2.alt.NTYI, k2.alt.smYI, s>>>(a);
      else
        k2.yinv<<<dim3(M / k2.TYI, a.G), k2.NTYI, k2.smYI, s>>>(a);
    else
      k_yinv<T><<<dim3(M / TY, a.G), bdYi, smYi, s>>>(a);
    prof_end(e, s);
    e = prof_begin(NS_PROF_XROW, s);
    if (use2)
      if (vsel & 4)
        k2.alt.xrow<<<(a.G * N + k2.alt.RX - 1) / k2.alt.RX, k2.alt.NTX, k2.alt.smX, s>>>(a);
      else
        k2.xrow<<<(a.G * N + k2.RX - 1) / k2.RX, k2.NTX, k2.smX, s>>>(a);
    else
      k_xrow<T><<<(a.G * N + RX - 1) / RX, bdX, smX, s>>>(a);
    prof_end(e, s);
    e = prof_begin(NS_PROF_YFWD, s);
    if (use2)
      if (vsel & 8)
        k2.alt.yfwd<<<dim3(M / k2.alt.TY, a.G), k2.alt.NTY, k2.alt.smY, s>>>(a);
      else
        k2.yfwd<<<dim3(M / k2.TY, a.G), k2.NTY, k2.smY, s>>>(a);
    else
      k_yfwd<T><<<dim3(M / TY, a.G), bdYf, smYf, s>>>(a);
    prof_end(e, s);
  }

  // slab pass over every plane group: mixed (5 fields) -> Ft (3 fields)
  void slab(const cpx<T>* mix, cpx<T>* out, bool umax = false) {
    SlabArgs<T> a = slab_args();
    a.mixed = mix;
    a.Ft = out;
    a.xmode = XMODE_NONLINEAR;
    if (umax) {
      CUDA_TRY(cudaMemsetAsync(d_umax, 0, 3 * sizeof(unsigned long long), st));
      a.umax = d_umax;
    }
    cudaEvent_t pass = prof_begin(NS_PROF_SLAB_PASS);
    if (clus && use2 && k2.slabcl[cl_var] && cl_clusters() > 0) {
      slab_cluster(mix, out, a.umax);
      prof_end(pass);
      LAUNCH_CHECK();
      return;
    }
    if (pipe && use2 && k2.slabpipe && pipe_ring >= 2 && pipe_ring <= Gmax) {
      const int nb = 3 * N;
      if (!d_pipe) CUDA_TRY(cudaMalloc(&d_pipe, nb * sizeof(int) + 16));
      if (!pipe_grid) {
        int per = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k2.slabpipe, k2.NTPIPE, k2.smPIPE));
        pipe_grid = (per > 0 ? per : 1) * nsm;
      }
      CUDA_TRY(cudaMemsetAsync(d_pipe, 0, nb * sizeof(int) + 16, st));
      PipeCtl ctl;
      ctl.done = reinterpret_cast<int*>(d_pipe);
      ctl.next = reinterpret_cast<unsigned long long*>(d_pipe + nb * sizeof(int));
      ctl.abort = reinterpret_cast<int*>(d_pipe + nb * sizeof(int) + 8);
      ctl.spin_limit = pipe_spin;
      ctl.ring = pipe_ring;
      ctl.lag = pipe_lag;
      ctl.stall = pipe_stall;
      a.z0 = 0;
      a.G = pipe_ring;
      a.scr = scr;
      cudaEvent_t e = prof_begin(NS_PROF_SLAB_PIPE);
      k2.slabpipe<<<pipe_grid, k2.NTPIPE, k2.smPIPE, st>>>(a, ctl);
      prof_end(e);
      prof_end(pass);
      LAUNCH_CHECK();
      return;
    }
    const bool two = use2 && slab_streams == 2 && G < N && 2 * G <= Gmax;
    if (two) {
      ensure_streams();
      CUDA_TRY(cudaEventRecord(ev_fork, st));
      for (int i = 0; i < 2; ++i) CUDA_TRY(cudaStreamWaitEvent(ss[i], ev_fork, 0));
    }
    int gi = 0;
    for (int z0 = 0; z0 < N; z0 += G, ++gi) {
      const cudaStream_t s = two ? ss[gi & 1] : st;
      a.z0 = z0;
      a.G = (z0 + G <= N) ? G : N - z0;
      a.scr = scr + (two ? (size_t)(gi & 1) * 6 * G * N * M : 0);  // double-buffered scratch
      slab_group(a, s);
    }
    if (two) {
      for (int i = 0; i < 2; ++i) {
        CUDA_TRY(cudaEventRecord(ev_join[i], ss[i]));
        CUDA_TRY(cudaStreamWaitEvent(st, ev_join[i], 0));
      }
    }
    prof_end(pass);
    LAUNCH_CHECK();
  }

  PencilArgs<T> pencil_args(int mode) {
    PencilArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.N = N; a.M = M; a.TX = TX; a.pz = pz; a.tw = tw; a.mode = mode;
    a.dt = (T)cur_dt; a.ifac = ifac; a.state = state; a.acc = acc;
    a.trunc = c->p.truncation; a.K2max = c->K2max; a.Kimax = c->Kimax;
    a.err = d_err;
    if (fkind != NS_FORCE_NONE) {
      a.shell = shell;
      a.fK = fK;
    }
    return a;
  }

  // the pencil pass over the ky rows [a.iy0, a.iy0 + rows) (rows < 0: every row)
  void pencil(const PencilArgs<T>& a, int rows = -1) {
    cudaEvent_t e = prof_begin(NS_PROF_PENCIL);
    const int R = rows < 0 ? N : rows;
    const bool rog = a.nF == 1 && a.nOut == 1 && !a.epart && (a.mode == MODE_ROG_1 || a.mode == MODE_ROG_2);
    if (use2 && rog && (vsel & 1))  // the autotuner's alternative pencil width
      k2.alt.pencil1r[a.mode == MODE_ROG_1 ? 0 : 1]<<<(M / k2.alt.TX) * R, k2.alt.NTP, k2.alt.smP1, st>>>(a);
    else if (use2 && rog && (vsel & 16))  // the alternative register budget
      k2.pencil1r64[a.mode == MODE_ROG_1 ? 0 : 1]<<<(M / k2.TX) * R, k2.NTP, k2.smP1, st>>>(a);
    else if (use2)
      (a.nF == 1 && a.nOut == 1   ? (a.epart                  ? (a.mode == MODE_ROG_2 ? k2.pencil1re : k2.pencil1e)
                                     : a.mode == MODE_ROG_1 ? k2.pencil1r[0]
                                     : a.mode == MODE_ROG_2 ? k2.pencil1r[1]
                                                            : k2.pencil1)
       : a.nF == 2 && a.nOut == 2 ? k2.pencil2
                                  : k2.pencil)<<<(M / k2.TX) * R, k2.NTP,
                                                  (a.nF == 1 && a.nOut == 1) ? k2.smP1
                                                  : (a.nF > 1 || a.nOut > 1) ? k2.smP5
                                                                             : k2.smP4, st>>>(a);
    else
      k_pencil<T><<<(M / TX) * R, bdP, smP, st>>>(a);
    prof_end(e);
    LAUNCH_CHECK();
  }

  // ---- rank-range passes of a field decomposed over ranks (Sec. 2: the distributed 3D FFT's
  // transposes); the exchanges between them are the caller's
  cpx<T>* rank_stg = nullptr;  // contiguous block staging (5 fields at most)
  cpx<T>* rank_buf(int which) {
    switch (which) {
      case NS_BUF_STATE: return state;
      case NS_BUF_MIXED: return mixed[0];
      case NS_BUF_FT: return Ft[0];
      default: return acc;  // NS_BUF_NL
    }
  }
  int rank_fields(int which) const { return which == NS_BUF_MIXED ? 5 : 3; }
  // block [lo, hi) of the z (or kz) axis (axis 0) or the ky axis (axis 1) of buffer `which`
  // between the device and host FP64 (re, im): axis 0 [F][hi-lo][N][M], axis 1 [F][N][hi-lo][M]
  void rank_copy(int which, int axis, int lo, int hi, bool to_dev, double* host) override {
    carry_step = -1;
    const int F = rank_fields(which), n = hi - lo;
    const size_t cs = sizeof(cpx<T>);
    if (!rank_stg) CUDA_TRY(cudaMalloc(&rank_stg, 5 * F1 * cs));
    cpx<T>* d = rank_buf(which);
    const size_t count = (size_t)F * N * n * M;  // complex values of the block
    size_t width, height, dpitch;
    cpx<T>* base;
    if (axis == 0) {  // F rows of n N M values, field pitch N N M
      width = (size_t)n * N * M * cs; height = F; dpitch = F1 * cs; base = d + (size_t)lo * N * M;
    } else {          // F N rows of n M values, row pitch N M
      width = (size_t)n * M * cs; height = (size_t)F * N; dpitch = (size_t)N * M * cs; base = d + (size_t)lo * M;
    }
    if (to_dev) {
      to_device(host, reinterpret_cast<T*>(rank_stg), 2 * count);
      CUDA_TRY(cudaMemcpy2DAsync(base, dpitch, rank_stg, width, width, height, cudaMemcpyDeviceToDevice, st));
      CUDA_TRY(cudaStreamSynchronize(st));
    } else {
      CUDA_TRY(cudaMemcpy2DAsync(rank_stg, width, base, dpitch, width, height, cudaMemcpyDeviceToDevice, st));
      to_host(reinterpret_cast<const T*>(rank_stg), host, 2 * count);
      sync_check();
    }
  }
  // pencil pass on the ky rows [lo, hi): NS_RANK_INIT: state -> mixed (shifted by delta);
  // NS_RANK_NL: Ft -> the shifted, de-shifted, truncated, projected nonlinear term (NL buffer)
  void rank_pencil(int kind, const double* delta, int lo, int hi) override {
    carry_step = -1;
    std::vector<double> sh(delta, delta + 3);
    upload_shifts(sh);
    PencilArgs<T> p = pencil_args(kind == NS_RANK_INIT ? MODE_INIT : MODE_NL);
    p.shell = nullptr;
    p.iy0 = lo;
    if (kind == NS_RANK_INIT) {
      p.src = state;
      p.nOut = 1; p.osh[0] = shift_tab(0); p.out[0] = mixed[0];
    } else {
      p.nF = 1; p.F[0] = Ft[0]; p.dsh[0] = shift_tab(0); p.wF[0] = (T)(1.0 / ((double)N * N * N));
      p.acc = acc;
    }
    pencil(p, hi - lo);
    sync_check();
  }
  // slab pass on the planes [lo, hi): mixed -> Ft (the three slab kernels, plane groups of G)
  void rank_slab(int lo, int hi) override {
    carry_step = -1;
    SlabArgs<T> a = slab_args();
    a.mixed = mixed[0];
    a.Ft = Ft[0];
    a.xmode = XMODE_NONLINEAR;
    for (int z0 = lo; z0 < hi; z0 += G) {
      a.z0 = z0;
      a.G = (z0 + G <= hi) ? G : hi - z0;
      slab_group(a, st);
    }
    LAUNCH_CHECK();
    sync_check();
  }

  // the pencil pass that writes a step's new state; with diagnostics on, also E and eps of that
  // state (Sec. 3.4): fused into the pass (per-tile sums) on the size-specialised kernels, a
  // separate reduction otherwise; no host synchronisation per step
  void final_pencil(PencilArgs<T> a) {
    if (!diag) {
      pencil(a);
      return;
    }
    const int ntiles = use2 ? (M / k2.TX) * N : 0;
    if (use2) a.epart = d_epart;
    pencil(a);
    double* out = d_series + 2 * (size_t)diag_n;
    if (use2) {
      k_sum_pairs<<<1, 256, 0, st>>>(d_epart, ntiles, out, 0.5, c->p.nu);
    } else {
      const int nb = red_blocks;
      k_energy<T><<<nb, 256, 0, st>>>(state, N, c->p.nu, red);
      k_sum_pairs<<<1, 256, 0, st>>>(red, nb, out);
    }
    LAUNCH_CHECK();
    ++diag_n;
  }

  void step_diag(double dt, int nsteps, double* E, double* eps) override {
    if ((size_t)nsteps > series_cap) {  // at least 4096 steps: later calls allocate nothing
      const size_t cap = nsteps > 4096 ? (size_t)nsteps : 4096;
      if (h_series) {
        CUDA_TRY(cudaStreamSynchronize(st));  // no kernel of this stream still writes into it
        CUDA_TRY(cudaFreeHost(h_series));
      }
      d_series = nullptr;
      h_series = nullptr;
      series_cap = 0;
      CUDA_TRY(cudaHostAlloc(&h_series, 2 * cap * sizeof(double), cudaHostAllocMapped));
      CUDA_TRY(cudaHostGetDevicePointer(&d_series, h_series, 0));
      series_cap = cap;
    }
    if (use2 && !d_epart) CUDA_TRY(cudaMalloc(&d_epart, 2 * (size_t)(M / k2.TX) * N * sizeof(double)));
    diag = true;
    diag_n = 0;
    try {
      step(dt, nsteps);
    } catch (...) {
      diag = false;
      throw;
    }
    diag = false;
    sync_check();
    for (int i = 0; i < nsteps; ++i) {
      E[i] = h_series[2 * (size_t)i];
      eps[i] = h_series[2 * (size_t)i + 1];
    }
  }

  const cpx<T>* shift_tab(int idx) const { return idx < 0 ? nullptr : shtab + (size_t)idx * 3 * N; }

  void upload_shifts(const std::vector<double>& sh) {
    const size_t n = sh.size() / 3;
    if (n == 0) return;
    if (n > shtab_cap) {
      cudaFree(shtab);
      cudaFree(d_shifts);
      shtab = nullptr;
      d_shifts = nullptr;
      CUDA_TRY(cudaMalloc(&shtab, n * 3 * N * sizeof(cpx<T>)));
      CUDA_TRY(cudaMalloc(&d_shifts, n * 3 * sizeof(double)));
      shtab_cap = n;
    }
    CUDA_TRY(cudaMemcpyAsync(d_shifts, sh.data(), n * 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    const int tot = (int)(n * 3 * N);
    k_shift_tables<T><<<(tot + 255) / 256, 256, 0, st>>>(shtab, N, d_shifts, (int)n);
    LAUNCH_CHECK();
  }

  void set_dt(double dt) {
    if (dt == cur_dt) return;
    k_ifac<T><<<(N + 255) / 256, 256, 0, st>>>(ifac, N, c->p.nu, dt, 0.5 * dt);
    LAUNCH_CHECK();
    cur_dt = dt;
  }

  // ---- forcing ------------------------------------------------------------------------
  int fD1() const { return 2 * fK + 1; }
  int fDn() const { return fD1() * fD1() * (fK + 1); }

  // projected random pattern j on the dense table [3][D] (reading documented in ns.h)
  void make_pattern(int64_t j, std::vector<cpx<double>>& out) {
    const int K = fK, D1 = fD1(), D = fDn();
    out.assign(3 * (size_t)D, mk<double>(0, 0));
    // canonical modes in counter order
    std::vector<int> modes;
    for (int kz = -K; kz <= K; ++kz)
      for (int ky = -K; ky <= K; ++ky)
        for (int kx = 0; kx <= K; ++kx) {
          const double k2 = kx * kx + ky * ky + kz * kz;
          if (k2 < fkmin * fkmin || k2 > fkmax * fkmax) continue;
          const bool canon = kx > 0 || kz > 0 || (kz == 0 && ky > 0);
          if (canon && kx < M) {
            modes.push_back(kx);
            modes.push_back(ky);
            modes.push_back(kz);
          }
        }
    const int64_t Mm = (int64_t)modes.size() / 3;
    auto idx = [&](int kx, int ky, int kz) { return ((kz + K) * D1 + (ky + K)) * (K + 1) + kx; };
    for (int64_t m = 0; m < Mm; ++m) {
      const int kx = modes[3 * m], ky = modes[3 * m + 1], kz = modes[3 * m + 2];
      double g[3][2];
      for (int comp = 0; comp < 3; ++comp) {
        const uint64_t n = (uint64_t)((j * Mm + m) * 3 + comp);
        const double u1 = uniform01(fseed, 2 * n), u2 = uniform01(fseed, 2 * n + 1);
        const double r = std::sqrt(-2.0 * std::log(1.0 - u1));
        const double th = 2.0 * M_PI * u2;
        g[comp][0] = r * std::cos(th);
        g[comp][1] = r * std::sin(th);
      }
      // Leray projection P(k) = I - k k / |k|^2
      const double k[3] = {(double)kx, (double)ky, (double)kz};
      const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
      double kd[2] = {0, 0};
      for (int q = 0; q < 3; ++q) {
        kd[0] += k[q] * g[q][0];
        kd[1] += k[q] * g[q][1];
      }
      for (int q = 0; q < 3; ++q) {
        const double re = g[q][0] - k[q] * kd[0] / k2, im = g[q][1] - k[q] * kd[1] / k2;
        out[(size_t)q * D + idx(kx, ky, kz)] = mk<double>(re, im);
        if (kx == 0) out[(size_t)q * D + idx(0, -ky, -kz)] = mk<double>(re, -im);
      }
    }
  }

  int64_t fj0 = 0;  // redraw index of fpat[0]

  void prepare_forcing(double t0, double t1) {
    const int64_t j0 = (int64_t)std::floor(t0 / ftcorr);
    const int64_t j1 = (int64_t)std::floor(t1 / ftcorr) + 2;  // margin for rounding of stage times
    const int n = (int)(j1 - j0 + 1);
    const int D = fDn();
    if (n > fpat_cap) {
      cudaFree(fpat);
      fpat = nullptr;
      CUDA_TRY(cudaMalloc(&fpat, (size_t)n * 3 * D * sizeof(cpx<double>)));
      fpat_cap = n;
    }
    std::vector<cpx<double>> all((size_t)n * 3 * D), one;
    for (int i = 0; i < n; ++i) {
      make_pattern(j0 + i, one);
      std::copy(one.begin(), one.end(), all.begin() + (size_t)i * 3 * D);
    }
    CUDA_TRY(cudaMemcpy(fpat, all.data(), all.size() * sizeof(cpx<double>), cudaMemcpyHostToDevice));
    fj0 = j0;
  }

  // forcing term of the coming pencil pass at time ts, from the state stored in `shell`
  void force_coef(double ts, PencilArgs<T>& a) {
    if (fkind == NS_FORCE_NONE) return;
    const double x = ts / ftcorr;
    const int64_t j = (int64_t)std::floor(x);
    const double th = x - (double)j;
    const int D = fDn();
    if (j < fj0 || j - fj0 + 1 >= fpat_cap)
      throw NsError{NS_ERR_INTERNAL, "forcing pattern index out of the prepared range"};
    const cpx<double>* pj = fpat + (size_t)(j - fj0) * 3 * D;
    k_force_coef<T><<<1, 256, 0, st>>>(pj, pj + 3 * D, th, shell, fK, cur_dt, feps, force, nullptr);
    LAUNCH_CHECK();
    a.force = force;
  }

  void set_forcing(int kind, double kfmin, double kfmax, double eps, double tcorr,
                   uint64_t seed) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    tape.valid = false;  // a recorded adjoint run used the previous forcing
    fkind = kind;
    if (kind == NS_FORCE_NONE) return;
    fkmin = kfmin; fkmax = kfmax; feps = eps; ftcorr = tcorr; fseed = seed;
    fK = (int)std::floor(kfmax);
    cudaFree(force);
    cudaFree(shell);
    force = shell = nullptr;
    CUDA_TRY(cudaMalloc(&force, 3 * (size_t)fDn() * sizeof(cpx<T>)));
    CUDA_TRY(cudaMalloc(&shell, 3 * (size_t)fDn() * sizeof(cpx<T>)));
    CUDA_TRY(cudaMemsetAsync(shell, 0, 3 * (size_t)fDn() * sizeof(cpx<T>), st));
  }

  // ---- autotuner of the plane-group size of the slab pass ------------------------------
  // Candidates G (planes per group of the scratch) with one or two streams are timed on the
  // slab pass with CUDA events; the fastest is kept and cached in a JSON file keyed by device,
  // N, precision and the slab tiles.  Results do not depend on G or on the streams (every
  // plane is transformed the same way).  NS_AUTOTUNE=0 disables it; NS_AUTOTUNE_CACHE sets the
  // cache file; NS_SLAB_PLANES=g forces a group size, NS_SLAB_STREAMS=1|2 the stream count,
  // NS_SLAB_PIPE=1 the pipeline (ring NS_PIPE_RING, lag NS_PIPE_LAG) and =0 excludes it;
  // NS_SLAB_CLUSTER=1 the cluster pass (thread variant NS_CL_VARIANT) and =0 excludes it;
  // NS_TILE_VARIANT=bits forces the compiled tile alternatives of the kernel families;
  // NS_PIPE_SPIN bounds its waits, NS_PIPE_TEST_STALL=1 makes them unsatisfiable (test hook).
  static std::string cache_path() {
    const char* e = std::getenv("NS_AUTOTUNE_CACHE");
    if (e && *e) return e;
    const char* h = std::getenv("HOME");
    return std::string(h && *h ? h : "/tmp") + "/.cache/libns_autotune.json";
  }
  std::string tune_key() {
    cudaDeviceProp pr;
    cudaGetDeviceProperties(&pr, c->p.device);
    std::string k = std::string(pr.name) + "|N=" + std::to_string(N) + "|" +
                    (sizeof(T) == 4 ? "fp32" : "fp64") + (use2 ? "|k2" : "|generic");
    if (use2)  // the slab kernels' tiles and thread counts: a change of kernels re-tunes
      k += "|" + std::to_string(k2.TYI) + "," + std::to_string(k2.NTYI) + "," + std::to_string(k2.TY) +
           "," + std::to_string(k2.NTY) + "," + std::to_string(k2.RX) + "," + std::to_string(k2.NTX);
    for (auto& ch : k)
      if (ch == '"' || ch == '\\') ch = '_';
    return k;
  }
  static bool cache_lookup(const std::string& path, const std::string& key, int* val) {
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
    std::fclose(f);
    const std::string pat = "\"" + key + "\":";
    const size_t pos = txt.find(pat);
    if (pos == std::string::npos) return false;
    *val = std::atoi(txt.c_str() + pos + pat.size());
    return *val > 0;
  }
  static void cache_store(const std::string& path, const std::string& key, int val) {
    // read-modify-write of a flat JSON object {"key": value, ...}
    std::string txt;
    if (FILE* f = std::fopen(path.c_str(), "r")) {
      char buf[4096];
      size_t n;
      while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
      std::fclose(f);
    }
    std::string body;
    const size_t a = txt.find('{'), b = txt.rfind('}');
    if (a != std::string::npos && b != std::string::npos && b > a) body = txt.substr(a + 1, b - a - 1);
    const std::string pat = "\"" + key + "\":";
    const size_t pos = body.find(pat);
    if (pos != std::string::npos) {
      size_t e = body.find_first_of(",}", pos);
      body.erase(pos, (e == std::string::npos ? body.size() : e) - pos);
      while (!body.empty() && (body.back() == ',' || body.back() == ' ' || body.back() == '\n')) body.pop_back();
      if (!body.empty() && body[0] == ',') body.erase(0, 1);
    }
    while (!body.empty() && (body.back() == ' ' || body.back() == '\n')) body.pop_back();
    if (!body.empty()) body += ",\n ";
    body += pat + " " + std::to_string(val);
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos && slash > 0) mkdir_p(path.substr(0, slash));
    if (FILE* f = std::fopen(path.c_str(), "w")) {
      std::fprintf(f, "{%s}\n", body.c_str());
      std::fclose(f);
    }
  }
  static void mkdir_p(const std::string& d) {
    std::string cur;
    for (size_t i = 0; i < d.size(); ++i) {
      cur += d[i];
      if (d[i] == '/' && cur.size() > 1) ::mkdir(cur.c_str(), 0755);
    }
    ::mkdir(d.c_str(), 0755);
  }

  // The cached value encodes the mode: 4 G + m, m = 0 one stream, 1 two streams (G planes per
  // group), 2 the pipeline (G = ring planes, lag G / 4), 3 the cluster pass (G = 1 + its
  // thread-count variant).
  void set_mode(int g, int m) {
    pipe = m == 2;
    clus = m == 3;
    if (clus) {
      cl_var = g == 2 ? 1 : 0;  // G field: 1 = 384 threads, 2 = 768 threads
      return;
    }
    if (pipe) {
      pipe_ring = g;
      pipe_lag = g / 4 > 0 ? g / 4 : 1;
    } else {
      G = g;
      slab_streams = m + 1;
    }
  }
  void autotune() {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    tuned = true;
    if (const char* e = std::getenv("NS_PIPE_SPIN")) pipe_spin = std::max(1ll, std::atoll(e));
    if (const char* e = std::getenv("NS_PIPE_TEST_STALL")) pipe_stall = std::atoi(e) ? 1 : 0;
    if (const char* e = std::getenv("NS_CL_SPIN")) cl_spin = std::max(1ll, std::atoll(e));
    // NS_TILE_VARIANT=bits forces the compiled tile alternatives (bits of K2Cfg's variant)
    const char* fv = std::getenv("NS_TILE_VARIANT");
    if (fv && *fv) vsel = (use2 && k2.has_alt) ? (std::atoi(fv) & 31) : 0;
    const char* fcl = std::getenv("NS_SLAB_CLUSTER");
    const bool can_cl = use2 && k2.slabcl[0] && !(fcl && std::string(fcl) == "0") && cl_clusters() > 0;
    if (fcl && std::string(fcl) == "1" && can_cl) {  // forced cluster pass (NS_CL_VARIANT 0 or 1)
      const char* fv = std::getenv("NS_CL_VARIANT");
      set_mode(fv && std::atoi(fv) == 0 ? 1 : 2, 3);
      return;
    }
    const char* fpipe = std::getenv("NS_SLAB_PIPE");
    const bool can_pipe = use2 && k2.slabpipe && !(fpipe && std::string(fpipe) == "0");
    if (fpipe && std::string(fpipe) == "1" && can_pipe) {  // forced pipeline
      const char* fr = std::getenv("NS_PIPE_RING");
      int r = fr ? std::atoi(fr) : 32;
      r = std::max(2, std::min(r, std::min(Gmax, N)));
      set_mode(r, 2);
      if (const char* fl = std::getenv("NS_PIPE_LAG")) pipe_lag = std::max(1, std::atoi(fl));
      if (2 * pipe_lag >= pipe_ring) pipe_lag = (pipe_ring - 1) / 2 > 0 ? (pipe_ring - 1) / 2 : 1;
      return;
    }
    if (const char* fs = std::getenv("NS_SLAB_STREAMS")) slab_streams = std::atoi(fs) == 2 ? 2 : 1;
    if (const char* fg = std::getenv("NS_SLAB_PLANES")) {  // forced group size
      const int g = std::atoi(fg);
      if (g >= 1) G = g < Gmax ? g : Gmax;
      return;
    }
    const char* en = std::getenv("NS_AUTOTUNE");
    if (en && std::string(en) == "0") return;
    if (Gmax <= 1 || N < 128) return;  // small grids: one group holds every plane
    const bool can_alt = use2 && k2.has_alt && !(fv && *fv);
    const std::string path = cache_path(),
                      key = tune_key() + (can_pipe ? "|g4p" : "|g4") + (can_cl ? "c" + std::to_string(k2.CLS) : "") +
                            (can_alt ? "|v" + std::to_string(k2.alt.TX) + "," + std::to_string(k2.alt.TYI) + "," +
                                           std::to_string(k2.alt.RX) + "," + std::to_string(k2.alt.TY) + ",p64"
                                     : "");
    int g = 0;
    if (cache_lookup(path, key, &g)) {  // value = 4096 vsel + 4 G + mode
      const int gm = g % 4096, vs = g / 4096;
      if (gm / 4 >= 1 && gm / 4 <= Gmax && ((gm & 3) <= 2 || can_cl) && (vs == 0 || can_alt)) {
        set_mode(gm / 4, gm & 3);
        if (can_alt) vsel = vs;
        return;
      }
    }
    std::vector<std::pair<int, int>> cand;  // (G or ring, mode)
    for (int q : {8, 12, 16, 19, 24, 28, 32, 38, 43, 48, 57, 64, 76, 96, 128, 171, 256, 384, 512, 768}) {
      if (q > Gmax) continue;
      cand.push_back({q, 0});
      if (q < N && 2 * q <= Gmax) cand.push_back({q, 1});  // two streams need two groups
    }
    if (can_pipe)
      for (int r : {16, 24, 32, 48})
        if (r <= Gmax && r <= N) cand.push_back({r, 2});
    if (can_cl)
      for (int v = 0; v < 2; ++v) cand.push_back({1 + v, 3});
    if (cand.empty()) return;
    CUDA_TRY(cudaMemsetAsync(mixed[0], 0, 5 * F1 * sizeof(cpx<T>), st));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const bool pon = prof.on;
    prof.on = false;
    float best = 1e30f;
    std::pair<int, int> bestc = {G, 0};
    for (const auto& cm : cand) {
      set_mode(cm.first, cm.second);
      slab(mixed[0], Ft[0]);  // warm-up
      CUDA_TRY(cudaEventRecord(e0, st));
      for (int r = 0; r < 8; ++r) slab(mixed[0], Ft[0]);
      CUDA_TRY(cudaEventRecord(e1, st));
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0;
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bestc = cm;
      }
    }
    sync_check();  // a pipeline candidate that gave up reports here
    pipe = false;
    clus = false;
    set_mode(bestc.first, bestc.second);
    // the compiled tile alternatives, one kernel family at a time: the slab kernels in the
    // chosen slab mode (three-kernel modes only), the pencil on the Rogallo stages
    if (can_alt) {
      auto time_slab = [&]() {
        slab(mixed[0], Ft[0]);
        CUDA_TRY(cudaEventRecord(e0, st));
        for (int r = 0; r < 8; ++r) slab(mixed[0], Ft[0]);
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
      };
      if (!pipe && !clus) {
        float base = time_slab();
        for (int bit : {2, 4, 8}) {
          vsel ^= bit;
          const float ms = time_slab();
          if (ms < base) base = ms;
          else vsel ^= bit;
        }
      }
      // pencil: both Rogallo stages on the work buffers (acc as the state, Ft[0] as the input,
      // mixed[0] as the output; all recomputed before any step uses them), zero inputs
      CUDA_TRY(cudaMemsetAsync(acc, 0, 3 * F1 * sizeof(cpx<T>), st));
      CUDA_TRY(cudaMemsetAsync(Ft[0], 0, 3 * F1 * sizeof(cpx<T>), st));
      cpx<T>* pout = mixed[0];
      auto time_pencil = [&]() {
        PencilArgs<T> a = pencil_args(MODE_ROG_1);
        a.shell = nullptr;
        a.state = acc;
        a.nF = 1; a.F[0] = Ft[0]; a.wF[0] = (T)1;
        a.nOut = 1; a.out[0] = pout;
        pencil(a);
        CUDA_TRY(cudaEventRecord(e0, st));
        for (int r = 0; r < 8; ++r) {
          a.mode = (r & 1) ? MODE_ROG_2 : MODE_ROG_1;
          pencil(a);
        }
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        return ms;
      };
      float pbest = time_pencil();
      for (int bit : {1, 16}) {  // the pencil alternatives are exclusive
        vsel ^= bit;
        const float ms = time_pencil();
        if (ms < pbest) {
          pbest = ms;
          vsel &= ~(bit == 1 ? 16 : 1);
        } else {
          vsel ^= bit;
        }
      }
      sync_check();
    }
    prof.on = pon;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cache_store(path, key, 4096 * vsel + 4 * bestc.first + bestc.second);
  }

  // ---- schemes ------------------------------------------------------------------------
  void invalidate_carry() override { carry_step = -1; }

  void step_cfl(double cfl_, double dt_max, int nsteps) override {
    cfl = cfl_;
    cfl_dtmax = dt_max;
    try {
      step(dt_max, nsteps);
    } catch (...) {
      cfl = 0.0;
      throw;
    }
    cfl = 0.0;
  }

  void step(double dt, int nsteps) override {
    if (!tuned) autotune();
    set_dt(dt);
    const int sch = c->p.scheme;
    const double dx = 2.0 * M_PI / N;
    const int CH = 256;  // steps per chunk of shift tables
    for (int s0 = 0; s0 < nsteps; s0 += CH) {
      const int ns = (s0 + CH <= nsteps) ? CH : nsteps - s0;
      const bool last_chunk = s0 + ns == nsteps;
      if (fkind != NS_FORCE_NONE) prepare_forcing(c->t, c->t + ns * dt);
      if (sch == NS_RK2_PS_RANDOM || sch == NS_RK2_PS_APPROX) {
        // shift vectors: [2n] alpha_n, [2n+1] beta_n, and alpha of the step after the chunk
        // (read without consuming an override shift) for the carried mixed fields
        std::vector<double> sh(6 * (size_t)ns + 3);
        for (int n = 0; n <= ns; ++n) {
          double da[3] = {0, 0, 0};
          if (sch == NS_RK2_PS_RANDOM) {
            if (c->override_pos < c->override_shifts.size()) {
              for (int i = 0; i < 3; ++i) da[i] = c->override_shifts[c->override_pos + i];
              if (n < ns) c->override_pos += 3;
            } else {
              for (int i = 0; i < 3; ++i)
                da[i] = dx * uniform01(c->p.seed, (uint64_t)(3 * (c->step + n) + i));
            }
          }
          for (int i = 0; i < 3; ++i) {
            sh[6 * n + i] = da[i];
            if (n < ns) sh[6 * n + 3 + i] = da[i] + 0.5 * dx;
          }
        }
        upload_shifts(sh);
        run_rogallo(dt, ns, sch == NS_RK2_PS_APPROX);
      } else if (sch == NS_RK2_PS_EXACT) {
        std::vector<double> sh = {0.5 * dx, 0.5 * dx, 0.5 * dx};
        upload_shifts(sh);
        run_rk2(dt, ns, true);
      } else if (sch == NS_RK2) {
        run_rk2(dt, ns, false);
      } else {
        run_rk4(dt, ns);
      }
      (void)last_chunk;
    }
    // stream-ordered: device-side checks are reported by the next synchronising call
  }

  void init_pass(int nOut, const cpx<T>* o0, const cpx<T>* o1) {
    PencilArgs<T> a = pencil_args(MODE_INIT);
    a.src = state;
    a.nOut = nOut;
    a.osh[0] = o0; a.out[0] = mixed[0];
    a.osh[1] = o1; a.out[1] = mixed[1];
    pencil(a);
  }

  // time step of the coming step: fixed, or from the maxima of the velocity that the step's
  // first slab pass has just formed (adaptive: one read-back per step)
  double step_dt(double dt) {
    if (cfl <= 0.0) return dt;
    // the kernels fold the maxima into T-sized words: unsigned[3] (FP32) or uint64[3] (FP64)
    unsigned char h[3 * sizeof(unsigned long long)];
    CUDA_TRY(cudaMemcpyAsync(h, d_umax, 3 * sizeof(T), cudaMemcpyDeviceToHost, st));
    sync_check();
    double freq = 0.0;
    for (int i = 0; i < 3; ++i) {
      T m;
      std::memcpy(&m, h + i * sizeof(T), sizeof(T));
      freq += (double)m / (2.0 * M_PI / N);
    }
    double d = freq > 0.0 ? cfl / freq : cfl_dtmax;
    if (d > cfl_dtmax) d = cfl_dtmax;
    set_dt(d);
    return d;
  }

  void run_rogallo(double dt0, int ns, bool approx) {
    const T w = (T)(1.0 / ((double)N * N * N));
    auto alpha = [&](int n) -> const cpx<T>* { return approx ? nullptr : shift_tab(2 * n); };
    auto beta = [&](int n) -> const cpx<T>* { return shift_tab(2 * n + 1); };
    if (carry_step != c->step) init_pass(1, alpha(0), nullptr);
    for (int n = 0; n < ns; ++n) {
      const double t = c->t;
      slab(mixed[0], Ft[0], cfl > 0.0);
      const double dt = step_dt(dt0);
      PencilArgs<T> a = pencil_args(MODE_ROG_1);
      force_coef(t, a);
      a.nF = 1; a.F[0] = Ft[0]; a.dsh[0] = alpha(n); a.wF[0] = w;
      a.nOut = 1; a.osh[0] = beta(n); a.out[0] = mixed[0];
      pencil(a);
      slab(mixed[0], Ft[0]);
      PencilArgs<T> b = pencil_args(MODE_ROG_2);
      force_coef(t + dt, b);
      b.nF = 1; b.F[0] = Ft[0]; b.dsh[0] = beta(n); b.wF[0] = w;
      b.nOut = 1;  // the last step of the chunk prepares the step after it
      b.osh[0] = alpha(n + 1);
      b.out[0] = mixed[0];
      final_pencil(b);
      c->t = t + dt;
      c->step += 1;
    }
    carry_step = c->step;
  }

  void run_rk2(double dt0, int ns, bool exact) {
    const T w = (T)(1.0 / ((double)N * N * N));
    const cpx<T>* iso = exact ? shift_tab(0) : nullptr;
    if (carry_step != c->step) init_pass(exact ? 2 : 1, nullptr, iso);
    for (int n = 0; n < ns; ++n) {
      const double t = c->t;
      double dt = dt0;
      for (int stg = 0; stg < 2; ++stg) {
        slab(mixed[0], Ft[0], stg == 0 && cfl > 0.0);
        if (stg == 0) dt = step_dt(dt0);
        if (exact) slab(mixed[1], Ft[1]);
        PencilArgs<T> a = pencil_args(stg == 0 ? MODE_RK2_1 : MODE_RK2_2);
        force_coef(stg == 0 ? t : t + 0.5 * dt, a);
        a.nF = exact ? 2 : 1;
        a.F[0] = Ft[0]; a.dsh[0] = nullptr; a.wF[0] = exact ? (T)0.5 * w : w;
        a.F[1] = Ft[1]; a.dsh[1] = iso; a.wF[1] = (T)0.5 * w;
        a.nOut = exact ? 2 : 1;  // the last pass prepares the next step
        a.osh[0] = nullptr; a.out[0] = mixed[0];
        a.osh[1] = iso; a.out[1] = mixed[1];
        if (stg == 1)
          final_pencil(a);
        else
          pencil(a);
      }
      c->t = t + dt;
      c->step += 1;
    }
    carry_step = c->step;
  }

  void run_rk4(double dt0, int ns) {
    const T w = (T)(1.0 / ((double)N * N * N));
    if (carry_step != c->step) init_pass(1, nullptr, nullptr);
    const int modes[4] = {MODE_RK4_1, MODE_RK4_2, MODE_RK4_3, MODE_RK4_4};
    const double ts[4] = {0.0, 0.5, 0.5, 1.0};
    for (int n = 0; n < ns; ++n) {
      const double t = c->t;
      double dt = dt0;
      for (int stg = 0; stg < 4; ++stg) {
        slab(mixed[0], Ft[0], stg == 0 && cfl > 0.0);
        if (stg == 0) dt = step_dt(dt0);
        PencilArgs<T> a = pencil_args(modes[stg]);
        force_coef(t + ts[stg] * dt, a);
        a.nF = 1; a.F[0] = Ft[0]; a.wF[0] = w;
        a.nOut = 1;  // the last pass prepares the next step
        a.out[0] = mixed[0];
        if (stg == 3)
          final_pencil(a);
        else
          pencil(a);
      }
      c->t = t + dt;
      c->step += 1;
    }
    carry_step = c->step;
  }

  // ---- transfers ----------------------------------------------------------------------
  // Host FP64 <-> device T arrays of n reals.  FP64 contexts copy; FP32 contexts copy the FP64
  // values through the slab scratch (in chunks of its size) and convert them on the device, so
  // the host only copies (the conversions round as the host's casts do).
  size_t stage_doubles() const { return 6 * (size_t)Gmax * N * M * sizeof(cpx<T>) / sizeof(double); }
  void to_device(const double* h, T* d, size_t n) {
    if constexpr (sizeof(T) == sizeof(double)) {
      CUDA_TRY(cudaMemcpyAsync(d, h, n * sizeof(double), cudaMemcpyHostToDevice, st));
    } else {
      double* stg = reinterpret_cast<double*>(scr);
      const size_t cap = stage_doubles();
      for (size_t o = 0; o < n; o += cap) {
        const size_t m = n - o < cap ? n - o : cap;
        CUDA_TRY(cudaMemcpyAsync(stg, h + o, m * sizeof(double), cudaMemcpyHostToDevice, st));
        k_real_from_double<T><<<8 * nsm, 256, 0, st>>>(stg, d + o, m);
        LAUNCH_CHECK();
      }
    }
  }
  // the device address of a page-locked host buffer (written by kernels directly), or null
  bool zero_copy = true;  // NS_ZERO_COPY=0: always stage and copy
  double* host_device_view(double* h) {
    if (!zero_copy) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer ? static_cast<double*>(at.devicePointer) : nullptr;
  }
  void to_host(const T* d, double* h, size_t n) {
    if constexpr (sizeof(T) == sizeof(double)) {
      CUDA_TRY(cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else if (double* hd = host_device_view(h)) {
      // page-locked destination: the conversion kernel stores into it over the host link
      k_real_to_double<T><<<8 * nsm, 256, 0, st>>>(d, hd, n);
      LAUNCH_CHECK();
    } else {
      double* stg = reinterpret_cast<double*>(scr);
      const size_t cap = stage_doubles();
      for (size_t o = 0; o < n; o += cap) {
        const size_t m = n - o < cap ? n - o : cap;
        k_real_to_double<T><<<8 * nsm, 256, 0, st>>>(d + o, stg, m);
        LAUNCH_CHECK();
        CUDA_TRY(cudaMemcpyAsync(h + o, stg, m * sizeof(double), cudaMemcpyDeviceToHost, st));
      }
    }
  }

  // physical reals [3][N][N][N] of T on the device -> wscale P T F(u) (unnormalised r2c of
  // x and y, z in the pencil; projection, truncation and k = 0 removed) into dst
  void r2c_project(const T* rin, cpx<T>* dst, double wscale) {
    SlabArgs<T> a = slab_args();
    a.rio = const_cast<T*>(rin);
    a.Ft = Ft[0];
    a.xmode = XMODE_R2C;
    for (int z0 = 0; z0 < N; z0 += G) {
      a.z0 = z0;
      a.G = (z0 + G <= N) ? G : N - z0;
      k_xrow<T><<<(a.G * N + RX - 1) / RX, bdX, smX, st>>>(a);
      k_yfwd<T><<<dim3(M / TY, a.G), bdYf, smYf, st>>>(a);
    }
    LAUNCH_CHECK();
    PencilArgs<T> p = pencil_args(MODE_PROJECT);
    p.shell = nullptr;
    p.nF = 1; p.F[0] = Ft[0]; p.wF[0] = (T)wscale;
    p.state = dst;
    pencil(p);
  }
  // spectral src -> physical reals [3][N][N][N] of T on the device (inverse z, y, x)
  void c2r(const cpx<T>* src, T* rout) {
    PencilArgs<T> p = pencil_args(MODE_INIT);
    p.shell = nullptr;
    p.src = src;
    p.nOut = 1; p.out[0] = mixed[0];
    pencil(p);
    SlabArgs<T> a = slab_args();
    a.mixed = mixed[0];
    a.rio = rout;
    a.xmode = XMODE_C2R;
    for (int z0 = 0; z0 < N; z0 += G) {
      a.z0 = z0;
      a.G = (z0 + G <= N) ? G : N - z0;
      k_yinv<T><<<dim3(M / TY, a.G), bdYi, smYi, st>>>(a);
      k_xrow<T><<<(a.G * N + RX - 1) / RX, bdX, smX, st>>>(a);
    }
    LAUNCH_CHECK();
  }

  void set_velocity(const double* u) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    T* rin = reinterpret_cast<T*>(mixed[0]);  // 5 N^3 reals >= 3 N^3
    to_device(u, rin, 3 * (size_t)N * N * N);
    r2c_project(rin, state, 1.0 / ((double)N * N * N));
    sync_check();
  }

  void get_velocity(double* u) override { to_physical(state, u); }

  // spectral [3][N][N][M] -> physical host [3][N][N][N] (inverse z, y, x transforms)
  void to_physical(const cpx<T>* src, double* u) {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    T* rout = reinterpret_cast<T*>(Ft[0]);  // 3 N^3 reals
    c2r(src, rout);
    to_host(rout, u, 3 * (size_t)N * N * N);
    sync_check();
  }

  // spectral [3][N][N][M] complex <-> host re_im[...][2] (the same layout as reals)
  void download(const cpx<T>* src, double* out) {
    to_host(reinterpret_cast<const T*>(src), out, 2 * 3 * F1);
    sync_check();
  }

  void upload(const double* in, cpx<T>* dst) {
    to_device(in, reinterpret_cast<T*>(dst), 2 * 3 * F1);
    CUDA_TRY(cudaStreamSynchronize(st));
  }

  void get_state(double* s) override { download(state, s); }
  void raw_state(std::vector<unsigned char>& out) override {
    out.resize(3 * F1 * sizeof(cpx<T>));
    CUDA_TRY(cudaMemcpyAsync(out.data(), state, out.size(), cudaMemcpyDeviceToHost, st));
    sync_check();
  }
  void set_raw_state(const unsigned char* in, size_t n) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    if (n != 3 * F1 * sizeof(cpx<T>)) throw NsError{NS_ERR_IO, "checkpoint state size mismatch"};
    CUDA_TRY(cudaMemcpyAsync(state, in, n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
  }
  void forcing_params(int* kind, double* v, uint64_t* seed) override {
    *kind = fkind;
    v[0] = fkmin; v[1] = fkmax; v[2] = feps; v[3] = ftcorr;
    *seed = fseed;
  }
  void set_state(const double* s) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    upload(s, state);
  }

  void nonlinear(const double* in, const double* delta, double* out) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    const cpx<T>* src = state;
    if (in) {
      upload(in, acc);
      src = acc;
    }
    std::vector<double> sh(delta, delta + 3);
    upload_shifts(sh);
    PencilArgs<T> p = pencil_args(MODE_INIT);
    p.shell = nullptr;
    p.src = src;
    p.nOut = 1; p.osh[0] = shift_tab(0); p.out[0] = mixed[0];
    pencil(p);
    slab(mixed[0], Ft[0]);
    PencilArgs<T> q = pencil_args(MODE_NL);
    q.shell = nullptr;
    q.nF = 1; q.F[0] = Ft[0]; q.dsh[0] = shift_tab(0); q.wF[0] = (T)(1.0 / ((double)N * N * N));
    pencil(q);
    download(acc, out);
  }

  // ---- adjoint (transposed linearisation) of the RK2 phase-shift random / split step ----
  // Formulas: oracle-independent restatement in include/ns.h (ns_vjp).  Buffers are
  // allocated on first use and kept by the context.
  std::vector<cpx<T>*> adj;  // work vectors of 3 fields
  cpx<T>* mixedB = nullptr;
  cpx<T>* FtB = nullptr;
  cpx<T>* shS = nullptr;
  cpx<T>* shR = nullptr;
  cpx<T>* ftab = nullptr;

  cpx<T>* vec(int i) { return adj[i]; }

  void ew(int op, const cpx<T>* x, const cpx<T>* y, const cpx<T>* z, cpx<T>* o, double c = 0.0) {
    k_elementwise<T><<<4 * nsm, 256, 0, st>>>(op, N, (T)cur_dt, (T)c, ifac, x, y, z, o);
    LAUNCH_CHECK();
  }

  // Nt_D(S) -> out  (D = shift table or null)
  void nl_eval(const cpx<T>* S, const cpx<T>* tab, cpx<T>* out) {
    PencilArgs<T> p = pencil_args(MODE_INIT);
    p.shell = nullptr;
    p.src = S;
    p.nOut = 1; p.osh[0] = tab; p.out[0] = mixed[0];
    pencil(p);
    slab(mixed[0], Ft[0]);
    PencilArgs<T> q = pencil_args(MODE_NL);
    q.shell = nullptr;
    q.acc = out;
    q.nF = 1; q.F[0] = Ft[0]; q.dsh[0] = tab; q.wF[0] = (T)(1.0 / ((double)N * N * N));
    pencil(q);
  }

  // slab pass of an adjoint cross product with the generic kernels
  void slab_adj(int xmode, cpx<T>* out) {
    SlabArgs<T> a = slab_args();
    a.mixed = mixed[0];
    a.mixedB = mixedB;
    a.Ft = out;
    a.xmode = xmode;
    for (int z0 = 0; z0 < N; z0 += G) {
      a.z0 = z0;
      a.G = (z0 + G <= N) ? G : N - z0;
      k_yinv<T><<<dim3(M / TY, a.G), bdYi, smYi, st>>>(a);
      k_xrow<T><<<(a.G * N + RX - 1) / RX, bdX, smX, st>>>(a);
      k_yfwd<T><<<dim3(M / TY, a.G), bdYf, smYf, st>>>(a);
    }
    LAUNCH_CHECK();
  }

  // J*(rho) at state S for shift table tab: T P e^{-ikD}[F(w x r) + ik x F(r x u)]
  void nl_vjp(const cpx<T>* S, const cpx<T>* tab, const cpx<T>* rho, cpx<T>* out, cpx<T>* tmpA,
              cpx<T>* tmpB) {
    PencilArgs<T> p = pencil_args(MODE_INIT);
    p.shell = nullptr;
    p.src = S;
    p.nOut = 1; p.osh[0] = tab; p.out[0] = mixed[0];
    pencil(p);
    p.src = rho;
    p.out[0] = mixedB;
    pencil(p);
    slab_adj(XMODE_ADJ_WR, Ft[0]);
    slab_adj(XMODE_ADJ_RU, FtB);
    PencilArgs<T> q = pencil_args(MODE_NL);
    q.shell = nullptr;
    q.nF = 1; q.dsh[0] = tab; q.wF[0] = (T)(1.0 / ((double)N * N * N));
    q.F[0] = Ft[0]; q.acc = tmpA;
    pencil(q);
    q.F[0] = FtB; q.acc = tmpB;
    pencil(q);
    ew(EW_CURL_ADD, tmpA, tmpB, nullptr, out);
  }

  const cpx<double>* pattern_ptr(double ts, double* theta) {
    const double x = ts / ftcorr;
    const int64_t j = (int64_t)std::floor(x);
    *theta = x - (double)j;
    if (j < fj0 || j - fj0 + 1 >= fpat_cap)
      throw NsError{NS_ERR_INTERNAL, "forcing pattern index out of the prepared range"};
    return fpat + (size_t)(j - fj0) * 3 * fDn();
  }

  // out += O(S) at time ts
  void add_forcing(const cpx<T>* S, double ts, cpx<T>* out) {
    if (fkind == NS_FORCE_NONE) return;
    double th;
    const cpx<double>* pj = pattern_ptr(ts, &th);
    k_shell_gather<T><<<1, 256, 0, st>>>(S, N, fK, shS);
    k_force_coef<T><<<1, 256, 0, st>>>(pj, pj + 3 * fDn(), th, shS, fK, cur_dt, feps, ftab, nullptr);
    k_shell_add<T><<<1, 256, 0, st>>>(out, N, fK, ftab);
    LAUNCH_CHECK();
  }

  // out += (dO/dS at S, time ts)^T rho
  void add_forcing_vjp(const cpx<T>* S, double ts, const cpx<T>* rho, cpx<T>* out) {
    if (fkind == NS_FORCE_NONE) return;
    double th;
    const cpx<double>* pj = pattern_ptr(ts, &th);
    k_shell_gather<T><<<1, 256, 0, st>>>(S, N, fK, shS);
    k_shell_gather<T><<<1, 256, 0, st>>>(rho, N, fK, shR);
    k_force_vjp<T><<<1, 256, 0, st>>>(pj, pj + 3 * fDn(), th, shS, shR, fK, cur_dt, feps, ftab);
    k_shell_add<T><<<1, 256, 0, st>>>(out, N, fK, ftab);
    LAUNCH_CHECK();
  }

  // Work vectors and tables of an adjoint run of nsteps steps with a checkpoint every ckpt
  // steps (kept by the context; a tape_forward leaves them for tape_backward).
  struct Tape {
    bool valid = false;
    int nsteps = 0, ckpt = 0;
    double dt = 0.0;
  } tape;
  void adj_alloc(int nsteps, int ckpt) {
    const size_t vb = 3 * F1 * sizeof(cpx<T>);
    const int nck = (nsteps + ckpt - 1) / ckpt + 1;
    const int nvec = 12 + ckpt + nck + 1;  // work, segment states, checkpoints, S_T
    if ((int)adj.size() < nvec) {
      for (auto* p : adj) cudaFree(p);
      adj.assign(nvec, nullptr);
      for (int i = 0; i < nvec; ++i) CUDA_TRY(cudaMalloc(&adj[i], vb));
    }
    if (!mixedB) CUDA_TRY(cudaMalloc(&mixedB, 5 * F1 * sizeof(cpx<T>)));
    if (!FtB) CUDA_TRY(cudaMalloc(&FtB, 3 * F1 * sizeof(cpx<T>)));
    if (fkind != NS_FORCE_NONE) {
      cudaFree(shS); cudaFree(shR); cudaFree(ftab);
      shS = shR = ftab = nullptr;
      CUDA_TRY(cudaMalloc(&shS, 3 * (size_t)fDn() * sizeof(cpx<T>)));
      CUDA_TRY(cudaMalloc(&shR, 3 * (size_t)fDn() * sizeof(cpx<T>)));
      CUDA_TRY(cudaMalloc(&ftab, 3 * (size_t)fDn() * sizeof(cpx<T>)));
    }
  }
  // shift tables of steps 0 .. nsteps-1 (context seed, step counter from 0), forcing record
  // over [0, nsteps dt]; the step times
  std::vector<double> adj_tables(int nsteps, double dt) {
    set_dt(dt);
    const double dx = 2.0 * M_PI / N;
    const bool approx = c->p.scheme == NS_RK2_PS_APPROX;
    std::vector<double> sh(6 * (size_t)nsteps);
    for (int n = 0; n < nsteps; ++n)
      for (int i = 0; i < 3; ++i) {
        const double da = approx ? 0.0 : dx * uniform01(c->p.seed, (uint64_t)(3 * n + i));
        sh[6 * n + i] = da;
        sh[6 * n + 3 + i] = da + 0.5 * dx;
      }
    upload_shifts(sh);
    std::vector<double> times(nsteps + 1, 0.0);
    for (int n = 0; n < nsteps; ++n) times[n + 1] = times[n] + dt;
    if (fkind != NS_FORCE_NONE) prepare_forcing(0.0, times[nsteps]);
    return times;
  }
  // one forward step of the adjoint's scheme (the same arithmetic as the stepping kernels,
  // as separate evaluations): S0 -> Sout, stage state in S1
  void adj_step(const cpx<T>* S0, cpx<T>* Sout, int n, double dt, const std::vector<double>& times) {
    cpx<T>* N0 = vec(0);
    cpx<T>* N1 = vec(1);
    cpx<T>* S1 = vec(2);
    nl_eval(S0, shift_tab(2 * n), N0);
    add_forcing(S0, times[n], N0);
    ew(EW_ROG_S1, S0, N0, nullptr, S1);
    nl_eval(S1, shift_tab(2 * n + 1), N1);
    add_forcing(S1, times[n] + dt, N1);
    ew(EW_ROG_SN, S0, N0, N1, Sout);
  }
  // forward sweep from `state` with the state kept every ckpt steps; leaves state = S_T
  void adj_forward(int nsteps, double dt, int ckpt) {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    adj_alloc(nsteps, ckpt);
    const std::vector<double> times = adj_tables(nsteps, dt);
    const size_t vb = 3 * F1 * sizeof(cpx<T>);
    cpx<T>* tmp = vec(11);
    cpx<T>** ck = &adj[12 + ckpt];
    CUDA_TRY(cudaMemcpyAsync(ck[0], state, vb, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(tmp, state, vb, cudaMemcpyDeviceToDevice, st));
    for (int n = 0; n < nsteps; ++n) {
      adj_step(tmp, tmp, n, dt, times);
      if ((n + 1) % ckpt == 0 && n + 1 < nsteps)
        CUDA_TRY(cudaMemcpyAsync(ck[(n + 1) / ckpt], tmp, vb, cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaMemcpyAsync(state, tmp, vb, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(adj[12 + ckpt + (nsteps + ckpt - 1) / ckpt + 1], tmp, vb,
                             cudaMemcpyDeviceToDevice, st));  // S_T of the tape
    tape.valid = true;
    tape.nsteps = nsteps;
    tape.ckpt = ckpt;
    tape.dt = dt;
    c->t = times[nsteps];
    c->step = nsteps;
  }
  // reverse sweep: lam holds the cotangent of S_T on entry and that of S_0 on exit; the
  // states of each segment are recomputed from its checkpoint
  void adj_reverse(cpx<T>* lam) {
    const int nsteps = tape.nsteps, ckpt = tape.ckpt;
    const double dt = tape.dt;
    const std::vector<double> times = adj_tables(nsteps, dt);  // (the tables may have changed)
    const size_t vb = 3 * F1 * sizeof(cpx<T>);
    cpx<T>* N0 = vec(0);
    cpx<T>* S1 = vec(2);
    cpx<T>* mu = vec(4);
    cpx<T>* rho = vec(5);
    cpx<T>* sig = vec(6);
    cpx<T>* rs = vec(7);
    cpx<T>* J = vec(8);
    cpx<T>* tA = vec(9);
    cpx<T>* tB = vec(10);
    cpx<T>** seg = &adj[12];
    cpx<T>** ck = &adj[12 + ckpt];
    for (int seg0 = ((nsteps - 1) / ckpt) * ckpt; seg0 >= 0; seg0 -= ckpt) {
      const int seg1 = seg0 + ckpt < nsteps ? seg0 + ckpt : nsteps;
      CUDA_TRY(cudaMemcpyAsync(seg[0], ck[seg0 / ckpt], vb, cudaMemcpyDeviceToDevice, st));
      for (int n = seg0; n < seg1 - 1; ++n) adj_step(seg[n - seg0], seg[n - seg0 + 1], n, dt, times);
      for (int n = seg1 - 1; n >= seg0; --n) {
        const cpx<T>* S0 = seg[n - seg0];
        const cpx<T>* ta = shift_tab(2 * n);
        const cpx<T>* tb = shift_tab(2 * n + 1);
        nl_eval(S0, ta, N0);
        add_forcing(S0, times[n], N0);
        ew(EW_ROG_S1, S0, N0, nullptr, S1);
        ew(EW_RHO, lam, nullptr, nullptr, rho);
        nl_vjp(S1, tb, rho, mu, tA, tB);
        add_forcing_vjp(S1, times[n] + dt, rho, mu);
        ew(EW_SIGMA, mu, nullptr, nullptr, sig);
        ew(EW_ADD, rho, sig, nullptr, rs);
        nl_vjp(S0, ta, rs, J, tA, tB);
        add_forcing_vjp(S0, times[n], rs, J);
        ew(EW_LAMBDA, lam, mu, J, lam);
      }
    }
  }
  // cotangent of S_T of a built-in loss of the final state S (E: S; eps: 2 nu k^2 S)
  void adj_loss_seed(int loss, const cpx<T>* S, cpx<T>* lam) {
    if (loss == NS_LOSS_ENERGY)
      ew(EW_SCALE, S, nullptr, nullptr, lam, 1.0);
    else
      ew(EW_LOSS, S, nullptr, nullptr, lam, c->p.nu);
  }

  void vjp(const double* u0, int nsteps, double dt, int ckpt, int loss, double* Lout,
           double* grad) override {
    set_velocity(u0);
    adj_forward(nsteps, dt, ckpt);
    cpx<T>* lam = vec(3);
    double E, eps;
    energy(&E, &eps);
    *Lout = loss == NS_LOSS_ENERGY ? E : eps;
    adj_loss_seed(loss, state, lam);
    adj_reverse(lam);
    // dL/du0 = F^{-1}(lambda_0) / N^3 (the initial truncation and projection are
    // self-adjoint and lambda_0 already lies in their range)
    cpx<T>* tmp = vec(11);
    ew(EW_SCALE, lam, nullptr, nullptr, tmp, 1.0 / ((double)N * N * N));
    to_physical(tmp, grad);
    tape.valid = false;  // the work vectors were reused for the output
  }

  // Gradient of a loss on the final velocity u(T) = F^{-1}(S_T), given gT = dL/du(T): the
  // cotangent of S_T is N^3 P T F(gT) (F: forward transform with the 1/N^3 factor; its
  // adjoint for <a,b> = sum_k Re(conj(a).b) over the full spectrum is F^{-1} / N^3).
  void vjp_state(const double* u0, int nsteps, double dt, int ckpt, const double* gT,
                 double* grad) override {
    set_velocity(u0);
    adj_forward(nsteps, dt, ckpt);
    cpx<T>* lam = vec(3);
    T* rin = reinterpret_cast<T*>(mixed[0]);
    to_device(gT, rin, 3 * (size_t)N * N * N);
    r2c_project(rin, lam, 1.0);
    adj_reverse(lam);
    cpx<T>* tmp = vec(11);
    ew(EW_SCALE, lam, nullptr, nullptr, tmp, 1.0 / ((double)N * N * N));
    to_physical(tmp, grad);
    tape.valid = false;
  }

  // device-buffer forms (the autograd path): u0, uT [3][N][N][N] reals of T on the device
  void tape_forward(const void* u0, int nsteps, double dt, int ckpt, void* uT) override {
    carry_step = -1;
    r2c_project(static_cast<const T*>(u0), state, 1.0 / ((double)N * N * N));
    adj_forward(nsteps, dt, ckpt);
    c2r(state, static_cast<T*>(uT));
    sync_check();
  }
  // gT: the cotangent of u(T) (device reals of T), or null for the built-in loss `loss`
  void tape_backward(const void* gT, int loss, void* grad) override {
    if (!tape.valid) throw NsError{NS_ERR_STATE, "no adjoint tape: call ns_tape_forward first"};
    carry_step = -1;
    cpx<T>* lam = vec(3);
    if (gT)
      r2c_project(static_cast<const T*>(gT), lam, 1.0);
    else
      adj_loss_seed(loss, adj[12 + tape.ckpt + (tape.nsteps + tape.ckpt - 1) / tape.ckpt + 1], lam);
    adj_reverse(lam);
    cpx<T>* tmp = vec(11);
    ew(EW_SCALE, lam, nullptr, nullptr, tmp, 1.0 / ((double)N * N * N));
    c2r(tmp, static_cast<T*>(grad));
    sync_check();
  }

  void energy(double* E, double* eps) override {
    const int nb = red_blocks;
    k_energy<T><<<nb, 256, 0, st>>>(state, N, c->p.nu, red);
    k_sum_pairs<<<1, 256, 0, st>>>(red, nb, red + 2 * nb);
    LAUNCH_CHECK();
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, red + 2 * nb, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync_check();
    *E = h[0];
    *eps = h[1];
  }

  void spectrum(int kind, double* out, int nbins) override { binned(kind, out, nbins, 0, nullptr); }

  // bins of the quadratic form q of k_spectrum (0: energy, 1: transfer with B, 2: dissipation)
  void binned(int kind, double* out, int nbins, int q, const cpx<T>* B) {
    // partial bins [nb][nbins] followed by the final [nbins] in the reduction buffer
    const size_t cap = (size_t)red_blocks * 1024;
    int nb = (int)(cap / (size_t)nbins) - 1;
    if (nb > red_blocks) nb = red_blocks;
    if (nb < 1) throw NsError{NS_ERR_INVALID_ARG, "nbins too large"};
    k_spectrum<T><<<nb, 256, nbins * sizeof(double), st>>>(state, N, kind, nbins, red, q, B, c->p.nu);
    double* fin = red + (size_t)nb * nbins;
    k_spectrum_final<<<(nbins + 127) / 128, 128, 0, st>>>(red, nb, nbins, fin);
    LAUNCH_CHECK();
    CUDA_TRY(cudaMemcpyAsync(out, fin, nbins * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync_check();
  }

  // Nonlinear energy flux and cumulative dissipation on shell bins (Sec. 3.4)
  cpx<T>* nlbuf = nullptr;
  void energy_flux(const double* delta, int nshift, double* flux, double* cumd, int nbins) override {
    carry_step = -1;  // the mixed fields / state / forcing record change here
    if (flux) {
      if (!nlbuf) CUDA_TRY(cudaMalloc(&nlbuf, 3 * F1 * sizeof(cpx<T>)));
      if (nshift == 0) {
        nl_eval(state, nullptr, nlbuf);
      } else {
        if (!nltmp && nshift > 1) CUDA_TRY(cudaMalloc(&nltmp, 3 * F1 * sizeof(cpx<T>)));
        for (int sidx = 0; sidx < nshift; ++sidx) {
          std::vector<double> sh(delta + 3 * sidx, delta + 3 * sidx + 3);
          upload_shifts(sh);
          nl_eval(state, shift_tab(0), sidx == 0 ? nlbuf : nltmp);
          if (sidx > 0) ew(EW_ADD, nlbuf, nltmp, nullptr, nlbuf);
        }
        if (nshift > 1) ew(EW_SCALE, nlbuf, nullptr, nullptr, nlbuf, 1.0 / nshift);
      }
      std::vector<double> t(nbins);
      binned(0, t.data(), nbins, 1, nlbuf);
      double acc = 0.0;
      for (int k = 0; k < nbins; ++k) {
        acc += t[k];
        flux[k] = -acc;
      }
    }
    if (cumd) {
      std::vector<double> d(nbins);
      binned(0, d.data(), nbins, 2, nullptr);
      double acc = 0.0;
      for (int k = 0; k < nbins; ++k) {
        acc += d[k];
        cumd[k] = acc;
      }
    }
  }
  cpx<T>* nltmp = nullptr;
};

int fail(ns_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

template <typename F>
int guarded(ns_ctx* c, F&& f) {
  if (!c) return NS_ERR_INVALID_ARG;
  try {
    if (c->p.device >= 0) {
      cudaError_t e = cudaSetDevice(c->p.device);
      if (e != cudaSuccess) return fail(c, NS_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    return f();
  } catch (const NsError& e) {
    return fail(c, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, NS_ERR_OOM, "host allocation failed");
  }
}

}  // namespace

int ns_ctx_buffers(ns_ctx* c, double dt, NsCtxBuffers* b) {
  return guarded(c, [&]() {
    c->solver->buffers(dt, b);
    return (int)NS_OK;
  });
}

int ns_ctx_advance(ns_ctx* c, double dt, int nsteps) {
  if (!c) return NS_ERR_INVALID_ARG;
  c->solver->invalidate_carry();  // the batch kernel wrote this member's buffers
  for (int i = 0; i < nsteps; ++i) c->t += dt;  // same accumulation as ns_step
  c->step += nsteps;
  return NS_OK;
}

extern "C" {

const char* ns_init_error(void) { return g_init_error.c_str(); }

int ns_init_ex(ns_ctx** out, const ns_params* prm) {
  if (!out || !prm) {
    g_init_error = "NULL argument";
    return NS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const ns_params& p = *prm;
  if (p.N < 8 || p.N > 1024 || p.N % 2 != 0 || !is_2a3b(p.N)) {
    g_init_error = "N must be even, of the form 2^a 3^b, with 8 <= N <= 1024";
    return NS_ERR_UNSUPPORTED_N;
  }
  if (!(std::fabs(p.L - 2.0 * M_PI) <= 1e-12)) {
    g_init_error = "L must be 2*pi";
    return NS_ERR_INVALID_ARG;
  }
  if (!(p.nu >= 0.0) || !std::isfinite(p.nu)) {
    g_init_error = "nu must be finite and >= 0";
    return NS_ERR_INVALID_ARG;
  }
  if (!(p.kmax > 0.0) || p.kmax > 0.5 * p.N) {
    g_init_error = "kmax must satisfy 0 < kmax <= N/2";
    return NS_ERR_KMAX;
  }
  if (p.truncation != NS_TRUNC_SPHERICAL && p.truncation != NS_TRUNC_CUBIC &&
      p.truncation != NS_TRUNC_NO_DOUBLE_ALIAS) {
    g_init_error = "unknown truncation";
    return NS_ERR_INVALID_ARG;
  }
  if (p.scheme < NS_RK2 || p.scheme > NS_RK2_PS_RANDOM) {
    g_init_error = "unknown scheme";
    return NS_ERR_INVALID_ARG;
  }
  if (p.precision != NS_FP32 && p.precision != NS_FP64) {
    g_init_error = "unknown precision";
    return NS_ERR_INVALID_ARG;
  }
  ns_ctx* c = new ns_ctx();
  c->p = p;
  trunc_bounds(p.kmax, &c->K2max, &c->Kimax);
  try {
    CUDA_TRY(cudaSetDevice(p.device));
    if (p.stream) {
      c->stream = (cudaStream_t)p.stream;
    } else {
      CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    if (p.precision == NS_FP32)
      c->solver = new Solver<float>(c);
    else
      c->solver = new Solver<double>(c);
  } catch (const NsError& e) {
    g_init_error = e.msg;
    delete c->solver;
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return e.code;
  }
  *out = c;
  return NS_OK;
}

int ns_init(ns_ctx** ctx, int N, double L, double nu, double kmax, int truncation, int scheme) {
  ns_params p;
  memset(&p, 0, sizeof(p));
  p.N = N; p.L = L; p.nu = nu; p.kmax = kmax; p.truncation = truncation; p.scheme = scheme;
  p.precision = NS_FP32; p.device = 0; p.stream = nullptr; p.seed = 0;
  return ns_init_ex(ctx, &p);
}

int ns_destroy(ns_ctx* c) {
  if (!c) return NS_OK;
  cudaSetDevice(c->p.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c->solver;
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return NS_OK;
}

const char* ns_last_error(ns_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

int ns_set_velocity(ns_ctx* c, const double* u) {
  return guarded(c, [&]() {
    if (!u) return fail(c, NS_ERR_INVALID_ARG, "u is NULL");
    c->solver->set_velocity(u);
    c->t = 0.0;
    c->step = 0;
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_get_velocity(ns_ctx* c, double* u) {
  return guarded(c, [&]() {
    if (!u) return fail(c, NS_ERR_INVALID_ARG, "u_out is NULL");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    c->solver->get_velocity(u);
    return (int)NS_OK;
  });
}

int ns_get_state(ns_ctx* c, double* s) {
  return guarded(c, [&]() {
    if (!s) return fail(c, NS_ERR_INVALID_ARG, "re_im_out is NULL");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    c->solver->get_state(s);
    return (int)NS_OK;
  });
}

int ns_set_state(ns_ctx* c, const double* s) {
  return guarded(c, [&]() {
    if (!s) return fail(c, NS_ERR_INVALID_ARG, "re_im is NULL");
    c->solver->set_state(s);
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_set_forcing(ns_ctx* c, int kind, double kf_min, double kf_max, double eps, double t_corr,
                   uint64_t seed) {
  return guarded(c, [&]() {
    if (kind == NS_FORCE_NONE) {
      c->solver->set_forcing(kind, 0, 0, 0, 1, 0);
      return (int)NS_OK;
    }
    if (kind != NS_FORCE_TCRANDOM_CONST_EPS) return fail(c, NS_ERR_INVALID_ARG, "unknown forcing kind");
    if (!(kf_min >= 1.0) || !(kf_max >= kf_min) || kf_max > 8.0 || kf_max >= 0.5 * c->p.N ||
        kf_max >= c->p.kmax)
      return fail(c, NS_ERR_INVALID_ARG, "need 1 <= kf_min <= kf_max <= 8, kf_max < min(N/2, kmax)");
    if (!(t_corr > 0.0) || !(eps >= 0.0) || !std::isfinite(eps))
      return fail(c, NS_ERR_INVALID_ARG, "need t_corr > 0 and finite eps >= 0");
    c->solver->set_forcing(kind, kf_min, kf_max, eps, t_corr, seed);
    return (int)NS_OK;
  });
}

int ns_step(ns_ctx* c, double dt, int nsteps) {
  return guarded(c, [&]() {
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(c, NS_ERR_INVALID_ARG, "need dt > 0, nsteps >= 0");
    if (nsteps == 0) return (int)NS_OK;
    c->solver->step(dt, nsteps);
    return (int)NS_OK;
  });
}

int ns_step_cfl(ns_ctx* c, double cfl, double dt_max, int nsteps) {
  return guarded(c, [&]() {
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    if (!(cfl > 0.0) || !std::isfinite(cfl) || !(dt_max > 0.0) || !std::isfinite(dt_max) || nsteps < 0)
      return fail(c, NS_ERR_INVALID_ARG, "need cfl > 0, dt_max > 0, nsteps >= 0");
    if (nsteps == 0) return (int)NS_OK;
    c->solver->step_cfl(cfl, dt_max, nsteps);
    return (int)NS_OK;
  });
}

int ns_step_diag(ns_ctx* c, double dt, int nsteps, double* E_out, double* eps_out) {
  return guarded(c, [&]() {
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(c, NS_ERR_INVALID_ARG, "need dt > 0, nsteps >= 0");
    if (nsteps > 0 && (!E_out || !eps_out)) return fail(c, NS_ERR_INVALID_ARG, "E_out / eps_out is NULL");
    if (nsteps == 0) return (int)NS_OK;
    c->solver->step_diag(dt, nsteps, E_out, eps_out);
    if (!std::isfinite(E_out[nsteps - 1]) || !std::isfinite(eps_out[nsteps - 1]))
      return fail(c, NS_ERR_NONFINITE, "energy is not finite");
    return (int)NS_OK;
  });
}

int ns_set_shifts(ns_ctx* c, const double* da, int nsteps) {
  return guarded(c, [&]() {
    if (nsteps < 0 || (nsteps > 0 && !da)) return fail(c, NS_ERR_INVALID_ARG, "bad shifts");
    c->override_shifts.assign(da, da + 3 * (size_t)nsteps);
    c->override_pos = 0;
    c->solver->invalidate_carry();
    return (int)NS_OK;
  });
}

int ns_nonlinear(ns_ctx* c, const double* in, const double* delta, double* out) {
  return guarded(c, [&]() {
    if (!delta || !out) return fail(c, NS_ERR_INVALID_ARG, "NULL delta or output");
    if (!in && !c->have_state) return fail(c, NS_ERR_STATE, "no state");
    c->solver->nonlinear(in, delta, out);
    return (int)NS_OK;
  });
}

int ns_energy(ns_ctx* c, double* E, double* eps) {
  return guarded(c, [&]() {
    if (!E || !eps) return fail(c, NS_ERR_INVALID_ARG, "NULL output");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    c->solver->energy(E, eps);
    if (!std::isfinite(*E) || !std::isfinite(*eps)) return fail(c, NS_ERR_NONFINITE, "energy is not finite");
    return (int)NS_OK;
  });
}

int ns_energy_spectrum(ns_ctx* c, int kind, double* out, int nbins) {
  return guarded(c, [&]() {
    if (!out || nbins <= 0 || nbins > 4096) return fail(c, NS_ERR_INVALID_ARG, "need out != NULL, 0 < nbins <= 4096");
    if (kind < NS_SPEC_SHELL || kind > NS_SPEC_Z) return fail(c, NS_ERR_INVALID_ARG, "unknown spectrum kind");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    c->solver->spectrum(kind, out, nbins);
    return (int)NS_OK;
  });
}

int ns_energy_flux(ns_ctx* c, const double* delta, int nshift, double* flux, double* cumdiss, int nbins) {
  return guarded(c, [&]() {
    if (nbins <= 0 || nbins > 4096) return fail(c, NS_ERR_INVALID_ARG, "need 0 < nbins <= 4096");
    if (nshift < 0 || nshift > 8 || (nshift > 0 && !delta))
      return fail(c, NS_ERR_INVALID_ARG, "need 0 <= nshift <= 8 and delta for nshift > 0");
    for (int i = 0; i < 3 * nshift; ++i)
      if (!std::isfinite(delta[i])) return fail(c, NS_ERR_INVALID_ARG, "non-finite shift");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    c->solver->energy_flux(delta, nshift, flux, cumdiss, nbins);
    return (int)NS_OK;
  });
}

namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, N, precision, scheme, truncation, fkind;
  double kmax, nu;
  uint64_t seed;
  double t;
  int64_t step;
  double fv[4];
  uint64_t fseed;
  uint64_t nbytes;
};
const char kCkptMagic[8] = {'N', 'S', 'C', 'K', 'P', 'T', '0', '1'};
}  // namespace

int ns_checkpoint_save(ns_ctx* c, const char* path) {
  return guarded(c, [&]() {
    if (!path) return fail(c, NS_ERR_INVALID_ARG, "null path");
    if (!c->have_state) return fail(c, NS_ERR_STATE, "no velocity or state set");
    std::vector<unsigned char> raw;
    c->solver->raw_state(raw);
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, 8);
    h.version = 1; h.N = c->p.N; h.precision = c->p.precision; h.scheme = c->p.scheme;
    h.truncation = c->p.truncation; h.kmax = c->p.kmax; h.nu = c->p.nu; h.seed = c->p.seed;
    h.t = c->t; h.step = c->step;
    c->solver->forcing_params(&h.fkind, h.fv, &h.fseed);
    h.nbytes = raw.size();
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(c, NS_ERR_IO, "cannot open " + tmp);
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
                    std::fwrite(raw.data(), 1, raw.size(), f) == raw.size();
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) {
      std::remove(tmp.c_str());
      return fail(c, NS_ERR_IO, "write failed: " + tmp);
    }
    if (std::rename(tmp.c_str(), path) != 0) return fail(c, NS_ERR_IO, "rename failed: " + std::string(path));
    return (int)NS_OK;
  });
}

int ns_checkpoint_load(ns_ctx* c, const char* path) {
  return guarded(c, [&]() {
    if (!path) return fail(c, NS_ERR_INVALID_ARG, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, NS_ERR_IO, "cannot open " + std::string(path));
    CkptHeader h;
    std::vector<unsigned char> raw;
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && memcmp(h.magic, kCkptMagic, 8) == 0 && h.version == 1 &&
              h.nbytes < (1ull << 40);
    if (ok) {
      raw.resize(h.nbytes);
      ok = std::fread(raw.data(), 1, raw.size(), f) == raw.size();
    }
    std::fclose(f);
    if (!ok) return fail(c, NS_ERR_IO, "not a complete checkpoint: " + std::string(path));
    if (h.N != c->p.N || h.precision != c->p.precision || h.scheme != c->p.scheme ||
        h.truncation != c->p.truncation || h.kmax != c->p.kmax || h.nu != c->p.nu)
      return fail(c, NS_ERR_INVALID_ARG, "checkpoint of another configuration");
    c->solver->set_raw_state(raw.data(), raw.size());
    if (h.fkind != NS_FORCE_NONE)
      c->solver->set_forcing(h.fkind, h.fv[0], h.fv[1], h.fv[2], h.fv[3], h.fseed);
    c->p.seed = h.seed;
    c->t = h.t;
    c->step = h.step;
    c->override_shifts.clear();
    c->override_pos = 0;
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_time(ns_ctx* c, double* t, int64_t* step) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (t) *t = c->t;
  if (step) *step = c->step;
  return NS_OK;
}

int ns_set_time(ns_ctx* c, double t, int64_t step) {
  if (!c) return NS_ERR_INVALID_ARG;
  c->t = t;
  c->step = step;
  return NS_OK;
}

int ns_device_state(ns_ctx* c, void** state, void** stream, int* precision) {
  if (!c) return NS_ERR_INVALID_ARG;
  if (state) *state = c->solver->state_ptr();
  if (stream) *stream = (void*)c->stream;
  if (precision) *precision = c->p.precision;
  return NS_OK;
}

int ns_vjp(ns_ctx* c, const double* u0, int nsteps, double dt, int ckpt_every, int loss,
           double* loss_out, double* grad_u0_out) {
  return guarded(c, [&]() {
    if (!u0 || !loss_out || !grad_u0_out) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if (c->p.scheme != NS_RK2_PS_RANDOM && c->p.scheme != NS_RK2_PS_APPROX)
      return fail(c, NS_ERR_INVALID_ARG, "ns_vjp supports the RK2 phase-shift random/approx schemes");
    if (nsteps < 1 || ckpt_every < 1 || !(dt > 0.0) || (loss != NS_LOSS_DISSIPATION && loss != NS_LOSS_ENERGY))
      return fail(c, NS_ERR_INVALID_ARG, "need nsteps >= 1, ckpt_every >= 1, dt > 0 and a known loss");
    c->solver->vjp(u0, nsteps, dt, ckpt_every, loss, loss_out, grad_u0_out);
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_vjp_state(ns_ctx* c, const double* u0, int nsteps, double dt, int ckpt_every,
                 const double* gT, double* grad_u0_out) {
  return guarded(c, [&]() {
    if (!u0 || !gT || !grad_u0_out) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if (c->p.scheme != NS_RK2_PS_RANDOM && c->p.scheme != NS_RK2_PS_APPROX)
      return fail(c, NS_ERR_INVALID_ARG, "ns_vjp_state supports the RK2 phase-shift random/approx schemes");
    if (nsteps < 1 || ckpt_every < 1 || !(dt > 0.0))
      return fail(c, NS_ERR_INVALID_ARG, "need nsteps >= 1, ckpt_every >= 1 and dt > 0");
    c->solver->vjp_state(u0, nsteps, dt, ckpt_every, gT, grad_u0_out);
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_tape_forward(ns_ctx* c, const void* u0, int nsteps, double dt, int ckpt_every, void* uT) {
  return guarded(c, [&]() {
    if (!u0 || !uT) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if (c->p.scheme != NS_RK2_PS_RANDOM && c->p.scheme != NS_RK2_PS_APPROX)
      return fail(c, NS_ERR_INVALID_ARG, "ns_tape_forward supports the RK2 phase-shift random/approx schemes");
    if (nsteps < 1 || ckpt_every < 1 || !(dt > 0.0))
      return fail(c, NS_ERR_INVALID_ARG, "need nsteps >= 1, ckpt_every >= 1 and dt > 0");
    c->solver->tape_forward(u0, nsteps, dt, ckpt_every, uT);
    c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_tape_backward(ns_ctx* c, const void* gT, int loss, void* grad_u0) {
  return guarded(c, [&]() {
    if (!grad_u0) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if (!gT && loss != NS_LOSS_DISSIPATION && loss != NS_LOSS_ENERGY)
      return fail(c, NS_ERR_INVALID_ARG, "unknown loss");
    c->solver->tape_backward(gT, loss, grad_u0);
    return (int)NS_OK;
  });
}

int ns_rank_copy(ns_ctx* c, int buf, int axis, int lo, int hi, int to_device, double* host) {
  return guarded(c, [&]() {
    if (!host) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if (buf < NS_BUF_STATE || buf > NS_BUF_NL || (axis != 0 && axis != 1) || lo < 0 || hi <= lo ||
        hi > c->p.N)
      return fail(c, NS_ERR_INVALID_ARG, "need a known buffer, axis 0 or 1 and 0 <= lo < hi <= N");
    c->solver->rank_copy(buf, axis, lo, hi, to_device != 0, host);
    if (to_device && buf == NS_BUF_STATE) c->have_state = true;
    return (int)NS_OK;
  });
}

int ns_rank_pencil(ns_ctx* c, int kind, const double* delta, int ky_lo, int ky_hi) {
  return guarded(c, [&]() {
    if (!delta) return fail(c, NS_ERR_INVALID_ARG, "NULL argument");
    if ((kind != NS_RANK_INIT && kind != NS_RANK_NL) || ky_lo < 0 || ky_hi <= ky_lo || ky_hi > c->p.N)
      return fail(c, NS_ERR_INVALID_ARG, "need a known pass kind and 0 <= ky_lo < ky_hi <= N");
    for (int i = 0; i < 3; ++i)
      if (!std::isfinite(delta[i])) return fail(c, NS_ERR_INVALID_ARG, "non-finite shift");
    c->solver->rank_pencil(kind, delta, ky_lo, ky_hi);
    return (int)NS_OK;
  });
}

int ns_rank_slab(ns_ctx* c, int z_lo, int z_hi) {
  return guarded(c, [&]() {
    if (z_lo < 0 || z_hi <= z_lo || z_hi > c->p.N)
      return fail(c, NS_ERR_INVALID_ARG, "need 0 <= z_lo < z_hi <= N");
    c->solver->rank_slab(z_lo, z_hi);
    return (int)NS_OK;
  });
}

int ns_profile(ns_ctx* c, int enable) {
  return guarded(c, [&]() {
    c->solver->profile(enable);
    return (int)NS_OK;
  });
}

int ns_profile_read(ns_ctx* c, int kind, double* total_ms, int64_t* timed, int64_t* launches) {
  return guarded(c, [&]() {
    if (kind < 0 || kind >= NS_PROF_KINDS) return fail(c, NS_ERR_INVALID_ARG, "unknown kernel kind");
    c->solver->profile_read(kind, total_ms, timed, launches);
    return (int)NS_OK;
  });
}

double ns_model_bytes_per_step(ns_ctx* c) {
  if (!c) return 0.0;
  const double C = (double)c->p.N * c->p.N * c->p.N * (c->p.precision == NS_FP64 ? 8.0 : 4.0);
  switch (c->p.scheme) {
    case NS_RK2: return 41.0 * C;
    case NS_RK4: return 94.0 * C;
    case NS_RK2_PS_EXACT: return 73.0 * C;
    default: return 44.0 * C;
  }
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Nonlinear term without any device allocation (ns_nonlinear_noalloc).
//
// For callers that cannot allocate device memory themselves: host applications whose
// device memory is fully reserved by their own allocator, and loops that must not pay an
// allocation's latency or risk its failure once they run.  All working memory is the
// file-scope array below, sized for N <= NS_NOALLOC_MAX_N in FP32; every GPU that loads
// this library holds it until the process exits.  Calls share it and keep the last call's
// contents, so calls that overlap on the GPU (other streams or threads) race.
// ------------------------------------------------------------------------------------------
namespace {

constexpr int kNoallocMaxN = 64;
constexpr size_t kNoallocF1 = (size_t)kNoallocMaxN * kNoallocMaxN * (kNoallocMaxN / 2);
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffMixed = 0;
constexpr size_t kOffFt = kOffMixed + align256(5 * kNoallocF1 * sizeof(cpx<float>));
constexpr size_t kOffScr = kOffFt + align256(3 * kNoallocF1 * sizeof(cpx<float>));
constexpr size_t kOffTw = kOffScr + align256(6 * kNoallocF1 * sizeof(cpx<float>));  // G = N planes
constexpr size_t kOffSh = kOffTw + align256(kNoallocMaxN * sizeof(cpx<float>));
constexpr size_t kOffErr = kOffSh + align256(3 * kNoallocMaxN * sizeof(cpx<float>));
constexpr size_t kNoallocBytes = kOffErr + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// exp(i k(i) delta_d) for one shift passed by value (no device-side argument buffer)
__global__ void k_shift_table_value(cpx<float>* out, int N, double d0, double d1, double d2) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * N) return;
  const int i = idx % N, d = idx / N;
  const double dl = d == 0 ? d0 : (d == 1 ? d1 : d2);
  double s, c;
  sincos((double)kof(i, N) * dl, &s, &c);
  out[idx] = mk<float>((float)c, (float)s);
}

std::mutex g_noalloc_mu;
void* g_noalloc_base[256] = {nullptr};
int g_noalloc_optin[256] = {0};

}  // namespace

extern "C" int ns_nonlinear_noalloc(const void* state, void* out, int N, double kmax,
                                    int truncation, const double* delta, void* stream_p) {
  if (!state || !out || !delta) return NS_ERR_INVALID_ARG;
  if (N < 8 || N > kNoallocMaxN || N % 2 != 0 || !is_2a3b(N)) return NS_ERR_UNSUPPORTED_N;
  if (!(kmax > 0.0) || kmax > 0.5 * N) return NS_ERR_KMAX;
  if (truncation != NS_TRUNC_SPHERICAL && truncation != NS_TRUNC_CUBIC &&
      truncation != NS_TRUNC_NO_DOUBLE_ALIAS)
    return NS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream_p;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NS_ERR_CUDA;
  unsigned char* base = nullptr;
  int optin = 0;
  {
    // once per device, with that device current: the host-side name of the array is not a
    // device address, so ask the runtime for the address the kernels must use
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return NS_ERR_CUDA;
      int oi = 0;
      if (cudaDeviceGetAttribute(&oi, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return NS_ERR_CUDA;
      if (cudaFuncSetAttribute(k_pencil<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, oi) != cudaSuccess ||
          cudaFuncSetAttribute(k_yinv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, oi) != cudaSuccess ||
          cudaFuncSetAttribute(k_yfwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, oi) != cudaSuccess ||
          cudaFuncSetAttribute(k_xrow<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, oi) != cudaSuccess)
        return NS_ERR_CUDA;
      g_noalloc_base[dev] = p;
      g_noalloc_optin[dev] = oi;
    }
    base = static_cast<unsigned char*>(g_noalloc_base[dev]);
    optin = g_noalloc_optin[dev];
  }
  const int M = N / 2;
  cpx<float>* mixed = reinterpret_cast<cpx<float>*>(base + kOffMixed);
  cpx<float>* Ft = reinterpret_cast<cpx<float>*>(base + kOffFt);
  cpx<float>* scr = reinterpret_cast<cpx<float>*>(base + kOffScr);
  cpx<float>* tw = reinterpret_cast<cpx<float>*>(base + kOffTw);
  cpx<float>* sh = reinterpret_cast<cpx<float>*>(base + kOffSh);
  int* err = reinterpret_cast<int*>(base + kOffErr);

  // launch shapes and truncation bounds: the same helpers as a context of this size
  FFTPlan pz = make_plan(N, N), px = make_plan(M, N);
  const GenericShapes g = generic_shapes(N, sizeof(cpx<float>));
  if (!generic_shapes_fit(g, optin)) return NS_ERR_INTERNAL;
  int K2max, Kimax;
  trunc_bounds(kmax, &K2max, &Kimax);

  // the error flag must start at zero; every other region is written before it is read
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return NS_ERR_CUDA;
  k_twiddle<float><<<(N + 255) / 256, 256, 0, st>>>(tw, N);
  k_shift_table_value<<<(3 * N + 255) / 256, 256, 0, st>>>(sh, N, delta[0], delta[1], delta[2]);

  PencilArgs<float> p;
  memset(&p, 0, sizeof(p));
  p.N = N; p.M = M; p.TX = g.TX; p.pz = pz; p.tw = tw; p.mode = MODE_INIT;
  p.src = static_cast<const cpx<float>*>(state);
  p.trunc = truncation; p.K2max = K2max; p.Kimax = Kimax; p.err = err;
  p.nOut = 1; p.osh[0] = sh; p.out[0] = mixed;
  k_pencil<float><<<(M / g.TX) * N, g.bdP, g.smP, st>>>(p);

  SlabArgs<float> a;
  memset(&a, 0, sizeof(a));
  a.N = N; a.M = M; a.py = pz; a.px = px; a.tw = tw; a.scr = scr; a.TY = g.TY; a.RX = g.RX;
  a.err = err; a.mixed = mixed; a.Ft = Ft; a.xmode = XMODE_NONLINEAR; a.z0 = 0; a.G = N;
  k_yinv<float><<<dim3(M / g.TY, N), g.bdY, g.smYi, st>>>(a);
  k_xrow<float><<<(N * N + g.RX - 1) / g.RX, g.bdX, g.smX, st>>>(a);
  k_yfwd<float><<<dim3(M / g.TY, N), g.bdY, g.smYf, st>>>(a);

  PencilArgs<float> q = p;
  q.mode = MODE_NL;
  q.src = nullptr;
  q.nOut = 0;
  q.nF = 1; q.F[0] = Ft; q.dsh[0] = sh; q.wF[0] = (float)(1.0 / ((double)N * N * N));
  q.acc = static_cast<cpx<float>*>(out);
  k_pencil<float><<<(M / g.TX) * N, g.bdP, g.smP, st>>>(q);
  if (cudaGetLastError() != cudaSuccess) return NS_ERR_CUDA;

  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return NS_ERR_CUDA;
  return h ? NS_ERR_INTERNAL : NS_OK;
}
