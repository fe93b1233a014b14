// ns_batch.cu -- C ABI of the batched ensembles (see ns_batch.cuh for the work list and the
// persistent kernel); the FP64 kernel is compiled in ns_batch_f64.cu.
#include "ns_batch.cuh"

#include <cstdio>
#include <cstdlib>

using namespace nsb;

int ns_batch_step_f64(ns_batch* b, const double* dt, int nsteps);
int ns_batch_max_ctas_f64();

namespace {

int batch_step_any(ns_batch* b, const double* dt, int nsteps) {
  return b->precision == NS_FP32 ? batch_step_t<float>(b, dt, nsteps) : ns_batch_step_f64(b, dt, nsteps);
}

// Schedule tuner of the persistent launch: the work-list granularity (tiles per ticket) and
// the CTAs per SM are timed on this ensemble, one step per candidate after an untimed one;
// the members' states, times and step counters are saved before and restored after, so the
// tuning leaves the simulation unchanged.  NS_BATCH_SCHEDULE="gran,ctas_per_sm" forces a
// schedule; NS_AUTOTUNE=0 keeps the default (1 tile per ticket, as many CTAs as fit).
int batch_tune(ns_batch* b, const double* dt) {
  b->tuned = true;
  if (const char* f = std::getenv("NS_BATCH_SCHEDULE")) {
    int g = 1, q = 0;
    if (std::sscanf(f, "%d,%d", &g, &q) >= 1) {
      b->gran = g >= 0 ? g : 1;
      b->per_sm_req = q > 0 ? q : 0;
    }
    return NS_OK;
  }
  const char* en = std::getenv("NS_AUTOTUNE");
  if ((en && std::string(en) == "0") || b->stall) return NS_OK;
  const int n = b->count;
  std::vector<NsCtxBuffers> cb(n);
  std::vector<size_t> bytes(n), off(n + 1, 0);
  std::vector<double> t0(n);
  std::vector<int64_t> s0(n);
  for (int m = 0; m < n; ++m) {
    int rc = ns_ctx_buffers(b->mem[m], dt[m], &cb[m]);
    if (rc != NS_OK) return rc;
    const size_t cs = cb[m].precision == NS_FP32 ? 8 : 16;
    bytes[m] = 3 * (size_t)cb[m].N * cb[m].N * (cb[m].N / 2) * cs;
    off[m + 1] = off[m] + bytes[m];
    ns_time(b->mem[m], &t0[m], &s0[m]);
  }
  unsigned char* save = nullptr;
  if (cudaMalloc(&save, off[n]) != cudaSuccess) {
    cudaGetLastError();
    return NS_OK;  // no room to tune: keep the default schedule
  }
  for (int m = 0; m < n; ++m)
    cudaMemcpyAsync(save + off[m], cb[m].state, bytes[m], cudaMemcpyDeviceToDevice, b->st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bg = 1, bq = 0, rc = NS_OK;
  int maxq = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = b->precision == NS_FP32 ? BCfg<float>::SM : BCfg<double>::SM;
    const int nt = b->precision == NS_FP32 ? BCfg<float>::NT : BCfg<double>::NT;
    if (b->precision == NS_FP32)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxq, k_batch<float>, nt, smem);
    else
      maxq = ns_batch_max_ctas_f64();  // (the FP64 kernel lives in its own translation unit)
  }
  for (int g : {0, 1, 2, 4, 8}) {  // 0: the grid schedule (one launch per pass and size class)
    for (int q : {0, 1}) {
      if (q == 1 && (maxq <= 1 || g == 0)) continue;
      b->gran = g;
      b->per_sm_req = q;
      rc = batch_step_any(b, dt, 1);  // untimed (graph capture)
      if (rc != NS_OK) break;
      cudaEventRecord(e0, b->st);
      rc = batch_step_any(b, dt, 1);
      cudaEventRecord(e1, b->st);
      if (rc != NS_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bg = g;
        bq = q;
      }
    }
    if (rc != NS_OK) break;
  }
  for (int m = 0; m < n; ++m) {
    cudaMemcpyAsync(cb[m].state, save + off[m], bytes[m], cudaMemcpyDeviceToDevice, b->st);
    ns_set_time(b->mem[m], t0[m], s0[m]);
  }
  cudaStreamSynchronize(b->st);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->gran = bg;
  b->per_sm_req = bq;
  return rc;
}

}  // namespace

extern "C" {

int ns_batch_init(ns_batch** out, int count, const int* N, const double* nu, const double* kmax,
                  const uint64_t* seeds, int scheme, int precision, void* stream) {
  if (!out || count < 1 || count > kMaxMembers || !N || !nu || !kmax) return NS_ERR_INVALID_ARG;
  *out = nullptr;
  if (scheme != NS_RK2_PS_RANDOM && scheme != NS_RK2_PS_APPROX) return NS_ERR_INVALID_ARG;
  if (precision != NS_FP32 && precision != NS_FP64) return NS_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (size_index(N[i]) < 0) return NS_ERR_UNSUPPORTED_N;
  ns_batch* b = new ns_batch();
  b->count = count;
  b->precision = precision;
  b->scheme = scheme;
  int dev = 0;
  cudaGetDevice(&dev);
  if (stream) {
    b->st = (cudaStream_t)stream;
  } else if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return NS_ERR_CUDA;
  } else {
    b->own_stream = true;
  }
  for (int i = 0; i < count; ++i) {
    ns_params p;
    memset(&p, 0, sizeof(p));
    p.N = N[i]; p.L = 2.0 * M_PI; p.nu = nu[i]; p.kmax = kmax[i]; p.truncation = NS_TRUNC_SPHERICAL;
    p.scheme = scheme; p.precision = precision; p.device = dev; p.stream = b->st;
    p.seed = seeds ? seeds[i] : (uint64_t)i;
    ns_ctx* c = nullptr;
    int rc = ns_init_ex(&c, &p);
    if (rc != NS_OK) {
      b->err = ns_init_error();
      ns_batch_destroy(b);
      return rc;
    }
    b->mem.push_back(c);
  }
  const size_t memsz = precision == NS_FP32 ? sizeof(BatchMem<float>) : sizeof(BatchMem<double>);
  if (cudaMalloc(&b->d_mems, count * memsz) != cudaSuccess ||
      cudaMalloc(&b->d_off, (size_t)(kPasses + 2) * (kMaxMembers + 1) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_next, sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&b->d_done, count * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_flags, 2 * sizeof(int)) != cudaSuccess) {
    ns_batch_destroy(b);
    return NS_ERR_OOM;
  }
  *out = b;
  return NS_OK;
}

int ns_batch_destroy(ns_batch* b) {
  if (!b) return NS_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto* m : b->mem) ns_destroy(m);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->d_mems);
  cudaFree(b->d_off);
  cudaFree(b->d_shifts);
  cudaFree(b->d_next);
  cudaFree(b->d_done);
  cudaFree(b->d_flags);
  cudaFree(b->d_tab);
  cudaFree(b->d_cls);
  if (b->own_stream) cudaStreamDestroy(b->st);  // members were given the stream, not its ownership
  delete b;
  return NS_OK;
}

const char* ns_batch_last_error(ns_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

ns_ctx* ns_batch_member(ns_batch* b, int i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->mem[i];
}

int ns_batch_set_velocity(ns_batch* b, int i, const double* u) {
  if (!b || i < 0 || i >= b->count) return NS_ERR_INVALID_ARG;
  const int rc = ns_set_velocity(b->mem[i], u);
  if (rc != NS_OK) b->err = ns_last_error(b->mem[i]);
  return rc;
}

int ns_batch_get_state(ns_batch* b, int i, double* re_im) {
  if (!b || i < 0 || i >= b->count) return NS_ERR_INVALID_ARG;
  const int rc = ns_get_state(b->mem[i], re_im);
  if (rc != NS_OK) b->err = ns_last_error(b->mem[i]);
  return rc;
}

int ns_batch_step(ns_batch* b, const double* dt, int nsteps) {
  if (!b || !dt || nsteps < 0) return NS_ERR_INVALID_ARG;
  if (nsteps == 0) return NS_OK;
  for (int i = 0; i < b->count; ++i)
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return NS_ERR_INVALID_ARG;
  if (!b->tuned) {
    const int rc = batch_tune(b, dt);
    if (rc != NS_OK) return rc;
  }
  return batch_step_any(b, dt, nsteps);
}

int ns_batch_set_schedule(ns_batch* b, int gran, int ctas_per_sm) {
  if (!b || gran < 0 || ctas_per_sm < 0) return NS_ERR_INVALID_ARG;
  b->gran = gran;
  b->per_sm_req = ctas_per_sm;
  b->tuned = true;
  return NS_OK;
}

int ns_batch_schedule(ns_batch* b, int* gran, int* ctas_per_sm) {
  if (!b || !gran || !ctas_per_sm) return NS_ERR_INVALID_ARG;
  *gran = b->gran;
  *ctas_per_sm = b->per_sm_req;
  return NS_OK;
}

int ns_batch_energy(ns_batch* b, double* E, double* eps) {
  if (!b || !E || !eps) return NS_ERR_INVALID_ARG;
  for (int i = 0; i < b->count; ++i) {
    const int rc = ns_energy(b->mem[i], &E[i], &eps[i]);
    if (rc != NS_OK) {
      b->err = ns_last_error(b->mem[i]);
      return rc;
    }
  }
  return NS_OK;
}

int ns_batch_set_spin_limit(ns_batch* b, long long polls) {
  if (!b || polls < 1) return NS_ERR_INVALID_ARG;
  b->spin_limit = polls;
  return NS_OK;
}

int ns_batch_test_stall(ns_batch* b, int on) {
  if (!b) return NS_ERR_INVALID_ARG;
  b->stall = on != 0;
  return NS_OK;
}

int ns_batch_grid(ns_batch* b) { return b ? b->grid : 0; }

}  // extern "C"
