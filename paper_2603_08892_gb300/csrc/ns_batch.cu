// ns_batch.cu -- C ABI of the batched ensembles (see ns_batch.cuh for the work list and the
// persistent kernel); the FP64 kernel is compiled in ns_batch_f64.cu.
#include "ns_batch.cuh"

int ns_batch_step_f64(ns_batch* b, const double* dt, int nsteps);

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
  return b->precision == NS_FP32 ? batch_step_t<float>(b, dt, nsteps)
                                 : ns_batch_step_f64(b, dt, nsteps);
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
