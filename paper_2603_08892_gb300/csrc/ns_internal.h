// ns_internal.h -- library-internal access to a context's device buffers (not part of the
// public C ABI): the batched ensemble kernel advances several contexts in one launch.
#pragma once

#include <stdint.h>

#include "../../include/ns.h"

struct NsCtxBuffers {
  int N, precision, scheme, truncation;
  int K2max, Kimax, G;
  double nu, kmax;
  void* state;   // [3][N][N][N/2]
  void* mixed;   // [5][N][N][N/2]
  void* Ft;      // [3][N][N][N/2]
  void* scr;     // [6][G][N][N/2]
  void* tw;      // [N]
  void* ifac;    // [2][N]  exp(-nu k^2 dt), exp(-nu k^2 dt/2)
  void* err;     // int device flag
  uint64_t seed;
  int64_t step;
  double t;
};

// Fills b (after preparing the integrating-factor tables for dt when dt > 0).
int ns_ctx_buffers(ns_ctx* c, double dt, NsCtxBuffers* b);
// Advances the context's time and step counters by nsteps of size dt.
int ns_ctx_advance(ns_ctx* c, double dt, int nsteps);
