/*
 * ns.h -- C ABI of libns: one GB300 (sm_103a) time-stepper for the triply periodic
 * incompressible Navier-Stokes equations with phase-shift dealiasing.
 *
 * Method (Lambert, Reneuve & Augier, "Aliasing and phase shifting in pseudo-spectral
 * simulations of the incompressible Navier-Stokes equations"):
 *   d_t S = sigma S + N(S) (+ O(S)),  sigma = -nu |k|^2          (Sec. 4.1, Eq. base-eq)
 *   N~_D(S) = T P exp(-ik.D) FFT[u_D x w_D]                       (Sec. 4.1-4.2, Eq. shift_operator_3d)
 *   schemes: RK2, RK4 (+ 2/3 truncation baseline), RK2 phase-shift exact
 *   (Patterson-Orszag), approx and random (Rogallo), and the forced "split" variant
 *   (Sec. 4.1, Eq. Rogallo1981; Sec. 4.2; Sec. 6.1, Eq. forcing-eq).
 *
 * Conventions shared by every call:
 *   - domain [0, 2*pi)^3 (L must be 2*pi), grid N^3, N = 2^a 3^b even, 8 <= N <= 1024;
 *   - physical fields: double u[3][N][N][N], C order [component][z][y][x], x fastest;
 *   - spectral fields: double re_im[3][N][N][N/2][2]: index [component][kz][ky][kx][re,im],
 *     kz, ky in FFT order (0..N/2-1, -N/2..-1), kx = 0..N/2-1 (real-to-complex half
 *     spectrum; the kx = N/2 plane is always zero because kmax <= N/2 truncates it);
 *     uh(k) = N^-3 sum_x u(x) exp(-i k.x) (supplementary Eq. dft_def);
 *   - every host buffer is owned by the caller and only read or written during the call;
 *   - every function returns an ns_status; on failure a message is kept in the context
 *     (ns_last_error) until the next failing call replaces it.
 *   - one context is used from one host thread at a time; it owns all its device memory.
 */
#ifndef NS_H_
#define NS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NS_OK = 0,
  NS_ERR_INVALID_ARG = 1,  /* NULL pointer, bad enum, L != 2*pi, nu < 0, dt <= 0 ...   */
  NS_ERR_UNSUPPORTED_N = 2,/* N not 2^a 3^b, odd, < 8 or > 1024                        */
  NS_ERR_KMAX = 3,         /* kmax <= 0 or kmax > N/2 (C_t = kmax / k_N > 1)           */
  NS_ERR_CUDA = 4,         /* a CUDA runtime call failed (message has the CUDA error)   */
  NS_ERR_OOM = 5,          /* device allocation failed                                  */
  NS_ERR_NONFINITE = 6,    /* energy or dissipation is NaN/Inf                          */
  NS_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up                        */
  NS_ERR_STATE = 8,        /* call out of order (e.g. step before a velocity was set)   */
  NS_ERR_INTERNAL = 9,     /* a device-side consistency check failed (bad launch shape) */
  NS_ERR_IO = 10           /* a checkpoint file could not be written or read, or is not one */
} ns_status;

/* Truncations (Sec. 3.2, Fig. truncation:common; Sec. 4.2, Fig.
 * truncation:spherical:double:aliases(b)): spherical keeps |k| < kmax, cubic keeps every
 * |k_i| < kmax, no-double-alias keeps the spherical set minus the modes that a double alias
 * (an aliased product with exactly two out-of-range components) can reach: every k with
 * |k + N e|^2 <= 4 m for some e in {-1,0,1}^3 with exactly one zero component, m the largest
 * integer below kmax^2.  It equals the spherical set for kmax <= (2 sqrt 2 / 3) N/2; with the
 * exact phase-shift scheme it makes the nonlinear term alias-free at any kmax <= N/2. */
enum { NS_TRUNC_SPHERICAL = 0, NS_TRUNC_CUBIC = 1, NS_TRUNC_NO_DOUBLE_ALIAS = 2 };
enum { NS_RK2 = 0, NS_RK4 = 1, NS_RK2_PS_EXACT = 2, NS_RK2_PS_APPROX = 3, NS_RK2_PS_RANDOM = 4 };
enum { NS_FP32 = 0, NS_FP64 = 1 };
enum { NS_FORCE_NONE = 0, NS_FORCE_TCRANDOM_CONST_EPS = 1 };
enum { NS_SPEC_SHELL = 0, NS_SPEC_X = 1, NS_SPEC_Y = 2, NS_SPEC_Z = 3 };

typedef struct ns_ctx ns_ctx;

typedef struct {
  int N;             /* grid points per direction                                       */
  double L;          /* domain size, must be 2*pi                                       */
  double nu;         /* kinematic viscosity >= 0                                        */
  double kmax;       /* truncation wavenumber, 0 < kmax <= N/2 (Sec. 3.2: kmax = C_t k_N) */
  int truncation;    /* NS_TRUNC_SPHERICAL, NS_TRUNC_CUBIC or NS_TRUNC_NO_DOUBLE_ALIAS (above) */
  int scheme;        /* NS_RK2 ... NS_RK2_PS_RANDOM                                     */
  int precision;     /* NS_FP32 (FP32 butterflies and products, FP64 tables/reductions) or NS_FP64 */
  int device;        /* CUDA device ordinal                                             */
  void* stream;      /* cudaStream_t to launch on (NULL: the context creates its own)   */
  uint64_t seed;     /* seed of the random shifts delta_alpha (splitmix64 counter)       */
} ns_params;

/* Creates a context (FP32, device 0, own stream, seed 0).  Sec. 3.2 (truncation), Sec. 4
 * (schemes).  *ctx is set to NULL on failure; the message is then in ns_init_error(). */
int ns_init(ns_ctx** ctx, int N, double L, double nu, double kmax, int truncation, int scheme);
/* Same with every option; params is read during the call only. */
int ns_init_ex(ns_ctx** ctx, const ns_params* params);
/* Message of the last failed ns_init / ns_init_ex in this thread. */
const char* ns_init_error(void);
/* Frees every device and host resource of the context. NULL is accepted. */
int ns_destroy(ns_ctx* ctx);
/* Message of the last failure on this context ("" if none). Valid until the next call. */
const char* ns_last_error(ns_ctx* ctx);

/* Physical velocity u (host, [3][N][N][N]) -> state: forward FFT, truncation T, Leray
 * projection P, mean mode zeroed (Sec. 3.2; Sec. 4.1 below Eq. base-eq).  A
 * non-solenoidal input is projected.  Resets time and step counter to 0.  Host arrays of
 * this and the following transfer calls are FP64; FP32 contexts copy them as they are and
 * round on the device (to nearest, as a host cast does), so a page-locked host buffer
 * transfers fastest. */
int ns_set_velocity(ns_ctx* ctx, const double* u);
/* State -> physical velocity u_out (host, [3][N][N][N]).  This call, ns_get_state, ns_step,
 * ns_step_cfl, ns_step_diag, ns_energy, ns_energy_spectrum and ns_energy_flux return
 * NS_ERR_STATE on a context that has no state yet (no ns_set_velocity, ns_set_state or
 * ns_checkpoint_load). */
int ns_get_velocity(ns_ctx* ctx, double* u_out);
/* Copies the spectral state to/from host re_im[3][N][N][N/2][2] (no truncation or
 * projection applied on set: resuming from ns_get_state output is bitwise exact). */
int ns_get_state(ns_ctx* ctx, double* re_im_out);
int ns_set_state(ns_ctx* ctx, const double* re_im);

/* Large-scale forcing O(S) (Sec. 2; Sec. 6.1, Eq. forcing-eq).  kind NS_FORCE_TCRANDOM_CONST_EPS:
 * modes kf_min <= |k| <= kf_max (kf_max <= 8), random projected pattern redrawn every
 * t_corr and linearly interpolated in time, amplitude chosen so that an Euler step dt of
 * the forcing alone injects exactly eps*dt of energy.  With forcing set, NS_RK2_PS_RANDOM
 * runs the "split" scheme; RK2 / RK4 / PS exact add O at every stage.  kind NS_FORCE_NONE
 * switches forcing off. */
int ns_set_forcing(ns_ctx* ctx, int kind, double kf_min, double kf_max, double eps,
                   double t_corr, uint64_t seed);

/* Advances nsteps time steps of size dt with the context's scheme (Sec. 4.1-4.2, 6.1).
 * The random scheme draws delta_alpha of step s from splitmix64(seed, 3s+i) unless
 * ns_set_shifts supplied them.  Stream-ordered: returns once the steps are queued on the
 * context's stream (argument and launch errors are returned here; a failed device-side
 * consistency check is returned by the next call that synchronises, e.g. ns_energy or
 * ns_get_state).  The last pencil pass prepares the next step, so consecutive calls cost
 * the same as one call over all their steps. */
int ns_step(ns_ctx* ctx, double dt, int nsteps);
/* Same, each step with an adaptive time step (Sec. 2: CFL condition, coefficient 0.4 for the
 * RK2 schemes and 1.0 for RK4 in the paper): dt = min(dt_max, cfl / sum_i (max_x |u_i| / dx)),
 * dx = 2 pi / N, the maxima taken over the grid values of the velocity that the step's first
 * nonlinear evaluation forms (the state shifted by that evaluation's shift: delta_alpha for
 * the random scheme, none otherwise), reduced inside the slab pass.  One 24-byte read-back
 * per step.  ns_time gives the accumulated time.  NS_ERR_INVALID_ARG unless cfl > 0,
 * dt_max > 0 (finite) and nsteps >= 0. */
int ns_step_cfl(ns_ctx* ctx, double cfl, double dt_max, int nsteps);
/* Same as ns_step, and E and eps (as ns_energy defines them, Sec. 3.4) of the state after each
 * step written to the host arrays E_out[nsteps] and eps_out[nsteps] (caller-owned).  The sums
 * are taken by the pencil pass that writes each step's state (per-tile partial sums, then a
 * fixed-order FP64 sum; sizes without the size-specialised kernels run a separate reduction),
 * and each step's pair is written by the device into mapped pinned host memory as it is
 * produced: no host synchronisation per step; the call returns once every step has
 * completed.  The first call allocates the series buffers (for max(nsteps, 4096) steps; a
 * longer call reallocates).  NS_ERR_INVALID_ARG unless dt > 0, nsteps >= 0 and both outputs
 * are non-NULL (nsteps > 0); NS_ERR_NONFINITE if the last pair is not finite.  The values
 * agree with ns_energy after each step to rounding (the summation order differs). */
int ns_step_diag(ns_ctx* ctx, double dt, int nsteps, double* E_out, double* eps_out);
/* Test hook: delta_alpha for the next nsteps steps (host [nsteps][3], radians), consumed
 * by the following ns_step calls in order; delta_beta = delta_alpha + (pi/N)(1,1,1). */
int ns_set_shifts(ns_ctx* ctx, const double* delta_alpha, int nsteps);

/* Shifted-and-de-shifted nonlinear term of Sec. 4.1-4.2 for the state re_im_in (host,
 * NULL = the context's state) with shift delta[3] (radians): N~ = T P exp(-ik.D)
 * FFT[u_D x w_D], mean mode zero.  Writes host re_im_out[3][N][N][N/2][2]. */
int ns_nonlinear(ns_ctx* ctx, const double* re_im_in, const double* delta, double* re_im_out);

/* Gradient of a loss on the final state with respect to the initial physical velocity
 * (hand-written adjoint; the paper has none).  From u0 (host [3][N][N][N]) runs nsteps steps
 * of size dt of the context's scheme (NS_RK2_PS_RANDOM or _APPROX, with the forcing if set;
 * shifts from the context's seed, step counter starting at 0), keeping the state every
 * ckpt_every steps; loss NS_LOSS_DISSIPATION: L = eps(T) = nu sum_k k^2 |uh|^2, or
 * NS_LOSS_ENERGY: L = E(T).  The reverse sweep recomputes each segment's states from its
 * checkpoint and applies the transposed step: with <a,b> = sum_k Re(conj(a).b) and
 * lambda the cotangent of S_{n+1}, rho = dt/2 E_{dt/2} lambda,
 *   mu = J*_beta(S1; rho) + O*(S1; rho),  sigma = dt E_dt mu,
 *   lambda_n = E_dt (lambda + mu) + J*_alpha(S0; rho + sigma) + O*(S0; rho + sigma),
 * J*_D(S; r) = T P e^{-ik.D} [F(w x r') + ik x F(r' x u)], r' = F^{-1}(e^{ik.D} r), and
 * O*(S; r) = (da/db) Re<f, r> f for the forcing O = a f.  Writes L to *loss_out and dL/du0
 * to grad_u0_out (host [3][N][N][N], gradient for the physical dot product).  Leaves the
 * context at the final state (t = nsteps dt). */
enum { NS_LOSS_DISSIPATION = 0, NS_LOSS_ENERGY = 1 };
int ns_vjp(ns_ctx* ctx, const double* u0, int nsteps, double dt, int ckpt_every, int loss,
           double* loss_out, double* grad_u0_out);

/* Gradient of any loss of the final velocity u(T) with respect to u0 (no counterpart in the
 * paper): the same forward and reverse sweeps as ns_vjp, the reverse sweep seeded with the
 * caller's cotangent gT = dL/du(T) (host [3][N][N][N] FP64, gradient for the physical dot
 * product); its cotangent of S_T is N^3 P T F(gT) (F the forward transform with the 1/N^3
 * factor, whose adjoint for the full-spectrum product is F^{-1} / N^3).  Writes dL/du0 to
 * grad_u0_out (host [3][N][N][N] FP64).  Errors as ns_vjp. */
int ns_vjp_state(ns_ctx* ctx, const double* u0, int nsteps, double dt, int ckpt_every,
                 const double* gT, double* grad_u0_out);

/* The same in two calls on device buffers, for a reverse-mode autodiff caller: u0, uT, gT and
 * grad_u0 are device pointers to [3][N][N][N] reals in the context's precision (float for
 * NS_FP32, double for NS_FP64), caller owned and not aliased with each other.
 * ns_tape_forward: sets the state from u0 (truncated and projected), runs nsteps steps of size
 * dt keeping the state every ckpt_every steps on the device (the tape), and writes u(T) to uT.
 * ns_tape_backward: the reverse sweep of the last ns_tape_forward, seeded with gT = dL/du(T)
 * or, when gT is NULL, with the built-in `loss` (NS_LOSS_*) of the final state; writes
 * dL/du0 to grad_u0.  It can be called again on the same tape.  NS_ERR_STATE without a tape
 * (none recorded, or one invalidated by ns_vjp, ns_vjp_state or ns_set_forcing).  Both are
 * ordered on the context's stream and synchronise it before returning; the caller makes its
 * own writes to u0 / gT complete before the call. */
int ns_tape_forward(ns_ctx* ctx, const void* u0, int nsteps, double dt, int ckpt_every, void* uT);
int ns_tape_backward(ns_ctx* ctx, const void* gT, int loss, void* grad_u0);

/* Kinetic energy E = (1/2) sum_k |uh|^2 and dissipation eps = nu sum_k k^2 |uh|^2 (full
 * spectrum sums, Sec. 3.4; FP64 states in FP64, FP32 states with each mode's terms in FP32,
 * compensated per-thread sums and FP64 across threads; fixed order, so repeatable).
 * NS_ERR_NONFINITE if either is not finite. */
int ns_energy(ns_ctx* ctx, double* E, double* eps);
/* Energy spectrum, FP64 bins k = 0..nbins-1: NS_SPEC_SHELL bins floor(|k| + 1/2),
 * NS_SPEC_X/Y/Z fold +-k_i onto |k_i| (Sec. 3.4, Eq. quality uses the 1D spectra). */
int ns_energy_spectrum(ns_ctx* ctx, int kind, double* out, int nbins);
/* Nonlinear energy flux and cumulative dissipation of the current state on shell bins
 * k = 0 .. nbins-1, bin floor(|k| + 1/2) (Sec. 3.4, Fig. spectra:192).  N is the mean over
 * nshift shift vectors delta[3 s .. 3 s + 2] (radians) of the shifted, truncated, projected
 * nonlinear term (nshift = 0: the unshifted term; the exact scheme's term is the mean over
 * {0, (dx/2)(1,1,1)}).  T(k) = sum over the shell of Re(uh* . Nh) over the full spectrum,
 * flux[k] = -sum_{k' <= k} T(k') (it vanishes at the last shell: the truncated rotational term
 * conserves energy), cumdiss[k] = sum_{k' <= k} 2 nu k'^2 E(k') (eps at the last shell).
 * Either output may be NULL.  The state is unchanged; the first call allocates one or two
 * work fields of the state's size; synchronises the context's stream.  Returns
 * NS_ERR_INVALID_ARG for nbins outside 1..4096, nshift outside 0..8 or a non-finite shift. */
int ns_energy_flux(ns_ctx* ctx, const double* delta, int nshift, double* flux, double* cumdiss, int nbins);

/* Checkpoint of a context to a file, for a bitwise resume: the state in the context's own
 * precision (FP32 or FP64 complex, [3][N][N][N/2], host byte order), time, step count, shift
 * seed and the forcing parameters, after a header with N, precision, scheme, truncation, kmax
 * and nu.  Written to path + ".tmp" and renamed over path.  ns_checkpoint_load reads such a
 * file into a context created with the same N, precision, scheme, truncation, kmax and nu
 * (else NS_ERR_INVALID_ARG) and restores the state, time, step, seed and forcing; stepping on
 * then gives the same bits as an uninterrupted run.  NS_ERR_IO for a file that cannot be
 * written or read, a wrong magic or a truncated file; NS_ERR_STATE to save a context without
 * a state.  Both synchronise the context's stream.  The paper has no counterpart (its runs
 * restart through Fluidsim's files). */
int ns_checkpoint_save(ns_ctx* ctx, const char* path);
int ns_checkpoint_load(ns_ctx* ctx, const char* path);

/* Simulated time and number of steps done since the last ns_set_velocity. */
int ns_time(ns_ctx* ctx, double* t, int64_t* step);
/* Overrides time and step counter (checkpoint resume). */
int ns_set_time(ns_ctx* ctx, double t, int64_t step);

/* Device pointers of the context (for callers that keep data on the GPU): the state
 * ([3][N][N][N/2] complex of the context's precision) and the stream. */
int ns_device_state(ns_ctx* ctx, void** state, void** stream, int* precision);

/* Per-kernel timing with CUDA events recorded on the context's stream around every launch
 * (at most 65536 launches are timed; all are counted).  ns_profile(ctx, 1) resets the
 * counters and starts timing, ns_profile(ctx, 0) stops.  ns_profile_read synchronises the
 * stream and returns, for one kind, the summed event time in ms, the number of timed
 * launches and the number of launches since the reset.  Kinds: */
enum { NS_PROF_PENCIL = 0, NS_PROF_YINV = 1, NS_PROF_XROW = 2, NS_PROF_YFWD = 3,
       NS_PROF_SLAB_PASS = 4, NS_PROF_SLAB_PIPE = 5, NS_PROF_SLAB_CLUSTER = 6, NS_PROF_KINDS = 7 };
int ns_profile(ns_ctx* ctx, int enable);
int ns_profile_read(ns_ctx* ctx, int kind, double* total_ms, int64_t* timed, int64_t* launches);

/* ---- Batched ensembles (no counterpart in the paper) -----------------------------------
 * Independent simulations of uneven N advanced together, each member running the RK2
 * phase-shift random (Rogallo, Sec. 4.2) or approx scheme exactly as a single context does.
 * Two schedules of the same tile bodies (the tuner picks one; the results are the same bits):
 *  - persistent: ONE kernel launch per ns_batch_step call (captured in a CUDA graph and
 *    replayed) whose CTAs take (step, pass, member, tile) work items in order from an atomic
 *    counter and wait, with a bounded spin, until the member's earlier passes are complete;
 *    an expired wait ends the launch with NS_ERR_TIMEOUT instead of hanging;
 *  - grid (gran 0): every pass of each size class is one ordinary grid launch (tiles x the
 *    class's members), the classes one after another on the batch's stream; nothing waits on
 *    the device.
 * Supported member sizes: N in {16, 32, 48, 64, 96, 128}; spherical truncation. */
typedef struct ns_batch ns_batch;
/* count members (1..1024) with sizes N[i], viscosities nu[i], truncation kmax[i] and shift
 * seeds seeds[i] (NULL: seed i); scheme NS_RK2_PS_RANDOM or NS_RK2_PS_APPROX; precision
 * NS_FP32 / NS_FP64; stream: cudaStream_t shared by all members (NULL: the batch creates one). */
int ns_batch_init(ns_batch** b, int count, const int* N, const double* nu, const double* kmax,
                  const uint64_t* seeds, int scheme, int precision, void* stream);
int ns_batch_destroy(ns_batch* b);
const char* ns_batch_last_error(ns_batch* b);
/* The member's own context (owned by the batch): every single-context call applies to it. */
ns_ctx* ns_batch_member(ns_batch* b, int i);
/* Same as ns_set_velocity / ns_get_state on member i. */
int ns_batch_set_velocity(ns_batch* b, int i, const double* u);
int ns_batch_get_state(ns_batch* b, int i, double* re_im_out);
/* Advances every member by nsteps steps of its own dt[i] (host array of count) in one launch. */
int ns_batch_step(ns_batch* b, const double* dt, int nsteps);
/* E[i], eps[i] of every member (host arrays of count). */
int ns_batch_energy(ns_batch* b, double* E, double* eps);
/* Poll budget of each bounded wait of the persistent kernel (default 2e6 polls of >= 100 ns). */
int ns_batch_set_spin_limit(ns_batch* b, long long polls);
/* Test hook: nonzero makes every per-step wait unreachable, so the next ns_batch_step must
 * return NS_ERR_TIMEOUT after the bounded waits expire (the GPU stays usable). */
int ns_batch_test_stall(ns_batch* b, int on);
/* CTAs of the last persistent launch (diagnostics). */
int ns_batch_grid(ns_batch* b);
/* Schedule: gran tiles per work-list ticket of the persistent launch (the ticket, the
 * bounded wait and the completion fence are paid once per gran tiles) and ctas_per_sm CTAs
 * per SM (0: as many as fit); gran 0 selects the grid schedule (ctas_per_sm unused).  The
 * first ns_batch_step tunes both on the ensemble (each candidate times one step; the
 * members' states, times and step counters are saved before and restored after) unless
 * ns_batch_set_schedule was called, NS_BATCH_SCHEDULE="g,q" is set or NS_AUTOTUNE=0.
 * Results do not depend on the schedule.  NS_ERR_INVALID_ARG for gran < 0 or ctas_per_sm < 0. */
int ns_batch_set_schedule(ns_batch* b, int gran, int ctas_per_sm);
int ns_batch_schedule(ns_batch* b, int* gran, int* ctas_per_sm);

/* Nonlinear term N~_D(S) like ns_nonlinear, on device buffers, without allocating any device
 * memory.  No counterpart in the paper: it serves callers that cannot call cudaMalloc --
 * host applications whose device memory is entirely reserved by their own allocator, and
 * loops that must not pay an allocation's latency or risk its failure once running.
 *   state, out: device pointers, complex FP32 [3][N][N][N/2] (layout of ns.h), caller owned;
 *               out may not alias state.
 *   N: 8 <= N <= 64 (NS_ERR_UNSUPPORTED_N beyond, or if N is not an even 2^a 3^b);
 *   kmax, truncation: as in ns_params (NS_ERR_KMAX if kmax <= 0 or kmax > N/2);
 *   delta: host double[3], the shift in radians; stream: cudaStream_t (NULL = default).
 * Working memory is one fixed array inside the library (about 15 MB, sized for N = 64 in
 * FP32), held by every GPU that loads the library until the process exits.  The first call
 * on a device looks up that array's device address and sets kernel attributes (make it
 * before any stream capture).  With CUDA's lazy module loading (the default), the library's
 * device code and this array are placed on the device when first used, which may be this
 * first call: make it (or load the process with CUDA_MODULE_LOADING=EAGER) before the
 * caller's allocator reserves the device's memory; later calls use no further memory.  All calls share the array and it keeps the last call's
 * contents, so calls that overlap on the GPU (other threads or streams) race.  The call is
 * stream ordered and synchronises `stream` before returning; it calls no cudaMalloc,
 * cudaFree or other allocating routine.  Returns NS_ERR_CUDA on a CUDA failure and
 * NS_ERR_INTERNAL if a device-side shape check failed. */
int ns_nonlinear_noalloc(const void* state, void* out, int N, double kmax, int truncation,
                         const double* delta, void* stream);

/* ---- Rank-range passes of a single field split over P ranks (Sec. 2: the slab
 * decomposition of a distributed 3D FFT, as in the paper's FFTW-MPI runs) --------------------
 * A rank holds the ky rows [lo, hi) of the spectral and pencil-pass fields (all z or kz) and
 * the planes [lo, hi) of the slab pass (all y or ky).  One nonlinear evaluation is
 *   ns_rank_pencil(INIT, delta, own ky rows)   state -> mixed fields u, d_z u_x, d_z u_y
 *   exchange 1 (all-to-all: the mixed fields, ky rows -> z planes)
 *   ns_rank_slab(own z planes)                 mixed -> FFT_xy(u x omega)
 *   exchange 2 (all-to-all back: z planes -> ky rows)
 *   ns_rank_pencil(NL, delta, own ky rows)     -> T P e^{-ik.delta} FFT(u x omega)
 * with the host exchanges in between (ns_rank_copy moves blocks between the context's buffers
 * and host memory).  Each call runs the single-field kernels on its range only, on the
 * context's stream, and synchronises it before returning.  No counterpart of the API in the
 * paper; the arithmetic is that of ns_nonlinear. */
enum { NS_BUF_STATE = 0, NS_BUF_MIXED = 1, NS_BUF_FT = 2, NS_BUF_NL = 3 };
enum { NS_RANK_INIT = 0, NS_RANK_NL = 1 };
/* Copies block [lo, hi) of axis `axis` of buffer `buf` (STATE [3][N][N][N/2], MIXED [5][..],
 * FT [3][..], NL [3][..]; complex [field][z or kz][ky][kx]) to (to_device = 0) or from host
 * FP64 (re, im) memory laid out as [F][hi-lo][N][N/2] (axis 0: z or kz planes) or
 * [F][N][hi-lo][N/2] (axis 1: ky rows).  NS_ERR_INVALID_ARG for a NULL host pointer, an
 * unknown buffer or axis, or a range outside [0, N). */
int ns_rank_copy(ns_ctx* ctx, int buf, int axis, int lo, int hi, int to_device, double* host);
/* The pencil pass on the ky rows [ky_lo, ky_hi), shift delta (host double[3], radians):
 * NS_RANK_INIT from the state to the mixed fields, NS_RANK_NL from FT to NL. */
int ns_rank_pencil(ns_ctx* ctx, int kind, const double* delta, int ky_lo, int ky_hi);
/* The slab pass on the planes [z_lo, z_hi): MIXED -> FT (the same plane-group kernels as a
 * whole-field pass). */
int ns_rank_slab(ns_ctx* ctx, int z_lo, int z_hi);

/* Bytes moved to/from HBM per time step by the algorithmic two-pass model (one slab and
 * one pencil pass per evaluation), for roofline reporting. */
double ns_model_bytes_per_step(ns_ctx* ctx);

/* The one-dimensional quadratic model of Sec. 3.3 (Eq. model-1d, the "nl1d" example of where
 * the aliases of a quadratic term land): dS/dt = -sign(S) S^2 on [0, 2 pi), pseudo-spectral on
 * N points (even, 4 <= N <= 2048; N need not be 2^a 3^b) with the truncation k < kmax
 * (0 < kmax <= N/2, Sec. 3.2) applied to the initial field and to every nonlinear term, and
 * the RK2 of Sec. 4.1 without viscosity (S_half = S + dt/2 N(S), S_new = S + dt N(S_half)),
 * N(S) = T FFT[-sign(S) S^2] with the product taken on the grid.  nbatch independent fields:
 * s0 host [nbatch][N] physical initial values; out host [nbatch][N/2 + 1][2] the half spectra
 * S(k) = (1/N) sum_j S(x_j) e^{-i k x_j} after nsteps steps (nsteps = 0: the truncated initial
 * spectra).  FP64, one block per field on the current device; synchronous; allocates and
 * frees its own device buffers.  NS_ERR_INVALID_ARG for sizes or pointers outside these
 * ranges, NS_ERR_OOM / NS_ERR_CUDA on a CUDA failure. */
int ns_nl1d(int N, double kmax, double dt, int nsteps, int nbatch, const double* s0, double* out);

/* Measured CUDA-core FMA throughput of `device` in flop/s (2 flops per FMA) for precision
 * NS_FP32 or NS_FP64: one timed launch of independent FMA chains filling every SM (a few ms
 * in FP32, tens of ms in FP64).  It is the peak of the secondary, arithmetic roofline of the
 * FFT passes; the paper has no counterpart.  Allocates and frees one scalar; synchronises the
 * device's default stream.  Returns NS_ERR_INVALID_ARG for a null pointer or another
 * precision, NS_ERR_CUDA on a CUDA failure.  The current device is restored. */
int ns_fma_peak(int device, int precision, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* NS_H_ */
