"""Thin ctypes binding over libns.so (include/ns.h); argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  Importing this module loads the
library and raises ImportError when it is missing: there is no CPU fallback.

Arrays follow ns.h: physical velocity float64 [3, N, N, N] (x fastest); spectral state
complex128 [3, N, N, N//2] (index [c, kz, ky, kx], kz and ky in FFT order).
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libns.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libns.so is not built (run `python -m paper_2603_08892_gb300.build` or "
        "`python -c 'import __graft_entry__ as g; g.build()'`); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

NS_OK = 0
ERRORS = {1: "NS_ERR_INVALID_ARG", 2: "NS_ERR_UNSUPPORTED_N", 3: "NS_ERR_KMAX", 4: "NS_ERR_CUDA",
          5: "NS_ERR_OOM", 6: "NS_ERR_NONFINITE", 7: "NS_ERR_TIMEOUT", 8: "NS_ERR_STATE",
          9: "NS_ERR_INTERNAL", 10: "NS_ERR_IO"}
TRUNC_SPHERICAL, TRUNC_CUBIC, TRUNC_NO_DOUBLE_ALIAS = 0, 1, 2
RK2, RK4, RK2_PS_EXACT, RK2_PS_APPROX, RK2_PS_RANDOM = 0, 1, 2, 3, 4
FP32, FP64 = 0, 1
FORCE_NONE, FORCE_TCRANDOM_CONST_EPS = 0, 1
SPEC_SHELL, SPEC_X, SPEC_Y, SPEC_Z = 0, 1, 2, 3

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("nu", ctypes.c_double),
                ("kmax", ctypes.c_double), ("truncation", ctypes.c_int), ("scheme", ctypes.c_int),
                ("precision", ctypes.c_int), ("device", ctypes.c_int), ("stream", _vp),
                ("seed", ctypes.c_uint64)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_init_ex = _sig("ns_init_ex", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(Params)])
_init_error = _sig("ns_init_error", ctypes.c_char_p, [])
_destroy = _sig("ns_destroy", ctypes.c_int, [_vp])
_last_error = _sig("ns_last_error", ctypes.c_char_p, [_vp])
_set_velocity = _sig("ns_set_velocity", ctypes.c_int, [_vp, _dp])
_get_velocity = _sig("ns_get_velocity", ctypes.c_int, [_vp, _dp])
_get_state = _sig("ns_get_state", ctypes.c_int, [_vp, _dp])
_set_state = _sig("ns_set_state", ctypes.c_int, [_vp, _dp])
_set_forcing = _sig("ns_set_forcing", ctypes.c_int,
                    [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double, ctypes.c_uint64])
_step = _sig("ns_step", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int])
_step_cfl = _sig("ns_step_cfl", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int])
_step_diag = _sig("ns_step_diag", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _dp, _dp])
_ckpt_save = _sig("ns_checkpoint_save", ctypes.c_int, [_vp, ctypes.c_char_p])
_ckpt_load = _sig("ns_checkpoint_load", ctypes.c_int, [_vp, ctypes.c_char_p])
_set_shifts = _sig("ns_set_shifts", ctypes.c_int, [_vp, _dp, ctypes.c_int])
_nonlinear = _sig("ns_nonlinear", ctypes.c_int, [_vp, _dp, _dp, _dp])
_energy = _sig("ns_energy", ctypes.c_int, [_vp, _dp, _dp])
_spectrum = _sig("ns_energy_spectrum", ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.c_int])
_flux = _sig("ns_energy_flux", ctypes.c_int, [_vp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int])
_time = _sig("ns_time", ctypes.c_int, [_vp, _dp, ctypes.POINTER(ctypes.c_int64)])
_set_time = _sig("ns_set_time", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64])
_device_state = _sig("ns_device_state", ctypes.c_int,
                     [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int)])
_model_bytes = _sig("ns_model_bytes_per_step", ctypes.c_double, [_vp])
_rank_copy = _sig("ns_rank_copy", ctypes.c_int,
                  [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp])
_rank_pencil = _sig("ns_rank_pencil", ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int])
_rank_slab = _sig("ns_rank_slab", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int])
BUF_STATE, BUF_MIXED, BUF_FT, BUF_NL = 0, 1, 2, 3
RANK_INIT, RANK_NL = 0, 1
_vjp_state = _sig("ns_vjp_state", ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp])
_tape_forward = _sig("ns_tape_forward", ctypes.c_int,
                     [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _vp])
_tape_backward = _sig("ns_tape_backward", ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp])
_fma_peak = _sig("ns_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp])
_nl1d = _sig("ns_nl1d", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, _dp, _dp])
_profile = _sig("ns_profile", ctypes.c_int, [_vp, ctypes.c_int])
_profile_read = _sig("ns_profile_read", ctypes.c_int,
                     [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ctypes.c_int64)])
_nonlinear_noalloc = _sig("ns_nonlinear_noalloc", ctypes.c_int,
                         [_vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _vp])
_vjp = _sig("ns_vjp", ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, _dp, _dp])
LOSS_DISSIPATION, LOSS_ENERGY = 0, 1
_batch_init = _sig("ns_batch_init", ctypes.c_int,
                   [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp, _dp,
                    ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int, _vp])
_batch_destroy = _sig("ns_batch_destroy", ctypes.c_int, [_vp])
_batch_last_error = _sig("ns_batch_last_error", ctypes.c_char_p, [_vp])
_batch_member = _sig("ns_batch_member", _vp, [_vp, ctypes.c_int])
_batch_set_velocity = _sig("ns_batch_set_velocity", ctypes.c_int, [_vp, ctypes.c_int, _dp])
_batch_get_state = _sig("ns_batch_get_state", ctypes.c_int, [_vp, ctypes.c_int, _dp])
_batch_step = _sig("ns_batch_step", ctypes.c_int, [_vp, _dp, ctypes.c_int])
_batch_energy = _sig("ns_batch_energy", ctypes.c_int, [_vp, _dp, _dp])
_batch_spin = _sig("ns_batch_set_spin_limit", ctypes.c_int, [_vp, ctypes.c_longlong])
_batch_stall = _sig("ns_batch_test_stall", ctypes.c_int, [_vp, ctypes.c_int])
_batch_grid = _sig("ns_batch_grid", ctypes.c_int, [_vp])
_batch_set_schedule = _sig("ns_batch_set_schedule", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int])
_batch_schedule = _sig("ns_batch_schedule", ctypes.c_int,
                       [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)])
PROF_KINDS = {"k_pencil": 0, "k_yinv": 1, "k_xrow": 2, "k_yfwd": 3, "slab_pass": 4, "k_slabpipe": 5,
              "k_slabcl": 6}

EXPORTED = ["ns_init", "ns_init_ex", "ns_init_error", "ns_destroy", "ns_last_error",
            "ns_set_velocity", "ns_get_velocity", "ns_get_state", "ns_set_state",
            "ns_set_forcing", "ns_step", "ns_step_cfl", "ns_step_diag", "ns_set_shifts",
            "ns_checkpoint_save", "ns_checkpoint_load", "ns_nonlinear", "ns_energy",
            "ns_energy_spectrum", "ns_energy_flux", "ns_time", "ns_set_time", "ns_device_state",
            "ns_model_bytes_per_step", "ns_nl1d", "ns_fma_peak", "ns_profile", "ns_profile_read", "ns_nonlinear_noalloc", "ns_vjp", "ns_vjp_state", "ns_rank_copy", "ns_rank_pencil", "ns_rank_slab",
            "ns_tape_forward", "ns_tape_backward", "ns_batch_init", "ns_batch_destroy", "ns_batch_last_error",
            "ns_batch_member", "ns_batch_set_velocity", "ns_batch_get_state", "ns_batch_step",
            "ns_batch_energy", "ns_batch_set_spin_limit", "ns_batch_test_stall", "ns_batch_grid",
            "ns_batch_set_schedule", "ns_batch_schedule"]


class NSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def _ptr(a):
    return a.ctypes.data_as(_dp)


class Solver:
    """One libns context (owns its device memory; one GB300 stream)."""

    def __init__(self, N, nu, kmax, scheme=RK2_PS_RANDOM, truncation=TRUNC_SPHERICAL,
                 precision=FP32, device=0, stream=None, seed=0, L=2 * math.pi):
        p = Params(N, L, nu, kmax, truncation, scheme, precision, device,
                   _vp(stream) if stream else None, seed)
        h = _vp()
        rc = _init_ex(ctypes.byref(h), ctypes.byref(p))
        if rc != NS_OK:
            raise NSError(rc, _init_error().decode())
        self._h = h
        self.N, self.nu, self.kmax, self.scheme, self.precision = N, nu, kmax, scheme, precision

    def _check(self, rc):
        if rc != NS_OK:
            raise NSError(rc, _last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --- state ---------------------------------------------------------------------
    def set_velocity(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (3, self.N, self.N, self.N)
        self._check(_set_velocity(self._h, _ptr(u)))

    def get_velocity(self, out=None):
        """The physical velocity float64 [3, N, N, N]; `out` (C-contiguous float64, e.g. a view
        of pinned host memory) receives it when given."""
        u = np.empty((3, self.N, self.N, self.N)) if out is None else out
        if u.dtype != np.float64 or not u.flags["C_CONTIGUOUS"] or u.shape != (3, self.N, self.N, self.N):
            raise ValueError("out must be C-contiguous float64 of shape (3, N, N, N)")
        self._check(_get_velocity(self._h, _ptr(u)))
        return u

    def get_state(self):
        N = self.N
        s = np.empty((3, N, N, N // 2), dtype=np.complex128)
        self._check(_get_state(self._h, s.ctypes.data_as(_dp)))
        return s

    def set_state(self, S):
        S = np.ascontiguousarray(S, dtype=np.complex128)
        assert S.shape == (3, self.N, self.N, self.N // 2)
        self._check(_set_state(self._h, S.ctypes.data_as(_dp)))

    def set_forcing(self, kf_min=2.0, kf_max=3.0, eps=1.0, t_corr=0.5, seed=0,
                    kind=FORCE_TCRANDOM_CONST_EPS):
        self._check(_set_forcing(self._h, kind, kf_min, kf_max, eps, t_corr, seed))

    def step(self, dt, nsteps=1):
        self._check(_step(self._h, dt, nsteps))

    def step_cfl(self, cfl, dt_max, nsteps=1):
        """nsteps steps with dt = min(dt_max, cfl / sum_i(max|u_i| / dx)) each (ns_step_cfl)."""
        self._check(_step_cfl(self._h, float(cfl), float(dt_max), int(nsteps)))

    def step_diag(self, dt, nsteps=1):
        """nsteps steps of size dt; returns (E, eps) after each step as two arrays (ns_step_diag)."""
        n = int(nsteps)
        E = np.zeros(max(n, 1))
        eps = np.zeros(max(n, 1))
        self._check(_step_diag(self._h, float(dt), n, _ptr(E), _ptr(eps)))
        return E[:n], eps[:n]

    def checkpoint_save(self, path):
        """Write the state, time, step, seed and forcing to a file (ns_checkpoint_save)."""
        self._check(_ckpt_save(self._h, os.fsencode(path)))

    def checkpoint_load(self, path):
        """Restore a checkpoint written by a context of the same configuration."""
        self._check(_ckpt_load(self._h, os.fsencode(path)))

    def set_shifts(self, delta_alpha):
        d = np.ascontiguousarray(delta_alpha, dtype=np.float64).reshape(-1, 3)
        self._check(_set_shifts(self._h, _ptr(d), d.shape[0]))

    def nonlinear(self, delta, S=None):
        N = self.N
        out = np.empty((3, N, N, N // 2), dtype=np.complex128)
        d = np.ascontiguousarray(delta, dtype=np.float64)
        if S is not None:
            S = np.ascontiguousarray(S, dtype=np.complex128)
            sp = S.ctypes.data_as(_dp)
        else:
            sp = None
        self._check(_nonlinear(self._h, sp, _ptr(d), out.ctypes.data_as(_dp)))
        return out

    def energy(self):
        e = ctypes.c_double()
        d = ctypes.c_double()
        self._check(_energy(self._h, ctypes.byref(e), ctypes.byref(d)))
        return e.value, d.value

    def spectrum(self, kind=SPEC_SHELL, nbins=None):
        nbins = self.N // 2 + 1 if nbins is None else nbins
        out = np.empty(nbins)
        self._check(_spectrum(self._h, kind, _ptr(out), nbins))
        return out

    def energy_flux(self, nbins=None, shifts=None):
        """(flux Pi(k), cumulative dissipation D(k)) on shell bins (ns_energy_flux).

        shifts: list of shift vectors whose shifted nonlinear terms are averaged (None: the
        unshifted term)."""
        nbins = int(math.ceil(math.sqrt(3) * self.N / 2)) + 1 if nbins is None else nbins
        d = np.ascontiguousarray(np.asarray(shifts if shifts else [[0.0, 0.0, 0.0]], dtype=np.float64))
        ns_ = len(shifts) if shifts else 0
        flux = np.empty(nbins)
        cum = np.empty(nbins)
        self._check(_flux(self._h, _ptr(d), ns_, _ptr(flux), _ptr(cum), nbins))
        return flux, cum

    def time(self):
        t = ctypes.c_double()
        s = ctypes.c_int64()
        self._check(_time(self._h, ctypes.byref(t), ctypes.byref(s)))
        return t.value, s.value

    def set_time(self, t, step):
        self._check(_set_time(self._h, t, step))

    def device_state(self):
        s = _vp()
        st = _vp()
        p = ctypes.c_int()
        self._check(_device_state(self._h, ctypes.byref(s), ctypes.byref(st), ctypes.byref(p)))
        return s.value, st.value, p.value

    def model_bytes_per_step(self):
        return _model_bytes(self._h)

    def rank_get(self, buf, axis, lo, hi):
        """Block [lo, hi) of axis 0 (z / kz planes) or 1 (ky rows) of a buffer, complex128."""
        N, F = self.N, 5 if buf == BUF_MIXED else 3
        shape = (F, hi - lo, N, N // 2) if axis == 0 else (F, N, hi - lo, N // 2)
        out = np.empty(shape, dtype=np.complex128)
        self._check(_rank_copy(self._h, buf, axis, lo, hi, 0, out.ctypes.data_as(_dp)))
        return out

    def rank_set(self, buf, axis, lo, hi, block):
        b = np.ascontiguousarray(block, dtype=np.complex128)
        self._check(_rank_copy(self._h, buf, axis, lo, hi, 1, b.ctypes.data_as(_dp)))

    def rank_pencil(self, kind, delta, lo, hi):
        d = np.ascontiguousarray(delta, dtype=np.float64)
        self._check(_rank_pencil(self._h, kind, _ptr(d), lo, hi))

    def rank_slab(self, lo, hi):
        self._check(_rank_slab(self._h, lo, hi))

    def vjp_state(self, u0, nsteps, dt, gT, ckpt_every=10):
        """dL/du0 of a loss of u(T) whose gradient dL/du(T) is gT (see ns_vjp_state)."""
        u = np.ascontiguousarray(u0, dtype=np.float64)
        g = np.ascontiguousarray(gT, dtype=np.float64)
        out = np.empty_like(u)
        self._check(_vjp_state(self._h, _ptr(u), nsteps, dt, ckpt_every, _ptr(g), _ptr(out)))
        return out

    def tape_forward(self, u0_ptr, nsteps, dt, ckpt_every, uT_ptr):
        """ns_tape_forward on device pointers (reals of the context's precision)."""
        self._check(_tape_forward(self._h, _vp(u0_ptr), nsteps, dt, ckpt_every, _vp(uT_ptr)))

    def tape_backward(self, gT_ptr, grad_ptr, loss=LOSS_DISSIPATION):
        """ns_tape_backward on device pointers; gT_ptr None seeds with the built-in loss."""
        self._check(_tape_backward(self._h, _vp(gT_ptr) if gT_ptr else None, loss, _vp(grad_ptr)))

    def vjp(self, u0, nsteps, dt, ckpt_every=10, loss=LOSS_DISSIPATION):
        """(L, dL/du0) of the loss on the state after nsteps steps from u0 (see ns_vjp)."""
        u = np.ascontiguousarray(u0, dtype=np.float64)
        g = np.empty_like(u)
        L = ctypes.c_double()
        self._check(_vjp(self._h, _ptr(u), nsteps, dt, ckpt_every, loss, ctypes.byref(L), _ptr(g)))
        return L.value, g

    def profile(self, enable=True):
        self._check(_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (total_ms, timed_launches, launches)} since the last profile() call."""
        out = {}
        for name, k in PROF_KINDS.items():
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            nl = ctypes.c_int64()
            self._check(_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(nl)))
            out[name] = (ms.value, n.value, nl.value)
        return out


def nl1d(s0, kmax, dt, nsteps):
    """The 1D quadratic model of Sec. 3.3 (ns_nl1d): s0 [nbatch][N] (or [N]) physical initial
    fields; returns the complex half spectra [nbatch][N/2 + 1] (or [N/2 + 1]) after nsteps RK2
    steps."""
    s = np.ascontiguousarray(s0, dtype=np.float64)
    one = s.ndim == 1
    s = s.reshape(1, -1) if one else s
    nb, N = s.shape
    out = np.zeros((nb, N // 2 + 1, 2))
    rc = _nl1d(N, float(kmax), float(dt), int(nsteps), nb, _ptr(s), _ptr(out))
    if rc != NS_OK:
        raise NSError(rc, "ns_nl1d failed")
    z = out[..., 0] + 1j * out[..., 1]
    return z[0] if one else z


def fma_peak(precision=None, device=0):
    """Measured CUDA-core FMA throughput of the device in flop/s (ns_fma_peak)."""
    out = ctypes.c_double()
    rc = _fma_peak(device, FP32 if precision is None else precision, ctypes.byref(out))
    if rc != NS_OK:
        raise NSError(rc, "ns_fma_peak failed")
    return out.value


def nonlinear_noalloc(state_ptr, out_ptr, N, kmax, delta, truncation=TRUNC_SPHERICAL, stream=None):
    """ns_nonlinear_noalloc on caller-owned device buffers (complex64 [3, N, N, N//2]).

    For callers that cannot allocate device memory: the library works in one fixed array of
    its own (N <= 64), shared by every call, so calls that overlap on the GPU race.
    """
    d = np.ascontiguousarray(delta, dtype=np.float64)
    rc = _nonlinear_noalloc(_vp(state_ptr), _vp(out_ptr), N, kmax, truncation, _ptr(d),
                            _vp(stream) if stream else None)
    if rc != NS_OK:
        raise NSError(rc, "ns_nonlinear_noalloc failed")


class Batch:
    """Ensemble of independent members of uneven N advanced together (one persistent launch
    per call, or one grid launch per pass and size class: the schedule the tuner picks)."""

    def __init__(self, Ns, nus, kmaxs, seeds=None, scheme=RK2_PS_RANDOM, precision=FP32,
                 stream=None):
        n = len(Ns)
        Na = (ctypes.c_int * n)(*Ns)
        nu = np.ascontiguousarray(nus, dtype=np.float64)
        km = np.ascontiguousarray(kmaxs, dtype=np.float64)
        sd = (ctypes.c_uint64 * n)(*seeds) if seeds is not None else None
        h = _vp()
        rc = _batch_init(ctypes.byref(h), n, Na, _ptr(nu), _ptr(km), sd, scheme, precision,
                         _vp(stream) if stream else None)
        if rc != NS_OK:
            raise NSError(rc, "ns_batch_init failed")
        self._h = h
        self.Ns = list(Ns)
        self.count = n

    def _check(self, rc):
        if rc != NS_OK:
            raise NSError(rc, _batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_velocity(self, i, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._check(_batch_set_velocity(self._h, i, _ptr(u)))

    def get_state(self, i):
        N = self.Ns[i]
        s = np.empty((3, N, N, N // 2), dtype=np.complex128)
        self._check(_batch_get_state(self._h, i, s.ctypes.data_as(_dp)))
        return s

    def step(self, dts, nsteps):
        d = np.ascontiguousarray(np.broadcast_to(dts, (self.count,)), dtype=np.float64)
        self._check(_batch_step(self._h, _ptr(d), nsteps))

    def energy(self):
        E = np.empty(self.count)
        eps = np.empty(self.count)
        self._check(_batch_energy(self._h, _ptr(E), _ptr(eps)))
        return E, eps

    def set_spin_limit(self, polls):
        self._check(_batch_spin(self._h, polls))

    def test_stall(self, on):
        self._check(_batch_stall(self._h, 1 if on else 0))

    def grid(self):
        return _batch_grid(self._h)

    def set_schedule(self, gran, ctas_per_sm=0):
        """Tiles per work-list ticket and CTAs per SM of the persistent launch (no tuning);
        gran 0: the grid schedule (one launch per pass and size class)."""
        self._check(_batch_set_schedule(self._h, gran, ctas_per_sm))

    def schedule(self):
        g, q = ctypes.c_int(), ctypes.c_int()
        self._check(_batch_schedule(self._h, ctypes.byref(g), ctypes.byref(q)))
        return g.value, q.value
