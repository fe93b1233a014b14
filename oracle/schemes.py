"""Time-stepping schemes of the oracle, written in the paper's stage notation.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).

Paper passages followed (Section 4.1, Eq. base-eq and the stage rule after it; Section
4.2; Section 6.1, Eq. forcing-eq):

* d_t S = sigma S + N(S) (+ O(S)), sigma = -nu |k|^2, the linear term integrated exactly;
* a stage of duration tau from t0 uses an approximate state S_a and nonlinear term N_a.
  Reading of the stage rule (the paper writes both the log form N_a/S_a and a first-order
  form): S(t0 + tau) = S0 E_tau + tau E_{tau - tau_a} N_a, where S_a is the state at time
  t0 + tau_a and E_t = exp(sigma t).  For tau_a = 0 this is (S0 + tau N_a) E_tau; with
  S_a = S0 E_{dt/2} it is exactly Eq. (Rogallo1981);
* RK2: stage 1 tau = dt/2 with N0; stage 2 tau = dt with N1 = N(S1), S1 at t0 + dt/2;
* RK2 phase-shift exact (Patterson & Orszag): RK2 with each N replaced by the average of
  the unshifted and the isotropically shifted (Delta = dx/2 in every direction) terms;
* RK2 phase-shift random (Rogallo): stage 1 tau = dt, S1 = (S0 + dt N~0a) E_dt; stage 2
  S = S0 E_dt + dt E_{dt/2} (N~0a + N~1b)/2 with shifts delta_alpha, delta_beta;
  "approx" is the special case delta_alpha = 0, delta_beta = dx/2 (1, 1, 1);
* RK2 phase-shift random split (forced): N~0a + O0 in stage 1, (N~0a + N~1b + O0 + O1)/2
  in stage 2, O1 = O(S1);
* RK4: the paper defers to the Fluidsim documentation; reading used: the textbook Lawson
  (integrating-factor) RK4 with unshifted evaluations.

Every scheme returns the new state; a forcing object (oracle.forcing.Forcing) is optional.
"""
import math

import numpy as np

from . import spectral as sp
from .nonlinear import nonlinear


class Problem:
    """Grid size, viscosity, truncation (N, nu, kmax, kind) of a run; L = 2*pi."""

    def __init__(self, N, nu, kmax, kind=sp.TRUNC_SPHERICAL):
        self.N, self.nu, self.kmax, self.kind = N, nu, kmax, kind
        self.dx = 2.0 * math.pi / N

    def E(self, tau):
        return sp.integrating_factor(self.N, self.nu, tau)

    def NL(self, S, delta=(0.0, 0.0, 0.0)):
        return nonlinear(S, delta, self.kmax, self.kind)

    def iso(self):
        return [0.5 * self.dx] * 3


def _force(forcing, S, t, dt):
    return 0.0 if forcing is None else forcing.term(S, t, dt)


def step_rk2(S0, dt, prob, t=0.0, forcing=None, nl=None):
    """Integrating-factor RK2 (midpoint): stages (dt/2, S0, N0) then (dt, S1, N1).

    ``nl`` overrides the nonlinear evaluation (used for phase-shift exact and the padded
    alias-free reference).
    """
    nl = prob.NL if nl is None else nl
    Eh, E1 = prob.E(0.5 * dt), prob.E(dt)
    N0 = nl(S0) + _force(forcing, S0, t, dt)
    S1 = (S0 + 0.5 * dt * N0) * Eh
    N1 = nl(S1) + _force(forcing, S1, t + 0.5 * dt, dt)
    return S0 * E1 + dt * Eh * N1


def step_ps_exact(S0, dt, prob, t=0.0, forcing=None):
    """RK2 phase-shift exact: N -> (N(S) + N~_iso(S)) / 2 at both stages (Sections 4.1-4.2)."""
    iso = prob.iso()

    def avg(S):
        return 0.5 * (prob.NL(S) + prob.NL(S, iso))

    return step_rk2(S0, dt, prob, t, forcing, nl=avg)


def step_ps_random(S0, dt, prob, delta_alpha, t=0.0, forcing=None, return_stages=False):
    """RK2 phase-shift random (Rogallo), and its split variant when ``forcing`` is given.

    Stage 1: tau = dt, S_a = S0, N_a = N~0a (+ O0)      -> S1 = (S0 + dt N_a) E_dt
    Stage 2: tau = dt, S_a = S0 E_{dt/2},
             N_a = (N~0a + N~1b (+ O0 + O1)) / 2          -> S0 E_dt + dt E_{dt/2} N_a
    delta_beta = delta_alpha + dx/2 (1, 1, 1).
    """
    da = list(delta_alpha)
    db = [d + 0.5 * prob.dx for d in da]
    Eh, E1 = prob.E(0.5 * dt), prob.E(dt)
    N0 = prob.NL(S0, da)
    O0 = _force(forcing, S0, t, dt)
    S1 = (S0 + dt * (N0 + O0)) * E1
    N1 = prob.NL(S1, db)
    O1 = _force(forcing, S1, t + dt, dt)
    S = S0 * E1 + dt * Eh * 0.5 * (N0 + N1 + O0 + O1)
    if return_stages:
        return S, S1
    return S


def step_ps_approx(S0, dt, prob, t=0.0, forcing=None):
    """RK2 phase-shift approx: the random scheme with delta_alpha = 0 (Section 4.1, Eq. Rogallo1981)."""
    return step_ps_random(S0, dt, prob, (0.0, 0.0, 0.0), t, forcing)


def step_rk4(S0, dt, prob, t=0.0, forcing=None, nl=None):
    """Lawson integrating-factor RK4 (reading: textbook form, unshifted evaluations).

    k1 = N(S0);               S1 = (S0 + dt/2 k1) E_{dt/2}
    k2 = N(S1);               S2 = S0 E_{dt/2} + dt/2 k2
    k3 = N(S2);               S3 = S0 E_dt + dt E_{dt/2} k3
    k4 = N(S3);  S = S0 E_dt + dt/6 (k1 E_dt + 2 E_{dt/2} (k2 + k3) + k4)
    """
    nl = prob.NL if nl is None else nl
    Eh, E1 = prob.E(0.5 * dt), prob.E(dt)
    k1 = nl(S0) + _force(forcing, S0, t, dt)
    S1 = (S0 + 0.5 * dt * k1) * Eh
    k2 = nl(S1) + _force(forcing, S1, t + 0.5 * dt, dt)
    S2 = S0 * Eh + 0.5 * dt * k2
    k3 = nl(S2) + _force(forcing, S2, t + 0.5 * dt, dt)
    S3 = S0 * E1 + dt * Eh * k3
    k4 = nl(S3) + _force(forcing, S3, t + dt, dt)
    return S0 * E1 + dt / 6.0 * (k1 * E1 + 2.0 * Eh * (k2 + k3) + k4)


SCHEME_RK2 = 0
SCHEME_RK4 = 1
SCHEME_PS_EXACT = 2
SCHEME_PS_APPROX = 3
SCHEME_PS_RANDOM = 4


def run(S0, dt, nsteps, prob, scheme, shifts=None, seed=None, forcing=None, t0=0.0,
        step0=0, callback=None):
    """Advance ``nsteps`` steps; ``shifts[n]`` (or the splitmix64 draw for ``seed``) gives
    delta_alpha of step n for the random scheme.  Time accumulates as t += dt."""
    from . import rng

    S, t = S0.copy(), t0
    for n in range(nsteps):
        if scheme == SCHEME_RK2:
            S = step_rk2(S, dt, prob, t, forcing)
        elif scheme == SCHEME_RK4:
            S = step_rk4(S, dt, prob, t, forcing)
        elif scheme == SCHEME_PS_EXACT:
            S = step_ps_exact(S, dt, prob, t, forcing)
        elif scheme == SCHEME_PS_APPROX:
            S = step_ps_approx(S, dt, prob, t, forcing)
        elif scheme == SCHEME_PS_RANDOM:
            if shifts is not None:
                da = shifts[n]
            else:
                da = rng.shift_alpha(seed, step0 + n, prob.N)
            S = step_ps_random(S, dt, prob, da, t, forcing)
        else:
            raise ValueError("unknown scheme")
        t = t + dt
        if callback is not None:
            callback(n, t, S)
    return S, t


def cfl_time_step(S, delta, cfl, dt_max, N):
    """Adaptive step of the CFL condition (Section 2; reading: dt = cfl / sum_i(max|u_i| / dx),
    the maxima over the grid values of the velocity shifted by ``delta``, capped at dt_max)."""
    u = sp.inverse(S * sp.shift_factor(N, delta))
    dx = 2.0 * math.pi / N
    freq = sum(float(np.abs(u[i]).max()) / dx for i in range(3))
    return dt_max if freq <= 0.0 else min(dt_max, cfl / freq)


def run_cfl(S0, cfl, dt_max, nsteps, prob, scheme, seed=None, forcing=None, t0=0.0, step0=0,
            callback=None):
    """Advance ``nsteps`` adaptive steps: each step's dt comes from the velocity that its
    first nonlinear evaluation forms (shifted by delta_alpha for the random scheme, unshifted
    otherwise).  Returns (S, t, list of the steps' dt)."""
    from . import rng

    S, t, dts = S0.copy(), t0, []
    N = prob.N
    for n in range(nsteps):
        da = rng.shift_alpha(seed, step0 + n, N) if scheme == SCHEME_PS_RANDOM else [0.0, 0.0, 0.0]
        dt = cfl_time_step(S, da, cfl, dt_max, N)
        if scheme == SCHEME_PS_RANDOM:
            S = step_ps_random(S, dt, prob, da, t, forcing)
        else:
            S, _ = run(S, dt, 1, prob, scheme, t0=t, forcing=forcing)
        t = t + dt
        dts.append(dt)
        if callback is not None:
            callback(n, t, S)
    return S, t, dts
