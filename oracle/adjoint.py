"""Adjoint (transposed linearisation) of the phase-shift RK2 step, for gradients.

TEST INFRASTRUCTURE ONLY (see :mod:`oracle`).  The paper has no adjoint; this module
differentiates the schemes of :mod:`oracle.schemes` exactly (discrete adjoint), so it is
pinned by a dot-product test and by central finite differences, not by the paper.

Inner products.  Spectral states use <a, b>_w = sum_half w Re(conj(a) . b) (w = 1 at kx = 0,
2 elsewhere), which is the full-spectrum sum and, by Parseval with the 1/N^3 forward
convention, (1/N^3) times the physical dot product.  With it:
  * pointwise multiplication by c(k) has adjoint conj(c(k)); the truncation T, the
    projection P and the integrating factors are self-adjoint; the curl ik x is self-adjoint;
  * the forward transform F (physical dot product -> <.,.>_w) has adjoint F^{-1} / N^3.

Nonlinear term N~_D(S) = T P e^{-ik.D} F[u x w], u = F^{-1}(e^{ik.D} S), w = F^{-1}(ik x e^{ik.D} S):
  J*(rho) = T P e^{-ik.D} [ F(w x r) + ik x F(r x u) ],   r = F^{-1}(e^{ik.D} P T rho)
(from r . (du x w + u x dw) = du . (w x r) + dw . (r x u)).

Forcing O(S) = a(S) f with a the root of smaller modulus of a^2 (dt/2)<f,f> + a b - eps = 0,
b = Re<S, f>_w:  da/db = -|a| / sqrt(b^2 + 4 c eps), so the adjoint of S -> O(S) maps rho to
(da/db) Re<f, rho>_w f.

Loss: L = eps(S_T) = nu <S, k^2 S>_w, gradient 2 nu k^2 S.  A loss of the physical velocity
u(T) = F^{-1}(S_T) with gradient g = dL/du(T) has the cotangent (F^{-1})^* g = N^3 F(g) of S_T,
restricted to the truncated, divergence-free states by T and P (both self-adjoint).
"""
import numpy as np

from . import spectral as sp
from . import nonlinear as nl
from . import rng


def inner(a, b):
    N = a.shape[-2]
    return float(np.sum(sp.hermitian_weights(N) * np.real(np.sum(np.conj(a) * b, axis=0))))


def nl_jvp(S, dS, delta, kmax, kind=sp.TRUNC_SPHERICAL):
    """Directional derivative J dS of N~_D at S (N~ is quadratic: N(S+dS) - N(S) - N(dS))."""
    return (nl.nonlinear(S + dS, delta, kmax, kind) - nl.nonlinear(S, delta, kmax, kind)
            - nl.nonlinear(dS, delta, kmax, kind))


def nl_vjp(S, rho, delta, kmax, kind=sp.TRUNC_SPHERICAL):
    """J*(rho) for N~_D at S (formula in the module doc)."""
    N = S.shape[-2]
    sh = sp.shift_factor(N, delta)
    mask = sp.truncation_mask(N, kmax, kind)
    us = S * sh
    u = sp.inverse(us)
    w = sp.inverse(sp.curl(us))
    r = sp.inverse(sp.project(rho * mask) * sh)
    A = sp.forward(nl.cross(w, r))
    B = sp.forward(nl.cross(r, u))
    G = (A + sp.curl(B)) * np.conj(sh)
    return sp.project(G * mask)


def forcing_vjp(forcing, S, t, dt, rho):
    """Adjoint of S -> O(S) at time t applied to rho (zero without forcing)."""
    if forcing is None:
        return 0.0
    f = forcing.pattern_at(t)
    a = forcing.amplitude(S, f, dt)
    b = inner(S, f)
    c = 0.5 * dt * inner(f, f)
    q = np.sqrt(b * b + 4.0 * c * forcing.eps)
    dadb = -abs(a) / q
    return dadb * inner(f, rho) * f


def step_ps_random_vjp(S0, lam, dt, prob, delta_alpha, t=0.0, forcing=None):
    """Cotangent of S_n given the cotangent lam of S_{n+1} for one RK2 phase-shift random
    (split, when forcing is given) step of :func:`oracle.schemes.step_ps_random`."""
    da = list(delta_alpha)
    db = [d + 0.5 * prob.dx for d in da]
    Eh, E1 = prob.E(0.5 * dt), prob.E(dt)
    N0 = prob.NL(S0, da)
    O0 = 0.0 if forcing is None else forcing.term(S0, t, dt)
    S1 = (S0 + dt * (N0 + O0)) * E1
    rho = 0.5 * dt * Eh * lam
    lam_S1 = nl_vjp(S1, rho, db, prob.kmax, prob.kind) + forcing_vjp(forcing, S1, t + dt, dt, rho)
    sigma = dt * E1 * lam_S1
    rs = rho + sigma
    return (E1 * (lam + lam_S1) + nl_vjp(S0, rs, da, prob.kmax, prob.kind)
            + forcing_vjp(forcing, S0, t, dt, rs))


def dissipation_grad(S, nu):
    KX, KY, KZ = sp.wavenumbers(S.shape[-2])
    return 2.0 * nu * (KX * KX + KY * KY + KZ * KZ) * S


def _reverse(u0, nsteps, dt, prob, seed, forcing, ckpt_every, approx, seed_lam):
    """Forward sweep from u0 with checkpoints, then the reverse sweep from the cotangent
    seed_lam(S_T); returns (S_T, dL/du0 for the physical dot product)."""
    from .schemes import step_ps_random

    N = prob.N

    def shift(n):
        return [0.0, 0.0, 0.0] if approx else rng.shift_alpha(seed, n, N)

    S = sp.set_velocity(u0, prob.kmax, prob.kind)
    ckpt = {0: S.copy()}
    t = 0.0
    times = [0.0]
    for n in range(nsteps):
        S = step_ps_random(S, dt, prob, shift(n), t, forcing)
        t = t + dt
        times.append(t)
        if (n + 1) % ckpt_every == 0:
            ckpt[n + 1] = S.copy()
    lam = seed_lam(S)
    for seg0 in sorted([k for k in ckpt if k < nsteps], reverse=True):
        seg1 = min(seg0 + ckpt_every, nsteps)
        states = [ckpt[seg0]]
        for n in range(seg0, seg1 - 1):
            states.append(step_ps_random(states[-1], dt, prob, shift(n), times[n], forcing))
        for n in range(seg1 - 1, seg0 - 1, -1):
            lam = step_ps_random_vjp(states[n - seg0], lam, dt, prob, shift(n), times[n], forcing)
    mask = sp.truncation_mask(N, prob.kmax, prob.kind)
    return S, sp.inverse(sp.project(lam * mask)) / float(N) ** 3


def grad_final_state(u0, gT, nsteps, dt, prob, seed, forcing=None, ckpt_every=10, approx=False):
    """dL/du0 of a loss of the final velocity u(T) whose gradient is gT = dL/du(T)
    (physical [3, N, N, N]); the cotangent of S_T is N^3 P T F(gT) (module doc)."""
    N = prob.N
    mask = sp.truncation_mask(N, prob.kmax, prob.kind)

    def seed_lam(S):
        return sp.project(sp.forward(gT) * mask) * float(N) ** 3

    return _reverse(u0, nsteps, dt, prob, seed, forcing, ckpt_every, approx, seed_lam)[1]


def grad_final_dissipation(u0, nsteps, dt, prob, seed, forcing=None, ckpt_every=10,
                           approx=False):
    """L = eps(S_T) after nsteps RK2 phase-shift random steps from u0 (physical) and dL/du0.

    Forward states are kept only every ckpt_every steps and recomputed segment by segment
    in the backward sweep.  Returns (L, grad) with grad a physical field [3, N, N, N]
    (gradient with respect to the physical dot product).
    """
    from .diagnostics import dissipation

    S, grad = _reverse(u0, nsteps, dt, prob, seed, forcing, ckpt_every, approx,
                       lambda S_: dissipation_grad(S_, prob.nu))
    return dissipation(S, prob.nu), grad
