"""Pins of the oracle adjoint: dot-product tests and central finite differences."""
import math

import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import forcing as fo
from oracle import rng
from oracle import schemes as sc
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs


def rand_state(N, kmax, seed):
    return sp.set_velocity(inputs.random_solenoidal(N, seed, kcut=N / 2, energy_total=1.0), kmax)


@pytest.mark.parametrize("frac", [1.0, 2.0 / 3.0])
def test_nonlinear_dot_product(frac):
    N = 12
    kmax = frac * N / 2
    S, dS, rho = (rand_state(N, kmax, s) for s in (1, 2, 3))
    dx = 2 * math.pi / N
    for delta in ([0, 0, 0], [0.3 * dx, 0.8 * dx, 0.55 * dx]):
        lhs = ad.inner(rho, ad.nl_jvp(S, dS, delta, kmax))
        rhs = ad.inner(ad.nl_vjp(S, rho, delta, kmax), dS)
        assert abs(lhs - rhs) < 1e-13 * max(abs(lhs), 1e-3)
        assert abs(lhs) > 1e-6


def test_step_dot_product_with_forcing():
    N = 12
    kmax = N / 2
    prob = sc.Problem(N, 0.01, kmax)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.5, seed=4)
    S0, dS, lam = (rand_state(N, kmax, s) for s in (5, 6, 7))
    da = rng.shift_alpha(9, 0, N)
    dt, h = 0.01, 1e-6
    # J dS by central differences of the step (the step is smooth), lam . J dS vs J* lam . dS
    fp = sc.step_ps_random(S0 + h * dS, dt, prob, da, 0.3, f)
    fm = sc.step_ps_random(S0 - h * dS, dt, prob, da, 0.3, f)
    jv = (fp - fm) / (2 * h)
    lhs = ad.inner(lam, jv)
    rhs = ad.inner(ad.step_ps_random_vjp(S0, lam, dt, prob, da, 0.3, f), dS)
    assert abs(lhs - rhs) < 1e-8 * abs(lhs)


def test_forcing_amplitude_derivative():
    N = 12
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.5, seed=4)
    S, dS, rho = (rand_state(N, N / 2, s) for s in (11, 12, 13))
    h = 1e-6
    jv = (f.term(S + h * dS, 0.2, 0.01) - f.term(S - h * dS, 0.2, 0.01)) / (2 * h)
    lhs = ad.inner(rho, jv)
    rhs = ad.inner(ad.forcing_vjp(f, S, 0.2, 0.01, rho), dS)
    assert abs(lhs - rhs) < 1e-8 * max(abs(lhs), 1e-12)


@pytest.mark.parametrize("forced", [False, True])
def test_gradient_matches_central_differences(forced):
    N, nu, dt, nsteps = 12, 0.01, 0.01, 6
    kmax = N / 2
    prob = sc.Problem(N, nu, kmax)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.02, seed=7) if forced else None
    u0 = inputs.hit_initial(N, 7)
    L, g = ad.grad_final_dissipation(u0, nsteps, dt, prob, seed=3, forcing=f, ckpt_every=4)
    rs = np.random.default_rng(0)
    h = 1e-4
    for _ in range(3):
        v = rs.standard_normal(u0.shape)
        Lp, _ = ad.grad_final_dissipation(u0 + h * v, nsteps, dt, prob, 3, f, ckpt_every=100)
        Lm, _ = ad.grad_final_dissipation(u0 - h * v, nsteps, dt, prob, 3, f, ckpt_every=100)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - float(np.sum(g * v))) < 1e-6 * abs(fd)


def test_grad_final_state_central_differences():
    # L(u0) = sum_x gT . u(T): a linear functional of the final velocity (any loss's gradient
    # at T enters the reverse sweep this way); FP64 central differences, h = 1e-4
    from oracle import adjoint as ad
    from oracle import forcing as fo
    from oracle import schemes as sc
    from oracle import spectral as sp
    from paper_2603_08892_gb300 import inputs

    N, nu, dt, nsteps = 8, 0.02, 0.02, 5
    prob = sc.Problem(N, nu, N / 2)
    u0 = inputs.hit_initial(N, 3)
    rs = np.random.default_rng(4)
    gT = rs.standard_normal(u0.shape)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.05, seed=2)

    def L(u):
        S = sp.set_velocity(u, prob.kmax)
        for n in range(nsteps):
            S = sc.step_ps_random(S, dt, prob, __import__("oracle").rng.shift_alpha(9, n, N), n * dt, f)
        return float(np.sum(gT * sp.inverse(S)))

    g = ad.grad_final_state(u0, gT, nsteps, dt, prob, seed=9, forcing=f, ckpt_every=2)
    h = 1e-4
    for _ in range(3):
        v = rs.standard_normal(u0.shape)
        fd = (L(u0 + h * v) - L(u0 - h * v)) / (2 * h)
        assert abs(fd - float(np.sum(g * v))) < 1e-7 * max(1.0, abs(fd))


def test_grad_final_state_energy_equals_builtin_energy_gradient():
    # E(T) = (1/2) mean_x |u(T)|^2 has dE/du(T) = u(T) / N^3; through the state cotangent it
    # must give the same gradient as seeding the reverse sweep with dE/dS_T = S_T directly
    from oracle import adjoint as ad
    from oracle import schemes as sc
    from oracle import spectral as sp
    from paper_2603_08892_gb300 import inputs

    N, nu, dt, nsteps = 8, 0.02, 0.02, 4
    prob = sc.Problem(N, nu, N / 2)
    u0 = inputs.hit_initial(N, 5)
    S, _ = sc.run(sp.set_velocity(u0, prob.kmax), dt, nsteps, prob, sc.SCHEME_PS_RANDOM, seed=1)
    gT = sp.inverse(S) / float(N) ** 3
    g1 = ad.grad_final_state(u0, gT, nsteps, dt, prob, seed=1, ckpt_every=3)
    _, g2 = ad._reverse(u0, nsteps, dt, prob, 1, None, 3, False, lambda S_: S_.copy())
    assert np.abs(g1 - g2).max() < 1e-13 * np.abs(g2).max()
