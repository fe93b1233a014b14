"""Independent pins of the Rogallo two-stage combination (Section 4.1, Eq. Rogallo1981) and of
its forced split variant (Section 6.1, Eq. forcing-eq).

The oracle's ``step_ps_random`` is run as it stands; what it is compared with is derived
from the equation being integrated, not from the scheme's formulas:

* Linear test problem.  With the nonlinear term replaced by N(S) = lam S (lam a per-mode
  scalar), dS/dt = (sigma + lam) S has the exact solution S0 exp((sigma + lam) dt).  Writing
  x = sigma dt and y = lam dt, a Taylor expansion of Eq. Rogallo1981 by hand (stage 1:
  S1 = (S0 + dt N0) E_dt; stage 2: S0 E_dt + dt E_{dt/2} (N0 + N1) / 2) gives the one-step
  error
        S_scheme - S_exact = (x^2 y / 8 + x y^2 / 4 - y^3 / 6) S0 + O(dt^4).
  The y^3 / 6 term is Heun's constant (sigma = 0); the two mixed terms exist only because
  of the integrating factors, and each factor changes them: E_dt -> 1 in stage 1 flips the
  sign of x y^2 / 4, Lawson's weights (E_dt N0 + N1) / 2 in stage 2 remove both, and
  E_{dt/2} -> E_dt in stage 2 (or E_dt -> E_{dt/2} in stage 1) leaves an O(dt^2) error.
* Nonlinear problem at C_t = 2/3 (alias-free, so every shift gives the same term) with a
  viscosity large enough for the integrating factor to matter: the one-step error against a
  sub-stepped RK4 reference falls as dt^3 (second order).

The split variant is the same scheme with N + O in both stages; a linear forcing
O(S) = mu S therefore gives the same constant with y = (lam + mu) dt, and only if O1 is
evaluated on S1.
"""
import math

import numpy as np
import pytest

from oracle import schemes as sc
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs


class _LinearProblem(sc.Problem):
    """N(S) = lam S for every shift: the nonlinear term replaced by a per-mode scalar."""

    def __init__(self, N, nu, lam):
        super().__init__(N, nu, N / 2)
        self.lam = lam

    def NL(self, S, delta=(0.0, 0.0, 0.0)):
        return self.lam * S


class _LinearForcing:
    """Forcing term O(S) = mu S (the split variant's non-aliased term, linearised)."""

    def __init__(self, mu):
        self.mu = mu

    def term(self, S, t, dt):
        return self.mu * S


def _setup(N=8, nu=0.05, seed=4):
    rng = np.random.default_rng(seed)
    S0 = rng.standard_normal((3, N, N, N // 2)) + 1j * rng.standard_normal((3, N, N, N // 2))
    lam = rng.uniform(-2.0, 2.0, (3, N, N, N // 2))
    KX, KY, KZ = sp.wavenumbers(N)
    sigma = -nu * (KX * KX + KY * KY + KZ * KZ)
    return S0, lam, np.broadcast_to(sigma, lam.shape)


def _constant(x, y):
    return x * x * y / 8.0 + x * y * y / 4.0 - y ** 3 / 6.0


def _residual_slope(step, S0, sigma, y_rate, dts=(0.004, 0.002)):
    """log2 of the ratio of max|S - S_exact - predicted cubic term| at dt and dt/2.

    With the predicted constant the residual is O(dt^4) (slope 4); any other constant leaves
    an O(dt^3) residual (slope 3), a lower order a smaller slope still.
    """
    res = []
    for dt in dts:
        exact = S0 * np.exp((sigma + y_rate) * dt)
        pred = _constant(sigma * dt, y_rate * dt) * S0
        res.append(np.abs(step(dt) - exact - pred).max())
    return math.log2(res[0] / res[1])


@pytest.mark.parametrize("delta", [(0.0, 0.0, 0.0), (0.1, 0.5, 0.3)])
def test_rogallo_local_error_constant_on_linear_problem(delta):
    N, nu = 8, 0.05
    S0, lam, sigma = _setup(N, nu)
    prob = _LinearProblem(N, nu, lam)
    slope = _residual_slope(lambda dt: sc.step_ps_random(S0, dt, prob, delta), S0, sigma, lam)
    assert 3.7 < slope < 4.3


def test_rogallo_constant_distinguishes_the_stage_weights():
    # the two nearest alternative readings, evaluated by the same route, leave an O(dt^3)
    # residual: the pin tells them apart
    N, nu = 8, 0.05
    S0, lam, sigma = _setup(N, nu)

    def no_if_stage1(dt):  # stage 1 without its integrating factor on N0
        E1, Eh = np.exp(sigma * dt), np.exp(0.5 * sigma * dt)
        S1 = S0 * E1 + dt * lam * S0
        return S0 * E1 + dt * Eh * 0.5 * (lam * S0 + lam * S1)

    def lawson_stage2(dt):  # Lawson's IF-Heun weights (E_dt N0 + N1) / 2 in stage 2
        E1 = np.exp(sigma * dt)
        S1 = (S0 + dt * lam * S0) * E1
        return S0 * E1 + 0.5 * dt * (E1 * lam * S0 + lam * S1)

    for alt in (no_if_stage1, lawson_stage2):
        assert _residual_slope(alt, S0, sigma, lam) < 3.4


def test_split_variant_local_error_constant_with_linear_forcing():
    N, nu = 8, 0.05
    S0, lam, sigma = _setup(N, nu)
    mu = np.random.default_rng(9).uniform(-1.0, 1.0, lam.shape)
    prob = _LinearProblem(N, nu, lam)
    f = _LinearForcing(mu)
    slope = _residual_slope(lambda dt: sc.step_ps_random(S0, dt, prob, (0.2, 0.1, 0.7), forcing=f),
                            S0, sigma, lam + mu)
    assert 3.7 < slope < 4.3


@pytest.mark.parametrize("scheme", ["random", "approx"])
def test_rogallo_second_order_with_strong_viscosity(scheme):
    # C_t = 2/3: aliases are all truncated, the shifts are immaterial and the only error is
    # the time discretisation; nu = 0.05 makes sigma dt comparable to the nonlinear rate
    N, nu = 12, 0.05
    kmax = 2.0 / 3.0 * N / 2
    prob = sc.Problem(N, nu, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 31, kcut=4, energy_total=2.0), kmax)

    def ref(dt, sub=64):
        S = S0
        for _ in range(sub):
            S = sc.step_rk4(S, dt / sub, prob)
        return S

    da = [0.37 * prob.dx, 0.11 * prob.dx, 0.83 * prob.dx]
    errs = []
    for dt in (0.04, 0.02, 0.01):
        S = sc.step_ps_approx(S0, dt, prob) if scheme == "approx" else sc.step_ps_random(S0, dt, prob, da)
        errs.append(np.abs(S - ref(dt)).max())
    assert 2 ** 2.7 < errs[0] / errs[1] < 2 ** 3.3
    assert 2 ** 2.7 < errs[1] / errs[2] < 2 ** 3.3


def test_fft_workers_do_not_change_the_oracle():
    # the threaded transforms (used at 256^3 and above) give the single-thread values
    N = 16
    S = sp.set_velocity(inputs.random_solenoidal(N, 5, kcut=N / 2, energy_total=1.0), N / 2)
    a = sc.step_ps_random(S, 0.01, sc.Problem(N, 0.01, N / 2), (0.1, 0.2, 0.3))
    old = sp.set_fft_workers(2)
    try:
        b = sc.step_ps_random(S, 0.01, sc.Problem(N, 0.01, N / 2), (0.1, 0.2, 0.3))
    finally:
        sp.set_fft_workers(old)
    assert np.abs(a - b).max() < 1e-15 * max(1.0, np.abs(a).max()) * 10
