"""Pins of the oracle's time schemes: exact solutions, orders, alias cancellation, forcing."""
import math

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import forcing as fo
from oracle import nonlinear as nl
from oracle import rng
from oracle import schemes as sc
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs

ALL = [sc.SCHEME_RK2, sc.SCHEME_RK4, sc.SCHEME_PS_EXACT, sc.SCHEME_PS_APPROX, sc.SCHEME_PS_RANDOM]


def test_splitmix64_published_first_output():
    # splitmix64 seeded with 0: first output 0xE220A8397B1DCDAF (published sequence)
    assert rng.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert rng.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    u = [rng.uniform01(12345, n) for n in range(2000)]
    assert min(u) >= 0.0 and max(u) < 1.0 and abs(np.mean(u) - 0.5) < 0.02
    N = 32
    da = rng.shift_alpha(12345, 7, N)
    db = rng.shift_beta(da, N)
    dx = 2 * math.pi / N
    assert all(0 <= d < dx for d in da)
    assert all(abs(b - a - dx / 2) < 1e-16 for a, b in zip(da, db))


@pytest.mark.parametrize("scheme", ALL)
def test_2d_taylor_green_decays_exactly(scheme):
    # P(u x w) = 0 for the 2D cells, so every integrating-factor scheme is exact: e^{-2 nu t}
    N, nu, dt = 12, 0.05, 0.1
    prob = sc.Problem(N, nu, N / 2)
    S0 = sp.set_velocity(inputs.taylor_green_2d(N), N / 2)
    S, t = sc.run(S0, dt, 5, prob, scheme, seed=3)
    np.testing.assert_allclose(S, S0 * math.exp(-2 * nu * t), atol=1e-15)


def _one_step_errors(step, ref, S0, dts):
    return [np.abs(step(S0, dt) - ref(S0, dt)).max() for dt in dts]


def _ref_rk4(prob, nlf=None, sub=64):
    def ref(S0, dt):
        S = S0
        for _ in range(sub):
            S = sc.step_rk4(S, dt / sub, prob, nl=nlf)
        return S
    return ref


def test_rk2_and_rk4_local_orders():
    N = 12
    kmax = 2.0 / 3.0 * N / 2  # alias-free: errors are pure time-discretisation errors
    prob = sc.Problem(N, 0.01, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 21, kcut=4, energy_total=2.0), kmax)
    ref = _ref_rk4(prob)
    dts = [0.04, 0.02]
    e2 = _one_step_errors(lambda S, dt: sc.step_rk2(S, dt, prob), ref, S0, dts)
    e4 = _one_step_errors(lambda S, dt: sc.step_rk4(S, dt, prob), ref, S0, dts)
    assert 2 ** 2.7 < e2[0] / e2[1] < 2 ** 3.3   # dt^3
    assert 2 ** 4.6 < e4[0] / e4[1] < 2 ** 5.4   # dt^5


def test_ps_exact_equals_padded_rk2_at_2sqrt2_over_3():
    N = 12
    kmax = 2 * math.sqrt(2) / 3 * N / 2
    prob = sc.Problem(N, 0.01, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 22, kcut=N / 2, energy_total=1.0), kmax)
    dt = 0.02
    a = sc.step_ps_exact(S0, dt, prob)
    b = sc.step_rk2(S0, dt, prob, nl=lambda S: nl.nonlinear_padded(S, kmax))
    assert np.abs(a - b).max() < 1e-15
    c = sc.step_rk2(S0, dt, prob)  # plain RK2 is aliased
    assert np.abs(c - b).max() > 1e-8


def _heun_padded(prob, kmax):
    """Rogallo's two-stage combination with alias-free (3/2-padded) products."""
    def step(S0, dt):
        Eh, E1 = prob.E(0.5 * dt), prob.E(dt)
        N0 = nl.nonlinear_padded(S0, kmax)
        S1 = (S0 + dt * N0) * E1
        N1 = nl.nonlinear_padded(S1, kmax)
        return S0 * E1 + dt * Eh * 0.5 * (N0 + N1)
    return step


@pytest.mark.parametrize("random_shift", [False, True])
def test_rogallo_residual_alias_is_dt2(random_shift):
    # at C_t = 2 sqrt(2)/3 the double aliases are truncated; single and triple aliases of
    # the two stages cancel up to O(dt) in N_a, so the one-step residual is O(dt^2)
    N = 12
    kmax = 2 * math.sqrt(2) / 3 * N / 2
    prob = sc.Problem(N, 0.01, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 23, kcut=N / 2, energy_total=1.0), kmax)
    da = [0.3 * prob.dx, 0.8 * prob.dx, 0.55 * prob.dx] if random_shift else [0, 0, 0]
    ref = _heun_padded(prob, kmax)
    dts = [0.02, 0.01, 0.005]
    e = [np.abs(sc.step_ps_random(S0, dt, prob, da) - ref(S0, dt)).max() for dt in dts]
    assert 2 ** 1.8 < e[0] / e[1] < 2 ** 2.2 and 2 ** 1.8 < e[1] / e[2] < 2 ** 2.2


def test_state_stays_solenoidal_hermitian_masked():
    N = 12
    kmax = N / 2
    prob = sc.Problem(N, 1e-3, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 24, kcut=N / 2, energy_total=1.0), kmax)
    for scheme in ALL:
        S, _ = sc.run(S0, 0.01, 3, prob, scheme, seed=5)
        assert sp.divergence_ratio(S) < 1e-13
        assert np.abs(S[:, ~sp.truncation_mask(N, kmax)]).max() == 0.0
        p0 = S[:, :, :, 0]
        mirror = np.conj(p0[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
        assert np.abs(p0 - mirror).max() < 1e-15


def test_inviscid_energy_drift_is_third_order():
    N = 12
    kmax = N / 2
    prob = sc.Problem(N, 0.0, kmax)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 25, kcut=N / 2, energy_total=1.0), kmax)
    E0 = dg.energy(S0)
    d = [abs(dg.energy(sc.step_rk2(S0, dt, prob)) - E0) for dt in (0.02, 0.01)]
    # at least third order per step (the truncated term conserves energy exactly)
    assert d[0] / d[1] > 2 ** 2.7 and d[1] > 0


def test_taylor_green_inviscid_enstrophy_series():
    # Z(t) = (3/8) [1 + (5/48) t^2 + O(t^4)] for the inviscid Taylor-Green vortex
    N = 16
    kmax = 2.0 / 3.0 * N / 2
    prob = sc.Problem(N, 0.0, kmax)
    S = sp.set_velocity(inputs.taylor_green(N), kmax)
    assert abs(dg.enstrophy(S) - 3 / 8) < 1e-15
    S, t = sc.run(S, 0.01, 10, prob, sc.SCHEME_RK4)
    coef = (dg.enstrophy(S) / (3 / 8) - 1) / t ** 2
    assert abs(coef - 5 / 48) < 0.002


def test_forcing_injects_eps_dt_exactly_and_is_real_solenoidal():
    N = 12
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.5, seed=2026)
    S = sp.set_velocity(inputs.hit_initial(N, 9), N / 2)
    modes = fo.shell_modes(N, 2.0, 3.0)
    assert len(modes) > 10
    for t, dt in ((0.0, 0.01), (0.37, 0.003), (1.2, 0.02)):
        O = f.term(S, t, dt)
        assert abs(dg.energy(S + dt * O) - dg.energy(S) - 1.0 * dt) < 1e-14
        assert sp.divergence_ratio(O) < 1e-14
        p0 = O[:, :, :, 0]
        mirror = np.conj(p0[:, (-np.arange(N)) % N][:, :, (-np.arange(N)) % N])
        assert np.abs(p0 - mirror).max() < 1e-16
        KX, KY, KZ = sp.wavenumbers(N)
        K2 = KX ** 2 + KY ** 2 + KZ ** 2
        assert np.abs(O[:, (K2 < 4) | (K2 > 9)]).max() == 0.0
    # time correlation: the pattern is continuous and piecewise linear in t
    a, b, c = f.pattern_at(0.2), f.pattern_at(0.25), f.pattern_at(0.3)
    np.testing.assert_allclose(b, 0.5 * (a + c), atol=1e-15)


def test_split_scheme_reduces_to_random_without_forcing():
    N = 12
    prob = sc.Problem(N, 1e-3, N / 2)
    S0 = sp.set_velocity(inputs.hit_initial(N, 10), N / 2)
    da = rng.shift_alpha(1, 0, N)
    a = sc.step_ps_random(S0, 0.01, prob, da)
    f = fo.Forcing(N, 2.0, 3.0, 0.0, 0.5, seed=1)  # eps = 0: a = 0
    b = sc.step_ps_random(S0, 0.01, prob, da, forcing=f)
    np.testing.assert_allclose(a, b, atol=0)


def test_cfl_step_taylor_green_closed_form():
    # Taylor-Green: max|u_x| = max|u_y| = 1 on grids with N divisible by 4, u_z = 0, so
    # dt = cfl dx / 2 (capped at dt_max)
    from oracle import schemes as scx
    for N in (8, 16, 32):
        S = sp.set_velocity(inputs.taylor_green(N), N / 2)
        dx = 2 * math.pi / N
        assert abs(scx.cfl_time_step(S, [0, 0, 0], 0.4, 1.0, N) - 0.4 * dx / 2) < 1e-15
        assert scx.cfl_time_step(S, [0, 0, 0], 0.4, 0.01, N) == 0.01
    # a half-cell shift samples the field away from its maxima: the step gets longer
    S = sp.set_velocity(inputs.taylor_green(8), 4.0)
    dx = 2 * math.pi / 8
    assert scx.cfl_time_step(S, [dx / 2] * 3, 0.4, 1.0, 8) > 0.4 * dx / 2


def test_cfl_run_scales_with_the_velocity_and_caps():
    from oracle import schemes as scx
    N = 16
    prob = scx.Problem(N, 0.01, N / 2)
    S0 = sp.set_velocity(inputs.random_solenoidal(N, 2, kcut=5, energy_total=1.0), N / 2)
    _, t1, d1 = scx.run_cfl(S0, 0.4, 1.0, 3, prob, scx.SCHEME_RK2)
    # a velocity twice as large gives half the first step (CFL ~ 1/|u|)
    _, _, d2 = scx.run_cfl(2 * S0, 0.4, 1.0, 1, prob, scx.SCHEME_RK2)
    assert abs(d2[0] - d1[0] / 2) < 1e-15 * d1[0]
    assert abs(t1 - sum(d1)) < 1e-15
    # with a cap below every CFL step the run is the fixed-step run
    S_a, t_a, d_a = scx.run_cfl(S0, 10.0, 1e-3, 3, prob, scx.SCHEME_PS_RANDOM, seed=4)
    S_b, t_b = scx.run(S0, 1e-3, 3, prob, scx.SCHEME_PS_RANDOM, seed=4)
    assert d_a == [1e-3] * 3 and np.array_equal(S_a, S_b) and t_a == t_b
