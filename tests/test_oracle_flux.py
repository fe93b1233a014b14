"""Pins of the oracle's flux, cumulative dissipation and windowed error metrics.

Energy conservation of the rotational nonlinear term (exact on the grid, aliased or not),
the total dissipation, the inviscid shell-energy rate from the time-stepping oracle, shell
separation of the Taylor-Green initial state, closed forms of the windowed metrics."""
import math

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import nonlinear as nl
from oracle import schemes as sc
from oracle import spectral as sp
from paper_2603_08892_gb300 import inputs


@pytest.mark.parametrize("N,ct", [(12, 1.0), (16, 2.0 / 3.0), (16, 1.0)])
def test_flux_vanishes_at_the_last_shell(N, ct):
    kmax = ct * N / 2
    S = sp.set_velocity(inputs.random_solenoidal(N, 3, kcut=N / 2), kmax)
    dx = 2 * math.pi / N
    nb = int(math.ceil(math.sqrt(3) * N / 2)) + 2
    for delta in ([0, 0, 0], [dx / 2] * 3, [0.3 * dx, 0.1 * dx, 0.8 * dx]):
        Nl = nl.nonlinear(S, delta, kmax)
        P = dg.energy_flux(S, Nl, nb)
        assert np.abs(P).max() > 1e-6
        assert abs(P[-1]) < 1e-13 * np.abs(P).max()


def test_cumulative_dissipation_reaches_eps():
    N, nu = 16, 0.013
    S = sp.set_velocity(inputs.random_solenoidal(N, 4, kcut=N / 2), N / 2)
    D = dg.cumulative_dissipation(S, nu, 20)
    assert abs(D[-1] - dg.dissipation(S, nu)) < 1e-15 * D[-1] * 20
    assert np.all(np.diff(D) >= 0) and D[0] == 0.0


def test_transfer_is_the_inviscid_shell_energy_rate():
    # dE(k)/dt = T(k) for du/dt = N(u) (nu = 0): central difference of the oracle's RK4
    N = 12
    kmax = 2 * math.sqrt(2) / 3 * N / 2  # alias-free: the unshifted term is the exact one
    prob = sc.Problem(N, 0.0, kmax)
    S = sp.set_velocity(inputs.random_solenoidal(N, 5, kcut=4), kmax)
    nb = 12
    T = dg.transfer_spectrum(S, prob.NL(S), nb)
    h = 1e-4
    Sp = sc.step_rk4(S, h, prob)
    Sm = sc.step_rk4(S, -h, prob)
    dE = (dg.spectrum(Sp, dg.SPEC_SHELL, nb) - dg.spectrum(Sm, dg.SPEC_SHELL, nb)) / (2 * h)
    assert np.abs(T).max() > 1e-3
    np.testing.assert_allclose(dE, T, atol=1e-7 * np.abs(T).max())


def test_taylor_green_initial_transfer_is_zero():
    # u on the shell sqrt(3), N(u) on the shells 2 and 2 sqrt(2): no overlap
    N = 16
    S = sp.set_velocity(inputs.taylor_green(N), N / 2)
    T = dg.transfer_spectrum(S, nl.nonlinear(S, [0, 0, 0], N / 2), 12)
    assert np.abs(T).max() < 1e-17


def test_windowed_error_metrics_closed_forms():
    k = np.arange(20, dtype=float)
    ref = (1.0 + k, 2.0 + k, 3.0 + k)
    up = tuple(1.1 * r for r in ref)
    down = tuple(0.9 * r for r in ref)
    # constant 10 % error: every metric is 10
    e, l, m = dg.error_index_windows([up, up, up, up], [ref] * 4, 15.0)
    assert abs(e - 10) < 1e-12 and abs(l - 10) < 1e-12 and abs(m - 10) < 1e-12
    # +10 % then -10 %: 10 in each window, 0 for the time-averaged spectra
    e, l, m = dg.error_index_windows([up, up, down, down], [ref] * 4, 15.0)
    assert abs(e - 10) < 1e-12 and abs(l - 10) < 1e-12 and abs(m) < 1e-12
    # early window only: late metric 0
    e, l, m = dg.error_index_windows([up, ref], [ref, ref], 15.0)
    assert abs(e - 10) < 1e-12 and l == 0.0 and abs(m - 5) < 1e-12
