"""Pins of the 1D quadratic-model oracle (Section 3.3) against closed forms and the paper's
statements about where the aliases of the first RK2 step land."""
import numpy as np

from oracle import nl1d


def test_first_evaluation_closed_form_aliased():
    # -S0^2 = -(1.245 + 1.4 cos 10x + 0.245 cos 20x); on N = 22 points cos 20x = cos 2x, so the
    # 2 k0 harmonic appears at 2 k_N - 20 = 2 (Section 3.3), with the half-spectrum weight 1/2
    N, kmax = 22, 11.0
    Nh = nl1d.nonlinear(nl1d.to_spectral(nl1d.initial(N)), N, kmax)
    ref = np.zeros(N // 2 + 1, complex)
    ref[0], ref[10], ref[2] = -1.245, -0.7, -0.1225
    assert np.max(np.abs(Nh - ref)) < 1e-14


def test_two_thirds_rule_removes_the_alias():
    # N = 32, C_t = 2/3 (kmax = 10.67, k0 = 10 kept): 20 aliases to 12 and is truncated
    N, kmax = 32, 2.0 / 3.0 * 16
    Nh = nl1d.nonlinear(nl1d.to_spectral(nl1d.initial(N)), N, kmax)
    ref = np.zeros(N // 2 + 1, complex)
    ref[0], ref[10] = -1.245, -0.7
    assert np.max(np.abs(Nh - ref)) < 1e-14
    # after one RK2 step only k = 0 and k0 carry energy: every alias was removed
    S1 = nl1d.run(nl1d.initial(N), 0.1, 1, kmax)
    nz = np.nonzero(np.abs(S1) > 1e-14)[0]
    assert set(nz) == {0, 10}


def test_one_step_aliases_of_the_paper():
    # N = 22, C_t = 1: the harmonics k_nl1 = 20 and k_nl2 = 30 land at 2 and 8; a resolved
    # grid has nothing there and carries them at 20 and 30 instead
    dt = 0.1
    S22 = nl1d.run(nl1d.initial(22), dt, 1, 11.0)
    S128 = nl1d.run(nl1d.initial(128), dt, 1, 64.0)
    assert abs(S22[2]) > 1e-3 and abs(S22[8]) > 1e-4
    assert abs(S128[2]) < 1e-14 and abs(S128[8]) < 1e-14
    assert abs(S128[20]) > 1e-3 and abs(S128[30]) > 1e-4
    # the k = 8 alias of 30 equals, to leading order, the resolved k = 30 amplitude
    assert abs(S22[8] - S128[30]) < 0.2 * abs(S128[30])


def test_one_step_taylor_expansion():
    # resolved: S(dt) = S0 - dt S0^2 + dt^2 S0^3 + O(dt^3) (Section 3.3)
    N = 256
    s0 = nl1d.initial(N)
    for dt in (1e-2, 5e-3):
        s1 = nl1d.to_physical(nl1d.run(s0, dt, 1, N / 2), N)
        err = np.max(np.abs(s1 - (s0 - dt * s0 ** 2 + dt ** 2 * s0 ** 3)))
        assert err < 2.0 * dt ** 3 * np.max(s0) ** 4


def test_converges_to_the_exact_solution():
    # S_exact = S0 / (1 + S0 t) (Eq. 1d_exact); RK2 global error ~ dt^2
    N, t = 256, 0.5
    s0 = nl1d.initial(N)
    exact = s0 / (1 + s0 * t)
    errs = []
    for n in (50, 100):
        s = nl1d.to_physical(nl1d.run(s0, t / n, n, N / 2), N)
        errs.append(np.max(np.abs(s - exact)))
    assert errs[1] < 1e-4 and 3.6 < errs[0] / errs[1] < 4.4


def test_sign_of_negative_fields():
    # -sign(S) S^2 = -S |S|: a negative constant field decays in magnitude too, as
    # S0 / (1 + |S0| t) (dS/dt = +S^2 for S < 0); -S^2 instead would make it blow up
    N = 16
    Sh = nl1d.run(-0.5 * np.ones(N), 0.01, 100, N / 2)
    assert abs(Sh[0].real - (-0.5 / (1 + 0.5 * 1.0))) < 1e-5 and np.max(np.abs(Sh[1:])) < 1e-15
