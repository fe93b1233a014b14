"""GPU tests of ns_step_diag (Sec. 3.4 diagnostics every step): the E and eps series it returns
agree with the oracle's energy and dissipation of the state after each step and with ns_energy;
the states it leaves are bitwise those of ns_step (the fused sums do not touch the step's
arithmetic); every scheme, both precisions, the forced split scheme, the generic kernels'
separate reduction, the full 256^3 bench workload, and the argument checks."""
import numpy as np
import pytest

from oracle import diagnostics as od
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

SCHEMES = [0, 1, 2, 3, 4]  # RK2, RK4, PS exact, PS approx, PS random


def _pair(ns, N, code, prec, nu, steps, dt, forced=False, seed=9):
    """(series of step_diag, per-step energy() and states of a twin context run by ns_step)"""
    kmax = N / 2 if code != 1 else N / 3
    u = inputs.taylor_green_perturbed(N, seed=4)
    with ns.Solver(N, nu, kmax, scheme=code, precision=prec, seed=seed) as a, \
            ns.Solver(N, nu, kmax, scheme=code, precision=prec, seed=seed) as b:
        for s in (a, b):
            if forced:
                s.set_forcing(2.0, 3.0, 0.1, 0.5, seed=3)
            s.set_velocity(u)
        E, eps = a.step_diag(dt, steps)
        ref, states = [], []
        for _ in range(steps):
            b.step(dt, 1)
            ref.append(b.energy())
            states.append(b.get_state())
        return E, eps, np.array(ref), states, a.get_state(), a.time()


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("code", SCHEMES)
def test_series_match_energy_and_oracle(ns, code, prec):
    N, nu, steps, dt = 32, 0.005, 4, 0.02
    E, eps, ref, states, last, (t, n) = _pair(ns, N, code, prec, nu, steps, dt)
    assert n == steps and abs(t - steps * dt) < 1e-12
    tol = 1e-12 if prec == 1 else 2e-6
    assert np.allclose(E, ref[:, 0], rtol=tol, atol=0) and np.allclose(eps, ref[:, 1], rtol=tol, atol=0)
    # the oracle's definitions (Hermitian weights, 1/2 and nu) on the states after each step
    oE = np.array([od.energy(S) for S in states])
    oD = np.array([od.dissipation(S, nu) for S in states])
    assert np.allclose(E, oE, rtol=tol, atol=0) and np.allclose(eps, oD, rtol=tol, atol=0)
    # step_diag's state is ns_step's, bit for bit
    assert np.array_equal(last, states[-1])


def test_forced_split_series(ns):
    E, eps, ref, states, last, _ = _pair(ns, 32, 4, 0, 0.01, 5, 0.01, forced=True)
    assert np.allclose(E, ref[:, 0], rtol=2e-6, atol=0) and np.allclose(eps, ref[:, 1], rtol=2e-6, atol=0)
    assert np.array_equal(last, states[-1])


def test_generic_kernels_reduction(ns, monkeypatch):
    # contexts created with the generic kernels take E, eps by a separate reduction per step
    monkeypatch.setenv("NS_GENERIC_KERNELS", "1")
    E, eps, ref, states, last, _ = _pair(ns, 16, 4, 1, 0.01, 3, 0.02)
    assert np.allclose(E, ref[:, 0], rtol=1e-14, atol=0) and np.allclose(eps, ref[:, 1], rtol=1e-14, atol=0)
    assert np.array_equal(last, states[-1])


def test_carry_across_calls_and_growth(ns):
    # a short call, a longer one (the series buffers grow), then plain steps: one trajectory
    N, dt = 32, 0.01
    u = inputs.taylor_green(N)
    with ns.Solver(N, 1 / 1600, N / 2, scheme=ns.RK2_PS_RANDOM, precision=ns.FP64, seed=2) as a, \
            ns.Solver(N, 1 / 1600, N / 2, scheme=ns.RK2_PS_RANDOM, precision=ns.FP64, seed=2) as b:
        a.set_velocity(u)
        b.set_velocity(u)
        E1, _ = a.step_diag(dt, 2)
        E2, _ = a.step_diag(dt, 7)
        a.step(dt, 1)
        b.step(dt, 10)
        assert np.array_equal(a.get_state(), b.get_state())
        Eb, _ = b.energy()
        Ea, _ = a.energy()
        assert Ea == Eb
    assert len(E1) == 2 and len(E2) == 7 and np.all(np.diff(np.concatenate([E1, E2])) < 0)


def test_full_size_bench_workload(ns):
    N, dt = 256, 9 / 1467
    with ns.Solver(N, 1 / 1600, 128.0, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=12345) as a:
        a.set_velocity(inputs.taylor_green(N))
        E, eps = a.step_diag(dt, 3)
        Ea, epsa = a.energy()
    assert abs(E[-1] - Ea) < 1e-6 * Ea and abs(eps[-1] - epsa) < 1e-6 * epsa
    # Taylor-Green: E0 = 1/8 decays by about eps0 dt per step (eps0 = 3 nu / 4)
    assert abs(E[0] - (0.125 - 0.75 / 1600 * dt)) < 1e-6
    assert np.all(np.diff(E) < 0)


def test_arguments(ns):
    with ns.Solver(16, 0.01, 8.0, precision=ns.FP64) as s:
        with pytest.raises(ns.NSError) as e:
            s.step_diag(0.01, 2)  # no state yet
        assert e.value.code == 8
        s.set_velocity(inputs.taylor_green(16))
        for dt, n in [(0.0, 1), (-1.0, 1), (float("nan"), 1), (0.01, -1)]:
            with pytest.raises(ns.NSError) as e:
                s.step_diag(dt, n)
            assert e.value.code == 1
        E, eps = s.step_diag(0.01, 0)
        assert len(E) == 0 and s.time() == (0.0, 0)
