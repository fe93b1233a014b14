"""GPU parity of the adaptive CFL time step (ns_step_cfl) against the oracle's adaptive run:
same per-step dt (from the velocity maxima reduced inside the slab pass), same states and
accumulated time, for every scheme; full-size behaviour at 256^3."""
import math

import numpy as np
import pytest

from oracle import schemes as sc
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

SCHEMES = {"rk2": (0, sc.SCHEME_RK2), "rk4": (1, sc.SCHEME_RK4), "exact": (2, sc.SCHEME_PS_EXACT),
           "approx": (3, sc.SCHEME_PS_APPROX), "random": (4, sc.SCHEME_PS_RANDOM)}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec,tol", [(1, 1e-11), (0, 1e-4)])
@pytest.mark.parametrize("name", list(SCHEMES))
def test_adaptive_steps_match_oracle(ns, name, prec, tol):
    code, oscheme = SCHEMES[name]
    N, nu, cfl = 16, 0.01, 0.4 if name != "rk4" else 1.0
    kmax = N / 2
    u = inputs.random_solenoidal(N, 12, kcut=6, energy_total=1.0)
    with ns.Solver(N, nu, kmax, scheme=code, precision=prec, seed=21) as s:
        s.set_velocity(u)
        s.step_cfl(cfl, 0.05, 12)
        got = s.get_state()
        t, n = s.time()
    prob = sc.Problem(N, nu, kmax)
    ref, tref, dts = sc.run_cfl(osp.set_velocity(u, kmax), cfl, 0.05, 12, prob, oscheme, seed=21)
    assert n == 12 and max(dts) < 0.05  # the CFL bound is active, not the cap
    assert abs(t - tref) < (1e-14 if prec == 1 else 1e-6) * tref
    assert rel(got, ref) < tol


def test_taylor_green_first_step_closed_form(ns):
    N = 32
    dx = 2 * math.pi / N
    with ns.Solver(N, 1.0 / 1600, N / 2, scheme=ns.RK2, precision=ns.FP64) as s:
        s.set_velocity(inputs.taylor_green(N))
        s.step_cfl(0.4, 1.0, 1)
        t, _ = s.time()
    assert abs(t - 0.4 * dx / 2) < 1e-14


def test_full_size_adaptive_rogallo(ns):
    N = 256
    dx = 2 * math.pi / N
    with ns.Solver(N, 1.0 / 1600, 128.0, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=3) as s:
        s.set_velocity(inputs.taylor_green(N))
        s.step_cfl(0.4, 1.0, 20)
        t, n = s.time()
        E, eps = s.energy()
    # max|u_x| = max|u_y| ~ 1 and u_z grows from 0 (du_z/dt = (cos 2x + cos 2y) sin 2z / 8 at
    # t = 0, so about 0.02 by t = 0.1): dt within a few per cent of 0.4 dx / 2
    nominal = 20 * 0.4 * dx / 2
    assert n == 20 and 0.97 * nominal <= t <= 1.02 * nominal
    assert np.isfinite(E) and abs(E - 0.125) < 1e-3


def test_cfl_argument_checks(ns):
    with ns.Solver(16, 0.01, 8.0) as s:
        s.set_velocity(inputs.taylor_green(16))
        for args in ((0.0, 0.1), (0.4, 0.0), (float("inf"), 0.1)):
            with pytest.raises(ns.NSError):
                s.step_cfl(*args, 1)
