"""The precision policy, measured: the error of each GPU result against the FP64 oracle.

Every test records its measured error through the ``report`` fixture (the table of errors per
result) and asserts the bound of the policy: FP64 path <= 1e-11 relative L2 after 100 steps;
FP32 <= 2e-5 relative L2 per step and <= 1e-4 relative error of the kinetic energy over a
run.  Results that are not a step (the nonlinear term alone, spectra) carry the bound derived
for them in their docstring.
"""
import math

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import nonlinear as onl
from oracle import schemes as sc
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

NU = 1.0 / 1600


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def field(N, seed):
    return inputs.random_solenoidal(N, seed, kcut=N / 2, energy_total=0.5)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N", [32, 64])
def test_step_error_per_size(ns, report, N, prec):
    kmax, dt = N / 2, 0.5 * math.pi / N
    u = field(N, 100 + N)
    da = [0.3 * 2 * math.pi / N, 0.7 * 2 * math.pi / N, 0.45 * 2 * math.pi / N]
    with ns.Solver(N, NU, kmax, scheme=ns.RK2_PS_RANDOM, precision=prec) as s:
        s.set_velocity(u)
        s.set_shifts([da])
        s.step(dt, 1)
        got = s.get_state()
    ref = sc.step_ps_random(osp.set_velocity(u, kmax), dt, sc.Problem(N, NU, kmax), da)
    err = rel(got, ref)
    tol = 2e-5 if prec == 0 else 1e-12
    report("rogallo_step_broadband_N%d_%s" % (N, "fp64" if prec else "fp32"), err, tol)
    assert err < tol


@pytest.mark.parametrize("N", [32, 64])
def test_fp64_after_100_steps(ns, report, N):
    kmax = N / 2
    dt = 0.5 * math.pi / N
    u = inputs.taylor_green_perturbed(N, 7)
    with ns.Solver(N, NU, kmax, scheme=ns.RK2_PS_RANDOM, precision=ns.FP64, seed=12345) as s:
        s.set_velocity(u)
        s.step(dt, 100)
        got = s.get_state()
    ref, _ = sc.run(osp.set_velocity(u, kmax), dt, 100, sc.Problem(N, NU, kmax),
                    sc.SCHEME_PS_RANDOM, seed=12345)
    err = rel(got, ref)
    report("rogallo_100_steps_taylor_green_1pct_N%d_fp64" % N, err, 1e-11)
    assert err < 1e-11


@pytest.mark.parametrize("N", [32, 64])
def test_fp32_energy_over_a_run(ns, report, N):
    # E(t) of a 100-step FP32 run (E of every step, fused into the final pencil pass) against
    # the oracle's FP64 trajectory; also the whole state after the run
    kmax = N / 2
    dt = 0.5 * math.pi / N
    u = inputs.taylor_green_perturbed(N, 8)
    with ns.Solver(N, NU, kmax, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=12345) as s:
        s.set_velocity(u)
        E, eps = s.step_diag(dt, 100)
        got = s.get_state()
    Er, Dr = [], []

    def cb(n, t, S):
        Er.append(dg.energy(S))
        Dr.append(dg.dissipation(S, NU))

    ref, _ = sc.run(osp.set_velocity(u, kmax), dt, 100, sc.Problem(N, NU, kmax),
                    sc.SCHEME_PS_RANDOM, seed=12345, callback=cb)
    eE = float(np.max(np.abs(np.asarray(E) - Er) / np.asarray(Er)))
    eD = float(np.max(np.abs(np.asarray(eps) - Dr) / np.asarray(Dr)))
    eS = rel(got, ref)
    report("energy_100_steps_N%d_fp32" % N, eE, 1e-4)
    report("dissipation_100_steps_N%d_fp32" % N, eD, 1e-4)
    report("state_after_100_steps_N%d_fp32" % N, eS, None)
    assert eE < 1e-4 and eD < 1e-4


@pytest.mark.parametrize("prec", [0, 1])
def test_spectra_error(ns, report, prec):
    """Shell and 1D spectra of the same state: FP64 sums of FP32 (or FP64) per-mode terms.

    Bound: a spectrum bin is a sum of |S|^2 over its modes; the state is stored in the
    working precision (relative rounding u = 2^-24 in FP32), so each term carries 2u and the
    bins (relative L2 over bins) at most a few u: 1e-6 FP32, 1e-13 FP64."""
    N = 64
    kmax = N / 2
    S = osp.set_velocity(field(N, 5), kmax)
    with ns.Solver(N, NU, kmax, precision=prec) as s:
        s.set_state(S)
        Sg = s.get_state()  # the stored state (FP32-rounded in FP32)
        worst = 0.0
        for kind in (ns.SPEC_SHELL, ns.SPEC_X, ns.SPEC_Y, ns.SPEC_Z):
            nb = N // 2 + 1 if kind != ns.SPEC_SHELL else int(math.ceil(math.sqrt(3) * N / 2)) + 1
            got = s.spectrum(kind, nb)
            worst = max(worst, rel(got, dg.spectrum(S, kind, nb)))
            # against the spectrum of the stored state: the reduction alone
            assert rel(got, dg.spectrum(Sg, kind, nb)) < (1e-12 if prec == 0 else 1e-14)
    tol = 1e-6 if prec == 0 else 1e-13
    report("spectra_N64_%s" % ("fp64" if prec else "fp32"), worst, tol)
    assert worst < tol


@pytest.mark.parametrize("N", [16, 32, 64, 96])
def test_fp32_nonlinear_term_error(ns, report, N):
    """FP32 nonlinear term N~(S) against the oracle.

    The term is formed from 6 inverse and 3 forward 3D transforms and a pointwise product;
    its relative error is that of the transforms (a few u sqrt(log2 N^3)), times the ratio
    |u x w| / |P(u x w)| that the projection's cancellation amplifies.  The bound 2e-5 is
    the per-step tolerance of the policy applied to the term itself."""
    kmax = N / 2
    S = osp.set_velocity(field(N, 11), kmax)
    dx = 2 * math.pi / N
    worst = 0.0
    with ns.Solver(N, 0.0, kmax, precision=ns.FP32) as s:
        for delta in ([0, 0, 0], [dx / 2] * 3, [0.31 * dx, 0.77 * dx, 0.05 * dx]):
            got = s.nonlinear(delta, S)
            worst = max(worst, rel(got, onl.nonlinear(S, delta, kmax)))
    report("nonlinear_term_broadband_N%d_fp32" % N, worst, 2e-5)
    assert worst < 2e-5
