"""GPU parity of the nonlinear energy flux and cumulative dissipation (ns_energy_flux)
against the FP64 oracle, and their invariants at the full bench size."""
import math

import numpy as np
import pytest

from oracle import diagnostics as dg
from oracle import nonlinear as onl
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(1, 1e-12), (0, 2e-5)])
@pytest.mark.parametrize("N,trunc", [(16, 0), (24, 2), (32, 0)])
def test_flux_and_cumulative_dissipation_match_oracle(ns, N, trunc, prec, tol):
    kmax, nu = N / 2, 0.02
    u = inputs.random_solenoidal(N, 9, kcut=N / 2, energy_total=1.0)
    S = osp.set_velocity(u, kmax, trunc)
    nb = int(math.ceil(math.sqrt(3) * N / 2)) + 1
    dx = 2 * math.pi / N
    with ns.Solver(N, nu, kmax, truncation=trunc, precision=prec) as s:
        s.set_velocity(u)
        for shifts in (None, [[dx / 2] * 3], [[0, 0, 0], [dx / 2] * 3], [[0.3 * dx, 0.9 * dx, 0.1 * dx]]):
            flux, cum = s.energy_flux(nb, shifts)
            sh = shifts if shifts else [[0, 0, 0]]
            Nl = sum(onl.nonlinear(S, d, kmax, trunc) for d in sh) / len(sh)
            ref = dg.energy_flux(S, Nl, nb)
            assert np.abs(flux - ref).max() < tol * np.abs(ref).max()
            cref = dg.cumulative_dissipation(S, nu, nb)
            assert np.abs(cum - cref).max() < tol * cref[-1]


def test_full_size_invariants(ns):
    N, kmax = 256, 128.0
    dt = 9.0 / math.ceil(9.0 / (0.5 * (2 * math.pi / N) / 2.0))
    with ns.Solver(N, 1.0 / 1600, kmax, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=1) as s:
        s.set_velocity(inputs.taylor_green(N))
        s.step(dt, 400)
        E, eps = s.energy()
        dx = 2 * math.pi / N
        flux, cum = s.energy_flux(230, [[0, 0, 0], [dx / 2] * 3])
        E2, eps2 = s.energy()
    assert E2 == E and eps2 == eps  # the state is unchanged
    assert abs(flux[-1]) < 1e-4 * np.abs(flux).max()  # conservation of the truncated term
    assert abs(cum[-1] - eps) < 1e-6 * eps
    assert flux.max() > 0  # a forward transfer towards small scales has begun
    assert np.all(cum[int(kmax) + 1:] == cum[-1])  # nothing beyond the truncation


def test_flux_argument_checks(ns):
    with ns.Solver(16, 0.01, 8.0) as s:
        with pytest.raises(ns.NSError):
            s.energy_flux(0)
        with pytest.raises(ns.NSError):
            s.energy_flux(10, [[float("nan"), 0, 0]])
