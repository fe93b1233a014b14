"""The cluster slab pass (one z-plane per thread-block cluster, kept on chip) against the oracle.

The pass computes the same slab transform as the three-kernel pass (inverse y, c2r x, u x omega,
r2c x, forward y; Sec. 3.1's pseudo-spectral product) with the plane exchanged through
distributed shared memory instead of an HBM scratch.  Forced on with NS_SLAB_CLUSTER=1 (the
autotuner may also choose it), it must give the oracle's step within the precision policy's
tolerances, the three-kernel pass's result to FP32 rounding, and the same CFL maxima.
"""
import math

import numpy as np
import pytest

from oracle import rng as orng
from oracle import schemes as sc
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

NU = 1.0 / 1600


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(ns, monkeypatch, tmp_path, cluster, N, prec, u, nsteps=1, dt=None, seed=12345, variant=1):
    monkeypatch.setenv("NS_SLAB_CLUSTER", "1" if cluster else "0")
    monkeypatch.setenv("NS_CL_VARIANT", str(variant))
    monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    dt = 0.5 * math.pi / N if dt is None else dt
    with ns.Solver(N, NU, N / 2, scheme=ns.RK2_PS_RANDOM, precision=prec, seed=seed) as s:
        s.set_velocity(u)
        s.profile(True)
        s.step(dt, nsteps)
        prof = s.profile_read()
        return s.get_state(), prof


@pytest.mark.parametrize("N,prec,variant", [(128, 0, 1), (128, 1, 0), (256, 0, 0), (256, 0, 1)])
def test_cluster_slab_step_matches_oracle(ns, report, monkeypatch, tmp_path, N, prec, variant):
    # variant 0: 384 threads per CTA (two butterflies each), 1: 768 threads
    u = inputs.random_solenoidal(N, 500 + N, kcut=N / 2, energy_total=0.5)
    got, prof = run(ns, monkeypatch, tmp_path, True, N, prec, u, variant=variant)
    assert prof["k_slabcl"][2] == 2, prof  # both slab passes of the step ran on clusters
    assert prof["k_yinv"][2] == 0
    old = osp.set_fft_workers(8)
    try:
        ref = sc.step_ps_random(osp.set_velocity(u, N / 2), 0.5 * math.pi / N, sc.Problem(N, NU, N / 2),
                                orng.shift_alpha(12345, 0, N))
    finally:
        osp.set_fft_workers(old)
    err = rel(got, ref)
    tol = 2e-5 if prec == 0 else 1e-12
    report("cluster_slab_rogallo_step_broadband_N%d_%s_v%d" % (N, "fp64" if prec else "fp32", variant), err, tol)
    assert err < tol
    three, prof3 = run(ns, monkeypatch, tmp_path, False, N, prec, u)
    assert prof3["k_slabcl"][2] == 0
    assert rel(got, three) < (1e-6 if prec == 0 else 1e-14)


def test_cluster_slab_many_steps_and_cfl(ns, monkeypatch, tmp_path):
    # 20 steps of the benchmark workload at 256^3 through both slab passes, and the adaptive
    # CFL step (its velocity maxima are reduced inside the slab pass)
    N = 256
    u = inputs.taylor_green_perturbed(N, 3)
    a, _ = run(ns, monkeypatch, tmp_path, True, N, 0, u, nsteps=20, dt=9.0 / 1467)
    b, _ = run(ns, monkeypatch, tmp_path, False, N, 0, u, nsteps=20, dt=9.0 / 1467)
    assert rel(a, b) < 1e-6
    dts = []
    for cluster in (True, False):
        monkeypatch.setenv("NS_SLAB_CLUSTER", "1" if cluster else "0")
        monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
        with ns.Solver(N, NU, N / 2, scheme=ns.RK2_PS_RANDOM, precision=0, seed=4) as s:
            s.set_velocity(u)
            s.step_cfl(0.4, 0.01, 3)
            t, n = s.time()
            dts.append(t)
    assert abs(dts[0] - dts[1]) < 1e-7 * dts[1]


@pytest.mark.parametrize("N", [128, 256])
def test_tile_variants_match_oracle(ns, report, monkeypatch, tmp_path, N):
    # every compiled tile alternative the autotuner may choose (pencil width, inverse-y width,
    # x rows, forward-y width), forced on, against the oracle and the defaults
    u = inputs.random_solenoidal(N, 900 + N, kcut=N / 2, energy_total=0.5)
    monkeypatch.setenv("NS_SLAB_CLUSTER", "0")
    monkeypatch.setenv("NS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    dt = 0.5 * math.pi / N
    states = {}
    for v in (0, 15, 16):
        monkeypatch.setenv("NS_TILE_VARIANT", str(v))
        with ns.Solver(N, NU, N / 2, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=12345) as s:
            s.set_velocity(u)
            s.step(dt, 1)
            states[v] = s.get_state()
    old = osp.set_fft_workers(8)
    try:
        ref = sc.step_ps_random(osp.set_velocity(u, N / 2), dt, sc.Problem(N, NU, N / 2),
                                orng.shift_alpha(12345, 0, N))
    finally:
        osp.set_fft_workers(old)
    err = rel(states[15], ref)
    report("tile_alternatives_rogallo_step_N%d_fp32" % N, err, 2e-5)
    assert err < 2e-5
    assert rel(states[15], states[0]) < 1e-6
    assert rel(states[16], ref) < 2e-5 and rel(states[16], states[0]) < 1e-6
