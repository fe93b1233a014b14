"""Element-wise parity of the size-specialised kernels that the benchmark times, at full size.

One step of the compiled instance at each size (256^3 FP32 -- the benchmarked Rogallo step --
and FP64; 128^3 and 192^3 FP32; RK4 + 2/3 at 384^3 FP32; the forced split step of the
512^3 HIT workload) through the C ABI, compared with
one FP64 oracle step on the whole state (relative L2, Sections 4.1-4.2: the shifted and
de-shifted term and Eq. Rogallo1981; RK4: the Lawson reading).  The oracle uses threaded
pocketfft transforms so each full-size step takes seconds.

Inputs: a broadband seeded solenoidal field filling the whole truncation sphere (every tile
and column of every kernel sees nonzero data), and the benchmark's own Taylor-Green field with
a seeded 1 % perturbation.  The launch configuration is the one the benchmark runs (the
autotuned slab plan of the device).

Tolerances: FP32 2e-5 relative L2 per step, FP64 1e-12 per step (the precision policy).
"""
import math
import os

import numpy as np
import pytest

from oracle import forcing as fo
from oracle import rng as orng
from oracle import schemes as sc
from oracle import spectral as osp
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu

NU = 1.0 / 1600
SEED = 12345


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dt_of(N):
    # the benchmark's step: CFL 0.5 with the frequency summed over directions, t = 9 on a step
    dt = 0.5 / (2.0 / (2 * math.pi / N))
    return 9.0 / math.ceil(9.0 / dt)


@pytest.fixture(scope="module", autouse=True)
def threaded_oracle():
    old = osp.set_fft_workers(len(os.sched_getaffinity(0)))
    yield
    osp.set_fft_workers(old)


_cache = {}


def broadband(N):
    if ("bb", N) not in _cache:
        _cache[("bb", N)] = inputs.random_solenoidal(N, 4242 + N, kcut=N / 2, energy_total=0.5)
    return _cache[("bb", N)]


def oracle_rogallo(N, u, key):
    if key not in _cache:
        kmax = N / 2
        S0 = osp.set_velocity(u, kmax)
        da = orng.shift_alpha(SEED, 0, N)
        _cache[key] = sc.step_ps_random(S0, dt_of(N), sc.Problem(N, NU, kmax), da)
    return _cache[key]


def gpu_rogallo(ns, N, u, prec):
    with ns.Solver(N, NU, N / 2, scheme=ns.RK2_PS_RANDOM, precision=prec, seed=SEED) as s:
        s.set_velocity(u)
        s.step(dt_of(N), 1)
        return s.get_state()


@pytest.mark.parametrize("N,prec", [(256, 0), (256, 1), (128, 0), (192, 0), (128, 1)])
def test_rogallo_step_broadband_full_size(ns, report, N, prec):
    u = broadband(N)
    ref = oracle_rogallo(N, u, ("rog", N))
    got = gpu_rogallo(ns, N, u, prec)
    err = rel(got, ref)
    tol = 2e-5 if prec == 0 else 1e-12
    report("rogallo_step_broadband_N%d_%s" % (N, "fp64" if prec else "fp32"), err, tol)
    assert err < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_rogallo_step_bench_field_256(ns, report, prec):
    # the benchmark's Taylor-Green field, with a seeded 1 % solenoidal perturbation on |k| <= 4
    N = 256
    u = inputs.taylor_green_perturbed(N, 2026)
    ref = oracle_rogallo(N, u, ("tgp", N))
    got = gpu_rogallo(ns, N, u, prec)
    err = rel(got, ref)
    tol = 2e-5 if prec == 0 else 1e-12
    report("rogallo_step_taylor_green_1pct_N256_%s" % ("fp64" if prec else "fp32"), err, tol)
    assert err < tol


def test_rk4_step_384_fp32(ns, report):
    # the comparison leg: RK4 + 2/3 spherical truncation at 384^3 (kmax = 128)
    N, kmax = 384, 128.0
    u = broadband(N)
    S0 = osp.set_velocity(u, kmax)
    ref = sc.step_rk4(S0, dt_of(N), sc.Problem(N, NU, kmax))
    with ns.Solver(N, NU, kmax, scheme=ns.RK4, precision=ns.FP32) as s:
        s.set_velocity(u)
        s.step(dt_of(N), 1)
        got = s.get_state()
    err = rel(got, ref)
    report("rk4_step_broadband_N384_fp32", err, 2e-5)
    assert err < 2e-5


def test_forced_split_step_hit_512_fp32(ns, report):
    # the forced-turbulence workload: 512^3 RK2 phase-shift random with the constant-rate
    # forcing on the shell 2 <= |k| <= 3 (the split reading of Sec. 6.1), seeded HIT field,
    # nu = kmax^(-4/3), CFL 0.4; one step against the FP64 oracle (about 50 GB of host memory)
    N, kmax = 512, 256.0
    nu = kmax ** (-4.0 / 3.0)
    u = inputs.hit_initial(N, 2026)
    umax = np.abs(u).reshape(3, -1).max(axis=1)
    dt = 0.4 / float(np.sum(umax / (2 * math.pi / N)))
    with ns.Solver(N, nu, kmax, scheme=ns.RK2_PS_RANDOM, precision=ns.FP32, seed=2026) as s:
        s.set_velocity(u)
        s.set_forcing(2.0, 3.0, 1.0, 0.5, seed=2026)
        s.step(dt, 1)
        got = s.get_state()
    forcing = fo.Forcing(N, 2.0, 3.0, 1.0, 0.5, seed=2026)
    S0 = osp.set_velocity(u, kmax)
    del u
    ref, _ = sc.run(S0, dt, 1, sc.Problem(N, nu, kmax), sc.SCHEME_PS_RANDOM, seed=2026, forcing=forcing)
    del S0
    err = rel(got, ref)
    report("forced_split_step_hit_N512_fp32", err, 2e-5)
    assert err < 2e-5
