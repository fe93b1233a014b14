"""GPU adjoint (ns_vjp) against the FP64 oracle adjoint and finite differences."""
import numpy as np
import pytest

from oracle import adjoint as ad
from oracle import forcing as fo
from oracle import schemes as sc
from paper_2603_08892_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("scheme", [4, 3])
def test_fp64_gradient_matches_oracle(ns, report, forced, scheme):
    N, nu, dt, nsteps = 16, 0.01, 0.01, 7
    kmax = N / 2
    u0 = inputs.hit_initial(N, 7)
    with ns.Solver(N, nu, kmax, scheme=scheme, precision=ns.FP64, seed=5) as s:
        if forced:
            s.set_forcing(2.0, 3.0, 1.0, 0.02, seed=7)
        L, g = s.vjp(u0, nsteps, dt, ckpt_every=3)
    prob = sc.Problem(N, nu, kmax)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.02, seed=7) if forced else None
    Lr, gr = ad.grad_final_dissipation(u0, nsteps, dt, prob, seed=5, forcing=f, ckpt_every=3,
                                       approx=scheme == 3)
    report("adjoint_gradient_%s_N16_7_steps_fp64" % ("forced" if forced else "decaying"), rel(g, gr), 1e-10)
    assert abs(L - Lr) < 1e-12 * Lr
    assert rel(g, gr) < 1e-10


def test_fp64_gradient_central_differences_on_gpu(ns):
    N, nu, dt, nsteps = 16, 0.01, 0.01, 6
    u0 = inputs.hit_initial(N, 8)
    rs = np.random.default_rng(1)
    h = 1e-4
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP64, seed=2) as s:
        s.set_forcing(2.0, 3.0, 1.0, 0.5, seed=3)
        L, g = s.vjp(u0, nsteps, dt, ckpt_every=4)
        for _ in range(3):
            v = rs.standard_normal(u0.shape)
            Lp, _ = s.vjp(u0 + h * v, nsteps, dt, ckpt_every=4)
            Lm, _ = s.vjp(u0 - h * v, nsteps, dt, ckpt_every=4)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - float(np.sum(g * v))) < 1e-6 * abs(fd)


def test_fp32_forced_gradient_against_fp64_oracle(ns, report):
    # reduced config-5 shape: forced HIT at 32^3, 20 steps, checkpoints every 10, FP32
    N, dt, nsteps = 32, 0.005, 20
    kmax = N / 2
    nu = kmax ** (-4.0 / 3.0)
    u0 = inputs.hit_initial(N, 7)
    with ns.Solver(N, nu, kmax, scheme=4, precision=ns.FP32, seed=7) as s:
        s.set_forcing(2.0, 3.0, 1.0, 0.5, seed=7)
        L, g = s.vjp(u0, nsteps, dt, ckpt_every=10)
    prob = sc.Problem(N, nu, kmax)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.5, seed=7)
    Lr, gr = ad.grad_final_dissipation(u0, nsteps, dt, prob, seed=7, forcing=f, ckpt_every=10)
    report("adjoint_loss_forced_N32_20_steps_fp32", abs(L - Lr) / Lr, 1e-4)
    report("adjoint_gradient_forced_N32_20_steps_fp32", rel(g, gr), 2e-5)
    assert abs(L - Lr) < 1e-4 * Lr
    assert rel(g, gr) < 2e-5  # measured 1.6e-6


def test_autograd_function(ns):
    import torch

    from paper_2603_08892_gb300.autograd import FinalLoss

    N = 16
    u0 = torch.from_numpy(inputs.hit_initial(N, 9)).requires_grad_(True)
    with ns.Solver(N, 0.01, N / 2, scheme=4, precision=ns.FP64, seed=1) as s:
        L = FinalLoss.apply(u0, s, 4, 0.01, 2)
        (3.0 * L).backward()
        L2, g = s.vjp(u0.detach().numpy(), 4, 0.01, 2)
    assert abs(L.item() - L2) < 1e-14 * L2
    np.testing.assert_allclose(u0.grad.numpy(), 3.0 * g, rtol=1e-12, atol=1e-18)
