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


@pytest.mark.parametrize("forced", [False, True])
def test_vjp_state_matches_oracle_fp64(ns, report, forced):
    # a loss of u(T) given by its gradient gT (a random linear functional)
    N, nu, dt, nsteps = 16, 0.01, 0.01, 7
    u0 = inputs.hit_initial(N, 11)
    gT = np.random.default_rng(3).standard_normal(u0.shape)
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP64, seed=5) as s:
        if forced:
            s.set_forcing(2.0, 3.0, 1.0, 0.02, seed=7)
        g = s.vjp_state(u0, nsteps, dt, gT, ckpt_every=3)
    f = fo.Forcing(N, 2.0, 3.0, 1.0, 0.02, seed=7) if forced else None
    gr = ad.grad_final_state(u0, gT, nsteps, dt, sc.Problem(N, nu, N / 2), seed=5, forcing=f,
                             ckpt_every=3)
    report("adjoint_state_cotangent_%s_N16_7_steps_fp64" % ("forced" if forced else "decaying"),
           rel(g, gr), 1e-10)
    assert rel(g, gr) < 1e-10


def test_vjp_state_central_differences_on_gpu(ns):
    # L(u0) = sum gT . u(T) through ns_step / ns_get_velocity, FP64, h = 1e-4
    N, nu, dt, nsteps = 16, 0.01, 0.01, 5
    u0 = inputs.hit_initial(N, 12)
    rs = np.random.default_rng(6)
    gT = rs.standard_normal(u0.shape)
    h = 1e-4
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP64, seed=2) as s:
        g = s.vjp_state(u0, nsteps, dt, gT, ckpt_every=2)

        def L(u):
            s.set_time(0.0, 0)
            s.set_velocity(u)
            s.step(dt, nsteps)
            return float(np.sum(gT * s.get_velocity()))

        for _ in range(3):
            v = rs.standard_normal(u0.shape)
            fd = (L(u0 + h * v) - L(u0 - h * v)) / (2 * h)
            assert abs(fd - float(np.sum(g * v))) < 1e-6 * abs(fd)


@pytest.mark.parametrize("prec", [1, 0])
def test_trajectory_autograd_with_a_torch_loss(ns, report, prec):
    # u(T) as a CUDA tensor, any torch loss on it, backward through the library's adjoint
    import torch

    from paper_2603_08892_gb300.autograd import Trajectory

    N, nu, dt, nsteps = 16, 0.01, 0.01, 6
    u0n = inputs.hit_initial(N, 13)
    w = np.random.default_rng(8).standard_normal(u0n.shape)
    dtype = torch.float64 if prec == 1 else torch.float32
    with ns.Solver(N, nu, N / 2, scheme=4, precision=prec, seed=4) as s:
        u0 = torch.tensor(u0n, dtype=dtype, device="cuda", requires_grad=True)
        uT = Trajectory.apply(u0, s, nsteps, dt, 2)
        assert uT.is_cuda and uT.dtype == dtype
        loss = (torch.tensor(w, dtype=dtype, device="cuda") * uT).sum() + 0.5 * (uT * uT).mean()
        loss.backward()
        got = u0.grad.double().cpu().numpy()
        # the same loss's gradient at T, through the host entry point
        s.set_time(0.0, 0)
        s.set_velocity(u0n)
        s.step(dt, nsteps)
        uTh = s.get_velocity()
        gT = w + uTh / uTh.size
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP64, seed=4) as s64:
        ref = s64.vjp_state(u0n, nsteps, dt, gT, ckpt_every=2)
    err = rel(got, ref)
    report("autograd_trajectory_torch_loss_N16_%s" % ("fp64" if prec else "fp32"), err,
           1e-10 if prec else 2e-5)
    assert err < (1e-10 if prec else 2e-5)


def test_final_loss_backward_only_when_asked(ns):
    import torch

    from paper_2603_08892_gb300.autograd import FinalLoss

    N, nu, dt, nsteps = 16, 0.01, 0.01, 4
    u0n = inputs.hit_initial(N, 9)
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP32, seed=1) as s:
        scratch = torch.empty((3, N, N, N), dtype=torch.float32, device="cuda")
        with pytest.raises(ns.NSError) as e:  # no tape yet
            s.tape_backward(None, scratch.data_ptr())
        assert e.value.code == 8
        u0 = torch.tensor(u0n, dtype=torch.float32, device="cuda", requires_grad=True)
        L = FinalLoss.apply(u0, s, nsteps, dt, 2)
        s.step(dt, 3)  # other work on the context between forward and backward
        (2.0 * L).backward()
        g = u0.grad.double().cpu().numpy()
    with ns.Solver(N, nu, N / 2, scheme=4, precision=ns.FP64, seed=1) as s64:
        L64, g64 = s64.vjp(u0n, nsteps, dt, 2)
    assert abs(L.item() - L64) < 1e-5 * L64
    assert rel(g, 2.0 * g64) < 2e-5
