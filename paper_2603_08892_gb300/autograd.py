"""torch.autograd.Functions over the library's hand-written adjoint (ns_tape_forward /
ns_tape_backward): the forward steps and the reverse sweep both run in the library's CUDA
kernels on device buffers of the solver's precision; torch only holds the tensors.

    u0 = torch.randn(3, N, N, N, device="cuda", dtype=torch.float32, requires_grad=True)
    uT = Trajectory.apply(u0, solver, nsteps, dt, ckpt_every)   # u(T), a CUDA tensor
    loss = my_loss(uT)                                          # any torch loss of u(T)
    loss.backward()                                             # u0.grad = dL/du0

    L = FinalLoss.apply(u0, solver, nsteps, dt, ckpt_every)      # built-in eps(T) (or E(T))

The forward keeps the state every ckpt_every steps on the device; backward recomputes each
segment from its checkpoint (only when backward is called).  Gradients are for the physical
dot product over the grid points.
"""
import torch

from . import binding


def _dtype(solver):
    return torch.float32 if solver.precision == binding.FP32 else torch.float64


def _on_device(x, solver):
    """x as a contiguous CUDA tensor of the solver's precision (no copy when it already is)."""
    return x.detach().to(device="cuda", dtype=_dtype(solver)).contiguous()


class Trajectory(torch.autograd.Function):
    """u(T) after nsteps RK2 phase-shift random / split steps from u0 (physical [3, N, N, N])."""

    @staticmethod
    def forward(ctx, u0, solver, nsteps, dt, ckpt_every=10):
        u = _on_device(u0, solver)
        uT = torch.empty_like(u)
        torch.cuda.current_stream().synchronize()  # u0's producers are done
        solver.tape_forward(u.data_ptr(), nsteps, dt, ckpt_every, uT.data_ptr())
        ctx.solver = solver
        ctx.src = (u0.device, u0.dtype)
        return uT

    @staticmethod
    def backward(ctx, grad_out):
        g = _on_device(grad_out, ctx.solver)
        grad = torch.empty_like(g)
        torch.cuda.current_stream().synchronize()
        ctx.solver.tape_backward(g.data_ptr(), grad.data_ptr())
        dev, dt = ctx.src
        return grad.to(device=dev, dtype=dt), None, None, None, None


class FinalLoss(torch.autograd.Function):
    """A built-in loss of the final state (binding.LOSS_DISSIPATION: eps(T), or LOSS_ENERGY:
    E(T)) after nsteps steps from u0; the reverse sweep runs only in backward."""

    @staticmethod
    def forward(ctx, u0, solver, nsteps, dt, ckpt_every=10, loss=binding.LOSS_DISSIPATION):
        u = _on_device(u0, solver)
        uT = torch.empty_like(u)
        torch.cuda.current_stream().synchronize()
        solver.tape_forward(u.data_ptr(), nsteps, dt, ckpt_every, uT.data_ptr())
        E, eps = solver.energy()
        ctx.solver, ctx.loss, ctx.src = solver, loss, (u0.device, u0.dtype, u.shape)
        return torch.tensor(eps if loss == binding.LOSS_DISSIPATION else E, dtype=u0.dtype,
                            device=u0.device)

    @staticmethod
    def backward(ctx, grad_out):
        dev, dt, shape = ctx.src
        grad = torch.empty(shape, device="cuda", dtype=_dtype(ctx.solver))
        ctx.solver.tape_backward(None, grad.data_ptr(), ctx.loss)
        return (grad_out.to(device="cuda", dtype=grad.dtype) * grad).to(device=dev, dtype=dt), \
            None, None, None, None, None
