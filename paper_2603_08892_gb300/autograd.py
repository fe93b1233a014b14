"""torch.autograd.Function over the library's hand-written adjoint (ns_vjp).

    u0 = torch.tensor(..., requires_grad=True)              # physical [3, N, N, N]
    L = FinalLoss.apply(u0, solver, nsteps, dt, ckpt_every)  # eps(T) by default
    L.backward()                                             # u0.grad = dL/du0

The forward and the reverse sweep both run in the library's CUDA kernels (one ns_vjp call
computes L and the gradient; backward scales the stored gradient by the incoming one).
"""
import torch

from . import binding


class FinalLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, nsteps, dt, ckpt_every=10, loss=binding.LOSS_DISSIPATION):
        L, g = solver.vjp(u0.detach().to("cpu", torch.float64).numpy(), nsteps, dt, ckpt_every, loss)
        ctx.save_for_backward(torch.from_numpy(g).to(device=u0.device, dtype=u0.dtype))
        return u0.new_tensor(L)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None
