"""torch.autograd.Function around the hand-written adjoint of the split step.

``fidelity(g, c, solver, psi0, target, nsteps, every)`` returns the fidelity
F = |<target|psi(T)>|^2 after ``nsteps`` real-time steps from ``psi0`` with
contact strength ``g`` and trap-modulation coefficients ``c``
(V(t) = V0 (1 + sum_m c_m sin(m t))) as a differentiable torch scalar: the
forward call runs the solver's forward sweep with checkpoints every ``every``
steps and its reverse sweep (libdgpe.so, dgpe_fidelity_gradient), and the
backward pass returns the gradients it produced.  Marshalling only: all
arithmetic runs in the CUDA kernels.
"""
import torch

from . import dgpe


class _Fidelity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, c, solver, psi0, target, nsteps, every):
        solver.set_g(float(g))
        cm = [float(v) for v in c.detach().cpu().reshape(-1)]
        solver.set_trap_modulation(cm)
        F, dg, dc = dgpe.dgpe_fidelity_gradient(solver.h, psi0, target, nsteps, every, len(cm))
        ctx.save_for_backward(torch.tensor(dg, dtype=torch.float64),
                              torch.tensor(dc, dtype=torch.float64).reshape(c.shape))
        return torch.tensor(F, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad):
        dg, dc = ctx.saved_tensors
        return grad * dg, grad * dc, None, None, None, None, None


def fidelity(g, c, solver, psi0, target, nsteps, every=32):
    """Differentiable fidelity (see module docstring); g a 0-d tensor, c 1-d."""
    return _Fidelity.apply(g, c, solver, psi0, target, nsteps, every)
