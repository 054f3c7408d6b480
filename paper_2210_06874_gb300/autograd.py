"""The pseudofermion action as a torch.autograd.Function with a hand-written
adjoint (§2, Eq. (2.1)).

forward(phi):  x = (M M^dag)^{-1} chi by hmc_cg_solve (FP64 or mixed), then
               S = sum(phi^2)/(2 delta U) + chi^dag x by hmc_action; x is kept.
backward(g):   g * dS/dphi, with dS/dphi = phi/(delta U) + 2 Im(x conj(M^dag x))
               from hmc_force on the kept x -- the solve is not repeated.

Every step runs in libhmc_gb300.so; this module only wires the calls into
torch's autograd graph.
"""
import torch

from . import hmc


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, chi, context, prec, tol):
        x, stats = context.cg_solve(phi.detach(), chi, tol=tol, prec=prec)
        S = context.action(phi.detach(), chi, x)
        ctx.save_for_backward(phi.detach(), x)
        ctx.context = context
        ctx.stats = stats
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, grad_out):
        phi, x = ctx.saved_tensors
        F = ctx.context.force(phi, x)
        return grad_out * F, None, None, None, None


def pseudofermion_action(phi, chi, context, prec=hmc.PREC_FP64, tol=None):
    """S(phi) for a fixed pseudofermion chi; differentiable in phi."""
    tol = context.params.cg_tol if tol is None else tol
    return PseudofermionAction.apply(phi, chi, context, prec, tol)
