"""torch.autograd.Function over (lambda, A) backed by stmf_fg.

Forward runs Alg. 2 (the fused pass over V plus the model terms) through the C ABI and keeps
the gradient it produces (eqs. gradl and gradb); backward scales that stored gradient by the
incoming scalar gradient (the chain rule for a scalar objective), so no second pass over V is
made. The samples V, the weights nu and alpha are constants of the objective.
"""

import torch

from . import stmf


def _colmajor(A):
    """(n, r) float64 CUDA tensor laid out column-major, as the C ABI expects."""
    n, r = A.shape
    if (A.stride(0) == 1 or n == 1) and (A.stride(1) == n or r == 1):
        return A
    return A.t().contiguous().t()


class STMFObjective(torch.autograd.Function):
    """f(lambda, A) = ||X - M||^2 (eq. optFunc) with X given implicitly by (nu, V)."""

    @staticmethod
    def forward(ctx, lam, A, V, nu, d, alpha):
        lam_c = lam.detach().contiguous()
        A_c = _colmajor(A.detach())
        f, g_lam, G_A = stmf.fg(V, nu, d, lam_c, A_c, alpha=alpha)
        ctx.save_for_backward(g_lam, G_A)
        return f.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        g_lam, G_A = ctx.saved_tensors
        return grad_out * g_lam, grad_out * G_A, None, None, None, None


def objective(lam, A, V, nu=None, d=3, alpha=None):
    """Differentiable f(lambda, A); lam (r,) and A (n, r) are float64 CUDA tensors."""
    return STMFObjective.apply(lam, A, V, nu, d, alpha)
