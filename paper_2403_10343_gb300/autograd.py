"""torch.autograd wrapper: E_x(D, C, V) with gradients from rix_backward."""
import torch

from .rix import Exchange


class ExchangeEnergy(torch.autograd.Function):
    """E_x = -1/4 Tr(D K(D; C, V)) through librix.

    forward(D, C, V, ex): ex is an ``Exchange`` set up with ``backward=1``;
    C and V are loaded into it (rix_set_CV) on every call.  backward returns
    dE/dD, dE/dC, dE/dV per stored packed entry (symmetrised partials).
    """

    @staticmethod
    def forward(ctx, D, C, V, ex):
        ex.set_CV(C.contiguous(), V.contiguous())
        K = ex.build_K(D.contiguous())
        E = ex.energy(D, K)
        ctx.ex = ex
        ctx.save_for_backward(D)
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE):
        (D,) = ctx.saved_tensors
        want = tuple(n for n, need in zip(("D", "C", "V"), ctx.needs_input_grad[:3]) if need)
        if not want:
            return None, None, None, None
        dD, dC, dV = ctx.ex.backward(D.contiguous(), float(gE.item()), want=want)
        return dD, dC, dV, None


def exchange_energy(D, C, V, ex):
    """Differentiable E_x of packed D, C, V (device FP64 tensors)."""
    return ExchangeEnergy.apply(D, C, V, ex)
