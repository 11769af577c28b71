"""torch.autograd wrapper: E_x(D, C, V) with gradients from rix_backward."""
import torch

from .rix import Exchange


def _stamp(t):
    """Identity of a tensor's current contents: storage, layout and in-place version counter."""
    return (t.data_ptr(), tuple(t.shape), t.dtype, t.device, t._version)


class ExchangeEnergy(torch.autograd.Function):
    """E_x = -1/4 Tr(D K(D; C, V)) through librix.

    forward(D, C, V, ex): ex is an ``Exchange`` set up with ``backward=1``.  C
    and V are loaded into it (rix_set_CV: a copy, the symmetry check and, in
    mixed precision, the slicing) only when they differ from the tensors of the
    previous call (another tensor, or the same one modified in place since); an
    SCF loop that changes only D pays for the build alone.  backward returns
    dE/dD, dE/dC, dE/dV per stored packed entry (symmetrised partials).
    """

    @staticmethod
    def forward(ctx, D, C, V, ex):
        C, V = C.contiguous(), V.contiguous()
        stamp = (_stamp(C), _stamp(V))
        if getattr(ex, "_cv_stamp", None) != stamp:
            ex.set_CV(C, V)
            ex._cv_stamp = stamp
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
