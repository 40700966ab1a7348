"""torch.autograd.Function around the CUDA adjoint of the forced FCLB update.

Forward: T steps of the D3Q27 FCLB update from a given state under a body
force F (lbm_adjoint_forward, checkpointing every `every` steps, 0 = the
library's choice); returns the final distributions f_T.  Backward: dL/dF
from dL/df_T by the hand-written adjoint stream-collide kernel
(lbm_adjoint_backward).  A context records one forward at a time: the node
keeps the generation of its forward and its backward refuses to run once
the context has recorded another (or its force was reset), instead of
returning the gradient of a different forward.  The distributions and
gradients move through the C ABI as float64 host arrays; all stepping,
recomputation and adjoint sweeps run in the CUDA library.
"""
import numpy as np
import torch

from . import lbm


class ForcedFclb(torch.autograd.Function):
    @staticmethod
    def forward(fctx, F, ctx, f0, T, every):
        lbm.lbm_set_state(ctx, 0, np.asarray(f0, dtype=np.float64))
        lbm.lbm_set_force(ctx, F.detach().cpu().double().numpy())
        lbm.lbm_adjoint_forward(ctx, T, every)
        fT = lbm.lbm_get_state(ctx, 0)
        fctx.lbm_ctx = ctx
        fctx.generation = lbm.lbm_adjoint_generation(ctx)[0]
        return torch.from_numpy(fT).to(device=F.device, dtype=F.dtype)

    @staticmethod
    def backward(fctx, grad_fT):
        if lbm.lbm_adjoint_generation(fctx.lbm_ctx)[0] != fctx.generation:
            raise RuntimeError("the lbm context has recorded another adjoint forward (or its force "
                               "changed) since this node's forward; run each forward's backward "
                               "before the next forward on the same context")
        g = lbm.lbm_adjoint_backward(fctx.lbm_ctx, grad_fT.detach().cpu().double().numpy())
        return torch.from_numpy(g).to(device=grad_fT.device, dtype=grad_fT.dtype), None, None, None, None


def forced_fclb(F, ctx, f0, T, every):
    """f_T of T forced FCLB steps from f0, differentiable w.r.t. F."""
    return ForcedFclb.apply(F, ctx, f0, T, every)
