"""torch.autograd.Function over the library's split evaluation.

``dd4dvar_J(w, ctx)`` returns the vector of local functionals J_s(w_s) of
every subdomain (Sec. 3.3, Eq. eq:cost:parallel1); its backward returns
sum_s gJ_s dJ_s/dw_s through the hand-written adjoint sweep (Alg. 6 ADJ).
The forward keeps what the adjoint needs on the device: the stored
trajectory, or with ``ckpt_k > 0`` in ``set_decomposition`` only every k-th
level, the adjoint then recomputing each k-step segment.

Both calls go through the C ABI (dd4dv_eval_forward / dd4dv_eval_backward);
this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import Context, DD4DVError


class DD4DVarJ(torch.autograd.Function):
    @staticmethod
    def forward(actx, w: torch.Tensor, dd: Context):
        if not (w.is_cuda and w.dtype == torch.float64 and w.is_contiguous()):
            raise TypeError("w must be a contiguous float64 CUDA tensor (packed controls)")
        if w.numel() != dd.ctrl_total:
            raise ValueError(f"w has {w.numel()} values, the layout needs {dd.ctrl_total}")
        J = dd.eval_forward(w)          # stream-ordered with torch (see Context)
        actx.dd = dd
        actx.save_for_backward(w)
        actx.token = dd.forward_token()
        return J

    @staticmethod
    def backward(actx, gJ: torch.Tensor):
        dd: Context = actx.dd
        (w,) = actx.saved_tensors
        if dd.forward_token() != actx.token:
            # another evaluation ran in between: redo this forward first
            dd.eval_forward(w)
        g = dd.eval_backward(scale=gJ.contiguous().to(torch.float64), like=w)
        return g, None


def dd4dvar_J(w: torch.Tensor, dd: Context) -> torch.Tensor:
    """Local functionals J_s(w_s) of all subdomains, differentiable in w."""
    return DD4DVarJ.apply(w, dd)
