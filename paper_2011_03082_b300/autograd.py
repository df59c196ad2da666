"""The CVAE loss as a ``torch.autograd.Function`` whose forward and backward run in the library's kernels.

Sec. 3.2 trains each CVAE by minimising the negative ELBO with a gradient optimiser in PyTorch.  Here the
loss and its gradient with respect to the packed parameter vector (encoder block then decoder block, as
``ms_cvae_num_params`` counts them) come from the hand-written kernels, so the parameters can be trained with
any ``torch.optim`` optimiser or composed with other autograd code:

    loss, rec, kl = cvae_loss(params, x, c, shape, eps_z=eps)      # ms_cvae_forward[_backward]
    loss.backward()                                                # params.grad from the same kernels

When ``params`` requires a gradient, the forward pass calls ``ms_cvae_forward_backward``, which forms the loss
and the gradient in one pass over the batch, and keeps the gradient for the backward pass; otherwise it calls
``ms_cvae_forward`` (the loss alone).  The backward pass hands that gradient on, scaled by the incoming
gradient of the loss.  ``rec`` and ``kl`` (the reconstruction and KL terms) are reported but not
differentiable, and no gradient flows to ``x``, ``c`` or ``eps_z`` (the kernels compute none).
"""
from __future__ import annotations

import torch

from . import ms


class CvaeNegElbo(torch.autograd.Function):
    """Negative ELBO of one batch (mean over the batch) and its parameter gradient, from libms."""

    @staticmethod
    def forward(ctx, params, x, c, shape, eps_z, seed, step):
        B = x.shape[0]
        loss3 = torch.empty(3, dtype=torch.float32, device=params.device)
        ws = ms.workspace(ms.ms_cvae_workspace_size(shape, B), params.device)
        p, xx, cc = params.detach().contiguous(), x.detach().contiguous(), c.detach().contiguous()
        e = None if eps_z is None else eps_z.detach().contiguous()
        if ctx.needs_input_grad[0]:
            grad = torch.empty_like(p)
            ms.ms_cvae_forward_backward(shape, p, xx, cc, B, eps_z=e, seed=seed, step=step, grad=grad, loss3=loss3,
                                        ws=ws)
            ctx.save_for_backward(grad)
        else:
            ms.ms_cvae_forward(shape, p, xx, cc, B, eps_z=e, seed=seed, step=step, loss3=loss3, ws=ws)
        loss, rec, kl = loss3[0].clone(), loss3[1].clone(), loss3[2].clone()
        ctx.mark_non_differentiable(rec, kl)
        return loss, rec, kl

    @staticmethod
    def backward(ctx, g_loss, g_rec, g_kl):
        if not ctx.needs_input_grad[0]:
            return (None,) * 7
        (grad,) = ctx.saved_tensors
        return grad * g_loss, None, None, None, None, None, None


def cvae_loss(params: torch.Tensor, x: torch.Tensor, c: torch.Tensor, shape: ms.CvaeShape, *, eps_z=None,
              seed: int = 1, step: int = 0):
    """(loss, rec, kl) of the batch (x [B][p_out], c [B][p_in], float32 CUDA tensors); eps_z [B][latent] standard
    normals or None to draw them in the kernel from (seed, step).  ``loss`` is differentiable in ``params``."""
    return CvaeNegElbo.apply(params, x, c, shape, eps_z, seed, step)
