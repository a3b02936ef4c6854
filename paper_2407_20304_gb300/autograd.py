"""torch.autograd.Function around the library's F2 and gradients.

`HoloLoss.apply(psi, q, holo)` returns F2 (Eq. min1) as an FP64 scalar tensor and makes
psi.grad / q.grad the gradients of Eq. gradpsi and the probe gradient after it.  These are
real gradients for <a, b> = Re sum conj(a) b, which is PyTorch's convention for a real
function of complex tensors (for L = |z|^2, z.grad = 2 z), so they are returned as they are,
scaled by the incoming gradient.

Two modes (no intermediate wavefield is ever stored; memory is input-sized):
* recompute=False: forward evaluates F2 and both gradients in one pass and keeps only the
  gradients for backward;
* recompute=True: forward evaluates F2 alone (passes A and B) and backward recomputes the
  planes with the adjoint passes.
All angles of `holo` (its chunk) are evaluated; psi is [chunk][n][n] complex64, q is
[P][P] complex64, both CUDA tensors.
"""

import torch


class HoloLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, q, holo, recompute=False, k0=0):
        psi_d = psi.detach().contiguous()
        q_d = q.detach().contiguous()
        holo.set_probe(q_d)
        if recompute:
            loss = holo.forward(psi_d, k0=k0)
            ctx.save_for_backward(psi_d, q_d)
        else:
            loss, gpsi, gq = holo.gradient(psi_d, k0=k0)
            ctx.save_for_backward(gpsi, gq)
        ctx.holo, ctx.recompute, ctx.k0 = holo, recompute, k0
        return torch.tensor(loss, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.recompute:
            psi_d, q_d = ctx.saved_tensors
            ctx.holo.set_probe(q_d)
            _, gpsi, gq = ctx.holo.gradient(psi_d, k0=ctx.k0, want_loss=False)
        else:
            gpsi, gq = ctx.saved_tensors
        s = grad_out.to(torch.float32)
        return gpsi * s, gq * s, None, None, None


def holo_loss(psi, q, holo, recompute=False, k0=0):
    """F2 of (psi, q) as a differentiable FP64 scalar."""
    return HoloLoss.apply(psi, q, holo, recompute, k0)
