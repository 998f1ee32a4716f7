"""The dipole increment of a run as a differentiable function of the pulse
samples, for torch.autograd.

    dmu = DipoleIncrement.apply(a_samples, context, ckpt_every)

a_samples: (n_steps, 3) float64 tensor, the midpoint samples A_k of the steps
(as for `Context.step`); the result is the 3-vector dmu(t0 + n dt) - dmu(t0)
from the context's current state, which the call leaves unchanged.  Both
directions go through `rttddft_adjoint`: the forward pass takes its dipole
increment, the backward pass the vector-Jacobian product with the incoming
gradient as the direction (reverse mode through the computed Chebyshev
polynomial, checkpoints every `ckpt_every` steps).  Argument marshalling
only; the arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch


class DipoleIncrement(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a_samples, context, ckpt_every=50):
        a = a_samples.detach().to("cpu", torch.float64).numpy()
        _, dmu = context.adjoint(a, np.zeros(3), ckpt_every=ckpt_every)
        fctx.context = context
        fctx.ckpt_every = ckpt_every
        fctx.save_for_backward(a_samples.detach())
        return torch.as_tensor(dmu, dtype=torch.float64, device=a_samples.device)

    @staticmethod
    def backward(fctx, grad_out):
        (a_samples,) = fctx.saved_tensors
        a = a_samples.to("cpu", torch.float64).numpy()
        g = grad_out.detach().to("cpu", torch.float64).numpy()
        grad, _ = fctx.context.adjoint(a, g, ckpt_every=fctx.ckpt_every)
        return torch.as_tensor(grad, dtype=a_samples.dtype, device=a_samples.device), None, None
