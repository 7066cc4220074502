"""torch.autograd.Function over the fused likelihood kernels.

The forward is the same fused log L + score evaluation the HSS walkers run
(``ns_lik_forward``); the backward is the hand-written adjoint
(``ns_lik_backward``), which returns gout_i * d log L_i / d x_i and
sum_i gout_i * d log L_i / d mu_k.  The component means are the likelihood
parameters theta whose log Z gradient the method's problem statement asks for
(Section 2.1; the posterior-weighted form over a finished run is
``Sampler.grad_logz``).  PyTorch supplies the tensors and the stream only:
every value comes from the CUDA kernels, and there is no other path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ggns

__all__ = ["LogLikelihood", "log_likelihood"]


class LogLikelihood(torch.autograd.Function):
    """log L(x_i; mu) for points x[n][d] (FP32, CUDA) and means mu[n_comp][d].

    ``sampler`` holds the likelihood (run 0 of its context); when ``means``
    differs from the means it holds they are replaced first (ns_set_means).
    """

    @staticmethod
    def forward(ctx, x: torch.Tensor, means: torch.Tensor, sampler: "ggns.Sampler"):
        if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
            raise ValueError("x must be a CUDA float32 tensor [n][d]")
        x = x.contiguous()
        m64 = means.detach().to(device="cpu", dtype=torch.float64).contiguous().numpy()
        cached = getattr(sampler, "_means_cache", None)
        if cached is None or cached.shape != m64.shape or not np.array_equal(cached, m64):
            sampler.set_means(m64, 0)
            sampler._means_cache = m64.copy()
        n = x.shape[0]
        logl = torch.empty(n, dtype=torch.float32, device=x.device)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        sampler.lik_forward(x.data_ptr(), n, logl.data_ptr(), None, stream)
        ctx.save_for_backward(x)
        ctx.sampler = sampler
        ctx.means_shape = tuple(means.shape)
        ctx.means_device = means.device
        return logl

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        (x,) = ctx.saved_tensors
        n = x.shape[0]
        gout = gout.detach().to(dtype=torch.float32).contiguous()
        gx = torch.empty_like(x) if ctx.needs_input_grad[0] else None
        gmu = None
        if ctx.needs_input_grad[1]:
            gmu = torch.zeros(ctx.means_shape, dtype=torch.float32, device=x.device)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        ctx.sampler.lik_backward(x.data_ptr(), n, gout.data_ptr(), None if gx is None else gx.data_ptr(),
                                 None if gmu is None else gmu.data_ptr(), stream)
        if gmu is not None:
            gmu = gmu.to(ctx.means_device)
        return gx, gmu, None


def log_likelihood(x: torch.Tensor, means: torch.Tensor, sampler: "ggns.Sampler") -> torch.Tensor:
    return LogLikelihood.apply(x, means, sampler)
