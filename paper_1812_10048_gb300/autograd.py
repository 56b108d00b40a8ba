"""Collapsed log marginal likelihood as a torch.autograd.Function.

Forward and backward both run in libdpmm.so: the forward sums lgamma terms
in FP64 on the device, the backward kernel sums digamma terms in FP32 (see
``dpmm_logml_forward`` / ``dpmm_logml_backward`` in include/dpmm.h).  The
statistics of the fixed labels are computed once, when ``LogML`` is built.
"""

import torch

from . import dpmm_logml_backward, dpmm_logml_create, dpmm_logml_forward, dpmm_logml_free


class LogML:
    """Collapsed log marginal likelihood of fixed labels on one CUDA device."""

    def __init__(self, indptr, indices, data, N, D, labels, K, stream=None):
        self.N, self.D, self.K = int(N), int(D), int(K)
        self.h = dpmm_logml_create(indptr, indices, data, N, D, labels, K, stream)

    def close(self):
        if self.h is not None:
            dpmm_logml_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, log_alpha, log_beta):
        return dpmm_logml_forward(self.h, float(log_alpha), log_beta)

    def backward(self, log_alpha, log_beta, grad_log_beta):
        return dpmm_logml_backward(self.h, float(log_alpha), log_beta, grad_log_beta)

    def __call__(self, log_alpha, log_beta):
        return LogMLFunction.apply(log_alpha, log_beta, self)


class LogMLFunction(torch.autograd.Function):
    """LML(log_alpha, log_beta): scalar FP64 output; grads from the backward kernel."""

    @staticmethod
    def forward(ctx, log_alpha, log_beta, model):
        lb = log_beta.detach().to(torch.float32).contiguous()
        la = float(log_alpha.detach())
        ctx.model, ctx.la = model, la
        ctx.save_for_backward(lb)
        val = model.forward(la, lb)
        return torch.tensor(val, dtype=torch.float64, device=log_beta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (lb,) = ctx.saved_tensors
        g_beta = torch.empty_like(lb)
        g_alpha = ctx.model.backward(ctx.la, lb, g_beta)
        go = grad_out.to(torch.float64)
        ga = (go * g_alpha).reshape(()).to(torch.float64)
        gb = (go.to(torch.float32) * g_beta)
        return ga, gb, None
