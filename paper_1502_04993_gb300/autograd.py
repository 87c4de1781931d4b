"""torch.autograd binding of the GLM log-likelihood.

`glm_loglik(g, W, b, tau)` returns L = sum_i L_i (Eq. 1) as a 0-d float64 tensor and makes W, b and tau
differentiable.  All arithmetic runs in libglm's kernels: when any input needs a gradient the forward
pass calls glm_loglik_grad with the gradient outputs (dL/dW and dL/db from the gradient product, dL/dtau
from the tau partials of the U-product epilogue and the spike part), and backward only scales them by the
incoming gradient.  tau enters through a = exp(-dt/tau) of the kernel (Eq. 3); a new tau re-runs the
per-problem caches (filter scan and spike term) before the evaluation.
"""
from __future__ import annotations

import torch


class GLMLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, W, b, tau):
        tau_v = float(tau)
        if abs(tau_v - g.tau) > 0.0:
            g.prepare(tau_v)
        need = ctx.needs_input_grad
        want_w, want_b, want_tau = bool(need[1]), bool(need[2]), bool(need[3])
        r = g.loglik_grad(W.detach(), b.detach(), grad=want_w or want_b, total=True,
                          tau_grad=want_tau and g.prec != "f32")
        if want_tau and g.prec == "f32":
            raise RuntimeError("dL/dtau needs a tensor-core precision (bf16 or f16)")
        ctx.save_for_backward(r["G"] if r["G"] is not None else torch.empty(0),
                              r["gb"] if r["gb"] is not None else torch.empty(0))
        ctx.gtau = r["gtau"]
        ctx.dtypes = (W.dtype, b.dtype, tau.dtype if torch.is_tensor(tau) else torch.float64)
        ctx.tau_device = tau.device if torch.is_tensor(tau) else torch.device("cpu")
        return torch.tensor(r["L_total"], dtype=torch.float64, device=W.device)

    @staticmethod
    def backward(ctx, grad_out):
        G, gb = ctx.saved_tensors
        gW = gB = gT = None
        if ctx.needs_input_grad[1]:
            gW = (grad_out * G).to(ctx.dtypes[0])
        if ctx.needs_input_grad[2]:
            gB = (grad_out * gb).to(ctx.dtypes[1])
        if ctx.needs_input_grad[3]:
            gT = (grad_out.to(ctx.tau_device) * ctx.gtau).to(ctx.dtypes[2])
        return None, gW, gB, gT


def glm_loglik(g, W: torch.Tensor, b: torch.Tensor, tau) -> torch.Tensor:
    """Differentiable log-likelihood of the problem held by context `g` (a paper_1502_04993_gb300.GLM)."""
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    return GLMLogLik.apply(g, W, b, tau)
