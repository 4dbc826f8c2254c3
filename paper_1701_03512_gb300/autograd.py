"""torch.autograd.Function over the exhaustive value and its derivative pass.

``exact_price(params, template)`` takes a tensor ``params[n, 4]`` holding
(S0, sigma, rate, K) per option and a list of option dicts for everything
else (N, tree, payoff, T); it returns the values as a tensor. The forward
runs ``bt_greeks_exact`` (one CUDA pass gives the value and dV/d(S0, sigma,
rate, K)); the backward multiplies those derivatives by the upstream gradient.
"""
from __future__ import annotations

import torch

from . import btree as bt


class ExactPrice(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, template, ctx_handle, prec):
        p = params.detach().to("cpu", torch.float64).numpy()
        opts = []
        for i, o in enumerate(template):
            o = dict(o)
            o["S0"], o["sigma"], o["rate"], o["K"] = (float(x) for x in p[i])
            opts.append(o)
        val, grad = bt.bt_greeks_exact(ctx_handle, opts, prec)
        g = torch.from_numpy(grad).to(device=params.device, dtype=params.dtype)
        fctx.save_for_backward(g)
        return torch.from_numpy(val).to(device=params.device, dtype=params.dtype)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return grad_out.unsqueeze(-1) * g, None, None, None


def exact_price(params: torch.Tensor, template, ctx_handle, prec=bt.BT_PREC_FP32_COMP) -> torch.Tensor:
    """Values of the options (differentiable in params [n, 4] = S0, sigma, rate, K)."""
    if params.ndim != 2 or params.shape[1] != 4 or params.shape[0] != len(template):
        raise ValueError("params must be [n, 4] = (S0, sigma, rate, K) per option")
    return ExactPrice.apply(params, list(template), ctx_handle, prec)
