"""torch.autograd.Function over the CUDA library: forward prices with the
forward-only kernel (lv_price), backward runs the hand-written reverse-sweep
adjoint kernel (lv_price_greeks_device) and returns grad * delta for S0 and
grad * vega for the local-vol grid (Sec. III, IV-C of arXiv 2002.02481:
back-propagation through the Euler scheme). All arithmetic runs in the
library; this module only moves tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lv


class LVPrice(torch.autograd.Function):
    """price = LVPrice.apply(S0, sigma, surface, r, K, T, n_steps, n_paths, seed)

    S0: 0-d tensor; sigma: [n_spot, n_time] tensor (any device, float64 or
    float32); surface: an lv.Surface whose node vectors define the grid (its
    sigma values are replaced by `sigma`). Returns a 0-d float64 tensor on
    sigma's device.

    The forward call records the surface's settings (this sigma, the option
    type, the accumulation, the adjoint method and the readings); backward
    passes them back to the handle before running the adjoint, so several
    terms priced on one Surface with different sigma or settings each get
    their own derivatives, whatever the surface holds when backward runs."""

    @staticmethod
    def forward(ctx, S0, sigma, surface, r, K, T, n_steps, n_paths, seed):
        s0 = float(S0.detach().cpu())
        sig = sigma.detach().to("cpu", torch.float64).numpy()
        surface.set_sigma(np.ascontiguousarray(sig))
        price, _ = surface.price(s0, r, K, T, n_steps, n_paths, seed)
        ctx.surface = surface
        ctx.state = surface.state()
        ctx.args = (s0, r, K, T, n_steps, n_paths, seed)
        ctx.shape = sigma.shape
        ctx.sigma_dtype, ctx.s0_dtype = sigma.dtype, S0.dtype
        ctx.device = sigma.device
        return torch.tensor(price, dtype=torch.float64, device=sigma.device)

    @staticmethod
    def backward(ctx, grad_out):
        s0, r, K, T, n_steps, n_paths, seed = ctx.args
        surface = ctx.surface
        n = 3 + surface.n_spot * surface.n_time
        dev = torch.device("cuda", torch.cuda.current_device())
        out = torch.empty(n, dtype=torch.float64, device=dev)
        surface.set_stream(torch.cuda.current_stream(dev).cuda_stream)
        surface.restore(ctx.state)               # the settings this term was priced with
        surface.price_greeks_device(s0, r, K, T, n_steps, n_paths, seed, out.data_ptr())
        g = grad_out.to(dev, torch.float64)
        d_s0 = (g * out[lv.LV_OUT_DELTA]).to(ctx.device, ctx.s0_dtype)
        d_sig = (g * out[lv.LV_OUT_VEGA:]).reshape(ctx.shape).to(ctx.device, ctx.sigma_dtype)
        return d_s0, d_sig, None, None, None, None, None, None, None


def lv_price(S0, sigma, surface, r, K, T, n_steps, n_paths, seed=1):
    """Differentiable Monte Carlo price (see LVPrice)."""
    return LVPrice.apply(S0, sigma, surface, r, K, T, n_steps, n_paths, seed)
