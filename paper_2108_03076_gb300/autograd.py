"""Differentiable Monte Carlo price: a torch.autograd.Function over pc_greeks.

``mc_price(ctx, contract, S0, sigma, corr, r, days, n_paths, seed)`` returns
the price as a 0-d float64 tensor.  Its gradient with respect to the tensors
``S0`` and ``sigma`` is the engine's pathwise delta and vega (tangent mode
on the same paths, decisions held fixed), so ``price.backward()`` or
``torch.autograd.grad`` work as for any differentiable torch expression.
The forward pass builds a model from the current S0 / sigma values, runs
pc_greeks (one launch per underlying) and keeps the sensitivities for the
backward pass; nothing is computed outside the library's kernels.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np
import torch

from . import pc_greeks, pc_model_create, pc_model_destroy


class PathwisePrice(torch.autograd.Function):
    @staticmethod
    def forward(ctx, S0: torch.Tensor, sigma: torch.Tensor, engine: int, contract: int,
                corr: Sequence[Sequence[float]], r: float, days: Sequence[int], n_paths: int,
                seed: int) -> torch.Tensor:
        s0 = S0.detach().double().cpu().numpy()
        sg = sigma.detach().double().cpu().numpy()
        model = pc_model_create(engine, s0, sg, corr, r, days)
        try:
            price, delta, vega, se = pc_greeks(model, contract, n_paths, seed, len(s0))
        finally:
            pc_model_destroy(model)
        ctx.save_for_backward(torch.from_numpy(np.asarray(delta)).to(S0.dtype),
                              torch.from_numpy(np.asarray(vega)).to(sigma.dtype))
        ctx.stderr = se
        return torch.tensor(price, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        delta, vega = ctx.saved_tensors
        g = grad.to(delta.dtype)
        return g * delta, g * vega, None, None, None, None, None, None, None


def mc_price(engine: int, contract: int, S0: torch.Tensor, sigma: torch.Tensor,
             corr: Sequence[Sequence[float]], r: float, days: Sequence[int], n_paths: int,
             seed: int) -> torch.Tensor:
    """Monte Carlo price, differentiable in S0 and sigma (pathwise)."""
    return PathwisePrice.apply(S0, sigma, engine, contract, corr, r, days, n_paths, seed)
