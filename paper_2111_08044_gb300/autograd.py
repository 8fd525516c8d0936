"""torch.autograd face of the device adjoint.

``final_energy(theta_p, hx_p, cfg)`` is the energy density <psi_P|H0|psi_P>/L
after P = len(theta_p) Floquet periods of the chain ``cfg`` (an
``inputs.ChainConfig``), as a differentiable function of the per-period kick
angles and drive fields.  The forward runs ``sv_adjoint``: P periods forward
on the device, then the reverse sweep that yields both gradients, which the
backward scales by the incoming gradient.  No states are stored between the
two: the reverse sweep recomputes them by un-applying each gate.
"""
from __future__ import annotations

import numpy as np
import torch

from .sim import FloquetSimulator, chain_params


class FinalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta_p, hx_p, cfg, precision):
        th = theta_p.detach().to("cpu", torch.float64).numpy()
        hx = hx_p.detach().to("cpu", torch.float64).numpy()
        if th.shape != hx.shape or th.ndim != 1 or th.size == 0:
            raise ValueError("theta_p and hx_p must be 1-D of the same nonzero length")
        with FloquetSimulator(cfg.L, precision=precision) as sim:
            sim.init_product_state(cfg.spinors())
            sim.build(**chain_params(cfg, theta_p=th, hx_p=hx))
            gt, gh, e = sim.adjoint()
        ctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(gt)),
                              torch.from_numpy(np.ascontiguousarray(gh)))
        return torch.tensor(e, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        gt, gh = ctx.saved_tensors
        g = grad_out.to(torch.float64).cpu()
        return g * gt, g * gh, None, None


def final_energy(theta_p: torch.Tensor, hx_p: torch.Tensor, cfg, precision: str = "c64"):
    return FinalEnergy.apply(theta_p, hx_p, cfg, precision)
