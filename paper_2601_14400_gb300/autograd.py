"""torch.autograd bridge for gradients of thermal observables.

``thermal_coefficients(alpha, prop, n_layers, obs_x, obs_z)`` returns the
coefficients c_j of the given Pauli strings in the normalised propagated
operator after ``n_layers`` Trotter layers from the identity, with the gate
coefficients ``alpha`` (one per gate of ``prop``'s Hamiltonian, in Trotter
order).  Its backward runs the library's adjoint sweep (``itpp_adjoint``:
frozen support, snapshots every ``ckpt_every`` layers) with the incoming
gradient as the observable weights.  Everything numeric runs in the CUDA
library; this module only moves arrays between torch and the C ABI.

An expectation value whose weights depend on the parameters, such as the
energy <H> = sum_k alpha_k c_{Q_k}, is then ordinary torch arithmetic on the
returned coefficients, and autograd adds the explicit term itself.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Propagator


class _ObsWeights:
    def __init__(self, x, z, w):
        self.x, self.z, self.w = x, z, w


class ThermalCoefficients(torch.autograd.Function):
    @staticmethod
    def forward(ctx, alpha, prop: Propagator, n_layers: int, obs_x, obs_z, ckpt_every: int):
        a = alpha.detach().to("cpu", torch.float64).numpy()
        prop.set_alpha(a)
        prop.reset()
        prop.apply_trotter_layer(n_layers)
        c = prop.coeffs(obs_x, obs_z)
        ctx.prop, ctx.n_layers, ctx.ckpt = prop, n_layers, ckpt_every
        ctx.obs = (obs_x, obs_z)
        ctx.alpha_np = a
        return torch.from_numpy(c).to(alpha.device)

    @staticmethod
    def backward(ctx, grad_c):
        w = grad_c.detach().to("cpu", torch.float64).numpy()
        prop = ctx.prop
        prop.set_alpha(ctx.alpha_np)
        _, g = prop.adjoint(ctx.n_layers, _ObsWeights(ctx.obs[0], ctx.obs[1], w), ctx.ckpt)
        return (torch.from_numpy(g).to(grad_c.device), None, None, None, None, None)


def thermal_coefficients(alpha, prop, n_layers, obs_x, obs_z, ckpt_every=10):
    return ThermalCoefficients.apply(alpha, prop, int(n_layers), np.ascontiguousarray(obs_x),
                                     np.ascontiguousarray(obs_z), int(ckpt_every))
