"""torch.autograd.Function for G_pq(w) with an adjoint backward (argument marshalling only).

forward: G_pq(w) for real frequencies w (tensor [nw]) and broadening eta (0-d tensor), computed by the
CUDA library together with the adjoint-solve derivatives dG/dw = -y_q^T x_p and dG/deta = i y_q^T x_p
(gfcc_green_derivatives). backward: for real inputs and a complex output the vector-Jacobian product is
Re(sum conj(grad_G) * dG/dinput). When the doubles amplitudes t2 (the tensor the context was built from)
are passed and require a gradient, backward also returns dL/dt2 from gfcc_green_grad_t2 (adjoint solves
weighted by grad_G; the forward solutions are recomputed there, not stored).
"""
from __future__ import annotations

import numpy as np
import torch


class GreenFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omegas, eta, t2, gfcc_ctx, orbitals, qorb=None):
        w = omegas.detach().to("cpu", torch.float64).numpy()
        G, dw, de = gfcc_ctx.green_derivatives(w, float(eta.detach().cpu()), orbitals, qorb)
        dev = omegas.device
        ctx.save_for_backward(torch.from_numpy(dw).to(dev), torch.from_numpy(de).to(dev))
        ctx.gfcc = (gfcc_ctx, w, float(eta.detach().cpu()), orbitals, qorb)
        return torch.from_numpy(G).to(dev)

    @staticmethod
    def backward(ctx, grad_G):
        dw, de = ctx.saved_tensors
        gw = (grad_G.conj() * dw).real.sum(dim=(1, 2))
        ge = (grad_G.conj() * de).real.sum()
        gt2 = None
        if ctx.needs_input_grad[2]:
            g, w, eta, orbitals, qorb = ctx.gfcc
            _, t2bar = g.green_grad_t2(w, eta, orbitals, grad_G.detach().cpu().numpy(), qorb)
            gt2 = torch.from_numpy(t2bar).to(grad_G.device)
        return gw, ge, gt2, None, None, None


def green(omegas, eta, gfcc_ctx, orbitals, qorb=None, t2=None):
    """Differentiable G_pq(w): omegas [nw] float64 tensor, eta 0-d float64 tensor; t2 (optional) the
    [o, o, v, v] float64 tensor of doubles amplitudes the context was built from, to receive dL/dt2."""
    return GreenFunction.apply(omegas, eta, t2, gfcc_ctx, list(orbitals), None if qorb is None else list(qorb))


def spectral(G: torch.Tensor) -> torch.Tensor:
    """A(w) = -(1/pi) sum_p Im G_pp for G [nw, n, n] with the same p and q sets."""
    return -torch.diagonal(G, dim1=1, dim2=2).imag.sum(dim=1) / np.pi
