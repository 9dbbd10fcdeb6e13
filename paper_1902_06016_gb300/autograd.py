"""torch.autograd.Function for G_pq(w) with an adjoint backward (argument marshalling only).

forward: G_pq(w) for real frequencies w (tensor [nw]) and broadening eta (0-d tensor), computed by the
CUDA library; when w or eta needs a gradient, together with the adjoint-solve derivatives
dG/dw = -y_q^T x_p and dG/deta = i y_q^T x_p (gfcc_green_derivatives), otherwise by the forward solves
alone (gfcc_solve_full). backward: for real inputs and a complex output the vector-Jacobian product is
Re(sum conj(grad_G) * dG/dinput). When the doubles amplitudes t2 (the tensor the context was built from)
are passed and require a gradient, backward also returns dL/dt2 from gfcc_green_grad_t2 (adjoint solves
weighted by grad_G; the forward solutions are recomputed there, not stored).
"""
from __future__ import annotations

import torch


class GreenFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omegas, eta, t2, gfcc_ctx, orbitals, qorb=None):
        w = omegas.detach().to("cpu", torch.float64).numpy()
        e = float(eta.detach().cpu())
        dev = omegas.device
        ctx.gfcc = (gfcc_ctx, w, e, orbitals, qorb)
        ctx.w_or_eta = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        if ctx.w_or_eta:   # forward and adjoint solves: G and its frequency / broadening derivatives
            G, dw, de = gfcc_ctx.green_derivatives(w, e, orbitals, qorb)
            ctx.save_for_backward(torch.from_numpy(dw).to(dev), torch.from_numpy(de).to(dev))
        else:              # no derivative in w or eta wanted: forward solves only
            G = gfcc_ctx.solve_full(w, e, orbitals, qorb=qorb, want_A=False)["G"]
        return torch.from_numpy(G).to(dev)

    @staticmethod
    def backward(ctx, grad_G):
        gw = ge = None
        if ctx.w_or_eta:
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


class SpectralFunction(torch.autograd.Function):
    """A(w) = -(1/pi) sum_p Im G_pp(w) by gfcc_spectral, its backward by the library's adjoint map."""

    @staticmethod
    def forward(ctx, G, orbitals, qorb=None):
        from . import gfcc
        ctx.sp = (list(orbitals), None if qorb is None else list(qorb), G.shape[2], G.device)
        Gc = G.detach().contiguous()
        Gh = Gc.cpu().numpy() if not Gc.is_cuda else Gc
        A = gfcc.spectral(Gh, orbitals, qorb)
        return torch.as_tensor(A).to(G.device)

    @staticmethod
    def backward(ctx, grad_A):
        from . import gfcc
        orbitals, qorb, nq, dev = ctx.sp
        ga = grad_A.detach().to(torch.float64).contiguous()
        gh = ga.cpu().numpy() if not ga.is_cuda else ga
        Gbar = gfcc.spectral_adjoint(gh, orbitals, nq, qorb)
        return torch.as_tensor(Gbar).to(dev), None, None


def spectral(G: torch.Tensor, orbitals=None, qorb=None) -> torch.Tensor:
    """A(w) = -(1/pi) sum_p Im G_pp for G [nw, np, nq] (differentiable). orbitals / qorb: the p and q
    sets G was computed for (default: the same set, G square)."""
    if orbitals is None:
        orbitals = list(range(G.shape[1]))
    return SpectralFunction.apply(G, list(orbitals), None if qorb is None else list(qorb))
