"""Differentiable energy: a torch.autograd.Function around mera_energy.

E(h, rho, u, w) = tr(A(h) rho) (Sec. II B).  The adjoint is the library's
mera_energy_adjoint (no tape of intermediates is kept; every backward call
recomputes what it needs):

    dE/dh   = D(rho^T)                       (A and D are adjoint)
    dE/drho = A(h^T)
    dE/du   = Gamma_u(h, rho) + Gamma_u(h^T, rho^T)
    dE/dw   = Gamma_w(h, rho) + Gamma_w(h^T, rho^T)

each times the upstream gradient, all of it computed on the device by the
library; this module only allocates the outputs.  The environments hold the
bra-side holes (Fig. 4c/d, A1); exchanging the ket and bra sides of the
network transposes h and rho, so the ket-side holes are the environments of
the transposed operators.  For symmetric h and rho this is the familiar
dE/du = 2 Gamma_u, dE/dw = 2 Gamma_w.
"""
from __future__ import annotations

import torch

from . import api


class MeraEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, rho, u, w, chi_b: int, chi_t: int, prec: int = api.PREC_F64):
        e = torch.empty(1, dtype=torch.float64, device=h.device)
        api.mera_energy(h.reshape(-1), rho.reshape(-1), u.reshape(-1), w.reshape(-1), chi_b, chi_t, e, prec=prec)
        ctx.save_for_backward(h, rho, u, w)
        ctx.dims = (chi_b, chi_t, prec)
        return e.reshape(())

    @staticmethod
    def backward(ctx, g):
        h, rho, u, w = ctx.saved_tensors
        chi_b, chi_t, prec = ctx.dims
        need = ctx.needs_input_grad
        out = [torch.empty(x.shape, dtype=torch.float64, device=h.device) if need[i] else None
               for i, x in enumerate((h, rho, u, w))]
        gd = g.detach().reshape(1).to(dtype=torch.float64).contiguous()
        api.mera_energy_adjoint(h.reshape(-1), rho.reshape(-1), u.reshape(-1), w.reshape(-1), chi_b, chi_t, gd,
                                dh=out[0], drho=out[1], du=out[2], dw=out[3], prec=prec)
        return tuple(out) + (None, None, None)


def mera_energy(h, rho, u, w, chi_b: int, chi_t: int, prec: int = api.PREC_F64):
    """Differentiable tr(A(h) rho) (a 0-dim float64 tensor)."""
    return MeraEnergy.apply(h, rho, u, w, chi_b, chi_t, prec)
