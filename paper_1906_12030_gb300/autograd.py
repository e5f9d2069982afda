"""Differentiable energy: a torch.autograd.Function around mera_energy.

E(h, rho, u, w) = tr(A(h) rho) (Sec. II B).  The adjoint is written by hand
from the library's own maps (no tape of intermediates is kept; every
backward call recomputes what it needs):

    dE/dh   = D(rho^T)                       (A and D are adjoint)
    dE/drho = A(h^T)
    dE/du   = Gamma_u(h, rho) + Gamma_u(h^T, rho^T)
    dE/dw   = Gamma_w(h, rho) + Gamma_w(h^T, rho^T)

The environments hold the bra-side holes (Fig. 4c/d, A1); exchanging the ket
and bra sides of the network transposes h and rho, so the ket-side holes are
the environments of the transposed operators.  For symmetric h and rho this
is the familiar dE/du = 2 Gamma_u, dE/dw = 2 Gamma_w.
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
        dev = h.device
        f = lambda n: torch.empty(n, dtype=torch.float64, device=dev)  # noqa: E731
        hf, rf, uf, wf = h.reshape(-1), rho.reshape(-1), u.reshape(-1), w.reshape(-1)
        ht = api.mera_op_transpose(hf, chi_b, f(chi_b ** 6))
        rt = api.mera_op_transpose(rf, chi_t, f(chi_t ** 6))
        grads = [None] * 4
        if ctx.needs_input_grad[0]:
            grads[0] = api.mera_descend(rt, uf, wf, chi_b, chi_t, f(chi_b ** 6), prec=prec).reshape(h.shape)
        if ctx.needs_input_grad[1]:
            grads[1] = api.mera_ascend(ht, uf, wf, chi_b, chi_t, f(chi_t ** 6), prec=prec).reshape(rho.shape)
        if ctx.needs_input_grad[2]:
            a = api.mera_env_u(hf, rf, uf, wf, chi_b, chi_t, f(chi_b ** 4), prec=prec)
            b = api.mera_env_u(ht, rt, uf, wf, chi_b, chi_t, f(chi_b ** 4), prec=prec)
            grads[2] = (a + b).reshape(u.shape)
        if ctx.needs_input_grad[3]:
            a = api.mera_env_w(hf, rf, uf, wf, chi_b, chi_t, f(chi_b ** 2 * chi_t), prec=prec)
            b = api.mera_env_w(ht, rt, uf, wf, chi_b, chi_t, f(chi_b ** 2 * chi_t), prec=prec)
            grads[3] = (a + b).reshape(w.shape)
        return tuple(None if x is None else g * x for x in grads) + (None, None, None)


def mera_energy(h, rho, u, w, chi_b: int, chi_t: int, prec: int = api.PREC_F64):
    """Differentiable tr(A(h) rho) (a 0-dim float64 tensor)."""
    return MeraEnergy.apply(h, rho, u, w, chi_b, chi_t, prec)
