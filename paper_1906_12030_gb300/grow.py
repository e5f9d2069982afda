"""Bond-dimension growth of a MERA: a warm start at a larger chi from a MERA
optimised at a smaller one (standard practice for variational MERA; the paper
states no schedule).

Every tensor is embedded in the larger index spaces (zero padding), a small
seeded perturbation is added so that the new directions are populated, and
the result is made isometric (w) or unitary (u) again by the library's polar
update: the polar factor of X is -mera_polar_update(-X), computed on the GPU
in binary64.  rho* is embedded the same way (it stays a density matrix of
unit trace) and serves as the fixed point's warm start.  Only data movement
runs in PyTorch; the polar iterations are the library's kernels.
"""
from __future__ import annotations

from . import api


def _polar(x, rows: int, cols: int):
    """Polar factor of the rows x cols matrix x (rows >= cols)."""
    import torch

    out = torch.empty(rows * cols, dtype=torch.float64, device=x.device)
    api.mera_polar_update((-x).reshape(-1).contiguous(), rows, cols, out)
    return out


def grow_state(state: api.MeraState, layer_dims_new, seed: int = 0, eps: float = 1e-3) -> api.MeraState:
    """A new MeraState with the layer dimensions `layer_dims_new` (list of
    (chi_b, chi_t), bottom layer first, each >= the old one) that contains
    `state` in the leading index ranges of every tensor."""
    import torch

    if len(layer_dims_new) != len(state.us):
        raise ValueError("the number of layers must not change")
    dev = state.rho_star.device
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    us, ws = [], []
    for (cb, ct), (nb, nt), u, w in zip(zip(state.chi_b, state.chi_t), layer_dims_new, state.us, state.ws):
        if nb < cb or nt < ct or nt > nb * nb:
            raise ValueError(f"cannot grow a ({cb}, {ct}) layer to ({nb}, {nt})")
        u2 = eps * torch.randn((nb,) * 4, dtype=torch.float64, device=dev, generator=g)
        u2[:cb, :cb, :cb, :cb] += u.reshape((cb,) * 4)
        w2 = eps * torch.randn((nb, nb, nt), dtype=torch.float64, device=dev, generator=g)
        w2[:cb, :cb, :ct] += w.reshape(cb, cb, ct)
        us.append(_polar(u2.reshape(nb * nb, nb * nb), nb * nb, nb * nb))
        ws.append(_polar(w2.reshape(nb * nb, nt), nb * nb, nt).reshape(nb, nb, nt))
    ct, nt = state.chi_t[-1], layer_dims_new[-1][1]
    rho = torch.zeros((nt,) * 6, dtype=torch.float64, device=dev)
    rho[:ct, :ct, :ct, :ct, :ct, :ct] = state.rho_star.reshape((ct,) * 6)
    return api.MeraState(us, ws, rho.reshape(-1))
