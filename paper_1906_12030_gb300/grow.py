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


def _leg_map(old: int, new: int, z2: bool):
    """New positions of a leg's old basis states when it grows from `old` to
    `new` states.  Without symmetry: the leading range.  With the Z2 parity
    (bond legs: the first ceil(dim/2) states even, the rest odd, as in the
    parity-symmetric initial states): the even states keep their place and
    the odd ones move to the start of the new odd range, so every state keeps
    its charge."""
    if not z2:
        return list(range(old))
    h_old, h_new = (old + 1) // 2, (new + 1) // 2
    return [i if i < h_old else h_new + (i - h_old) for i in range(old)]


def grow_state(state: api.MeraState, layer_dims_new, seed: int = 0, eps: float = 1e-3, z2: bool = False,
               bottom_parity=None) -> api.MeraState:
    """A new MeraState with the layer dimensions `layer_dims_new` (list of
    (chi_b, chi_t), bottom layer first, each >= the old one) that contains
    `state` in every tensor, at the positions of _leg_map.  z2: keep the
    chain's Z2 parity -- the old states keep their charges and the
    perturbation only fills parity-conserving entries, so a parity-symmetric
    MERA grows into a parity-symmetric one; bottom_parity gives the charges
    of the bottom layer's (physical, never grown) basis states."""
    import torch

    if len(layer_dims_new) != len(state.us):
        raise ValueError("the number of layers must not change")
    if z2 and (bottom_parity is None or len(bottom_parity) != state.chi_b[0]):
        raise ValueError("z2 growth needs the parity of the bottom layer's basis states")
    dev = state.rho_star.device
    g = torch.Generator(device=dev)
    g.manual_seed(seed)

    def charges(dim, bottom):
        if bottom:
            return torch.tensor([int(x) for x in bottom_parity], device=dev)
        return (torch.arange(dim, device=dev) >= (dim + 1) // 2).long()

    def embed(dst, src, maps):
        """dst[map0[i0], map1[i1], ...] += src[i0, i1, ...] (the maps are
        one-to-one)."""
        nd = len(maps)
        idx = tuple(torch.tensor(mp, device=dev).view([-1 if a == j else 1 for a in range(nd)])
                    for j, mp in enumerate(maps))
        dst[idx] += src
        return dst

    us, ws = [], []
    for k, ((cb, ct), (nb, nt), u, w) in enumerate(zip(zip(state.chi_b, state.chi_t), layer_dims_new, state.us,
                                                       state.ws)):
        if nb < cb or nt < ct or nt > nb * nb or (k == 0 and nb != cb and z2):
            raise ValueError(f"cannot grow a ({cb}, {ct}) layer to ({nb}, {nt})")
        mb = _leg_map(cb, nb, z2 and k > 0)  # the bottom layer's physical legs keep their basis
        mt = _leg_map(ct, nt, z2)
        u2 = eps * torch.randn((nb,) * 4, dtype=torch.float64, device=dev, generator=g)
        w2 = eps * torch.randn((nb, nb, nt), dtype=torch.float64, device=dev, generator=g)
        if z2:
            pb, pt = charges(nb, k == 0), charges(nt, False)
            pair = (pb.view(-1, 1) ^ pb.view(1, -1))
            u2 *= (pair.view(nb, nb, 1, 1) == pair.view(1, 1, nb, nb)).to(torch.float64)
            w2 *= (pair.view(nb, nb, 1) == pt.view(1, 1, nt)).to(torch.float64)
        embed(u2, u.reshape((cb,) * 4), [mb] * 4)
        embed(w2, w.reshape(cb, cb, ct), [mb, mb, mt])
        us.append(_polar(u2.reshape(nb * nb, nb * nb), nb * nb, nb * nb))
        ws.append(_polar(w2.reshape(nb * nb, nt), nb * nb, nt).reshape(nb, nb, nt))
    ct, nt = state.chi_t[-1], layer_dims_new[-1][1]
    rho = torch.zeros((nt,) * 6, dtype=torch.float64, device=dev)
    embed(rho, state.rho_star.reshape((ct,) * 6), [_leg_map(ct, nt, z2)] * 6)
    return api.MeraState(us, ws, rho.reshape(-1))
