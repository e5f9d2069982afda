"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module draws random numbers and shapes them into valid inputs: it holds
none of the MERA arithmetic (no superoperator, environment, update or
Hamiltonian).  Both sides receive the very same arrays, so the sign convention
of the QR factorisation used to make isometries is irrelevant to parity.

Tensor conventions (real arithmetic, row-major):

* isometry   w[a, b, c]      : a, b lower (fine) legs, c upper (coarse) leg,
                                sum_ab w[a,b,c] w[a,b,c'] = delta_cc'   (Eq. iso)
* disentangler u[a, b, m, n] : a, b lower legs, m, n upper legs,
                                sum_ab u[a,b,m,n] u[a,b,m',n'] = delta delta (Eq. unitarity)
* 3-site operator X[i1,i2,i3, j1,j2,j3]: ket legs first, then bra legs.

Layer dimensions follow the scale-invariant MERA of Sec. II A with tau* = 3:
two transitional layers and one scale-invariant layer.  The physical sites are
spins blocked in pairs (local dimension 4); the first layer maps 4 -> min(16, chi),
the second min(16, chi) -> chi, the scale-invariant layer chi -> chi.
"""
from __future__ import annotations

import numpy as np

D_PHYS = 4  # two spin-1/2 sites blocked into one site


def layer_dims(chi: int, n_layers: int = 3, d: int = D_PHYS) -> list[tuple[int, int]]:
    """(chi_bottom, chi_top) of every layer, bottom layer first."""
    dims = []
    bottom = d
    for tau in range(n_layers):
        top = min(bottom * bottom, chi)
        dims.append((bottom, top))
        bottom = top
    return dims


def random_isometry(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Orthonormal columns from the QR factorisation of an N(0,1) matrix."""
    if cols > rows:
        raise ValueError("an isometry needs rows >= cols")
    g = rng.standard_normal((rows, cols))
    q, _ = np.linalg.qr(g)
    return np.ascontiguousarray(q[:, :cols])


def random_w(rng: np.random.Generator, chi_b: int, chi_t: int) -> np.ndarray:
    return random_isometry(rng, chi_b * chi_b, chi_t).reshape(chi_b, chi_b, chi_t)


def random_u(rng: np.random.Generator, chi_b: int) -> np.ndarray:
    return random_isometry(rng, chi_b * chi_b, chi_b * chi_b).reshape(chi_b, chi_b, chi_b, chi_b)


def parity_labels(dim: int, physical: bool = False) -> np.ndarray:
    """Z2 charge of each basis state of a leg.  Physical (blocked) site:
    index 2 s0 + s1 of two spins in the Z basis, charge = s0 xor s1 (the
    parity prod Z of the transverse-field Ising chain).  Bond legs: the first
    ceil(dim/2) states even, the rest odd."""
    if physical:
        return np.array([bin(i).count("1") % 2 for i in range(dim)])
    return (np.arange(dim) >= (dim + 1) // 2).astype(int)


def _block_isometry(rng, rows_p, cols_p, n_rows, n_cols):
    """An n_rows x n_cols isometry that maps only rows of charge p to columns
    of charge p (rows_p, cols_p: charge of each row / column)."""
    q = np.zeros((n_rows, n_cols))
    for p in (0, 1):
        r = np.flatnonzero(rows_p == p)
        c = np.flatnonzero(cols_p == p)
        if len(c) == 0:
            continue
        q[np.ix_(r, c)] = random_isometry(rng, len(r), len(c))
    return q


def init_mera(seed: int, chi: int, n_layers: int = 3, d: int = D_PHYS, z2: bool = False):
    """Seeded initial tensors: list of (u, w) per layer, bottom layer first.
    z2: tensors that commute with the chain's Z2 parity (block-diagonal in
    the charges of parity_labels), which the sweep then keeps."""
    rng = np.random.default_rng(seed)
    layers = []
    pb = parity_labels(d, physical=True)
    for chi_b, chi_t in layer_dims(chi, n_layers, d):
        if not z2:
            u = random_u(rng, chi_b)
            w = random_w(rng, chi_b, chi_t)
        else:
            pt = parity_labels(chi_t)
            pair = (pb[:, None] ^ pb[None, :]).reshape(-1)
            u = _block_isometry(rng, pair, pair, chi_b * chi_b, chi_b * chi_b).reshape((chi_b,) * 4)
            w = _block_isometry(rng, pair, pt, chi_b * chi_b, chi_t).reshape(chi_b, chi_b, chi_t)
            pb = pt
        layers.append((u, w))
    return layers


def random_operator(rng: np.random.Generator, chi: int, symmetric: bool = True) -> np.ndarray:
    """A random 3-site operator (chi^3 x chi^3), optionally symmetric."""
    n = chi ** 3
    x = rng.standard_normal((n, n))
    if symmetric:
        x = 0.5 * (x + x.T)
    return x.reshape((chi,) * 6)


def random_density(rng: np.random.Generator, chi: int) -> np.ndarray:
    """A random 3-site density matrix: symmetric, positive semidefinite, unit trace."""
    n = chi ** 3
    g = rng.standard_normal((n, n))
    r = g @ g.T
    r /= np.trace(r)
    return r.reshape((chi,) * 6)


def random_diagonal_density(rng: np.random.Generator, chi: int) -> np.ndarray:
    """A random full-rank diagonal 3-site density matrix (entries U[0.5, 1.5],
    normalised to unit trace)."""
    n = chi ** 3
    d = rng.uniform(0.5, 1.5, n)
    r = np.zeros((n, n))
    r[np.arange(n), np.arange(n)] = d / d.sum()
    return r.reshape((chi,) * 6)


def random_low_rank_density(rng: np.random.Generator, chi: int, rank: int) -> np.ndarray:
    """A random 3-site density matrix of the given rank (V V^T / tr): cheap to
    draw at large chi, where a full-rank Gram matrix costs chi^9."""
    n = chi ** 3
    v = rng.standard_normal((n, rank))
    r = v @ v.T
    r /= np.trace(r)
    return r.reshape((chi,) * 6)
