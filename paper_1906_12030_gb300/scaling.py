"""Scaling dimensions from the scale-invariant ascending superoperator.

Sec. II B / III A: the eigenvalues lambda of the scale-invariant ascending
map A are lambda = 2^-Delta; the paper reads the lowest twelve Delta at
chi = 16 (Fig. 7).  A acts on chi^6-dimensional operators, so its leading
eigenvalues come from an implicitly restarted Arnoldi iteration (ARPACK
through scipy, binary64 on the host) whose every matrix-vector product is
one `mera_ascend` call on the GPU -- the O(chi^9) part runs in the library's
kernels; only the small Krylov eigen-problem is solved on the host.
"""
from __future__ import annotations

import numpy as np

from . import api


def ascend_eigenvalues(u, w, chi: int, k: int = 12, prec: int = api.PREC_F64, tol: float = 1e-12,
                       stream=None):
    """The k eigenvalues of largest modulus of A_SI (u, w: device tensors of
    one chi -> chi layer).  Returns a complex numpy array sorted by |lambda|."""
    import torch
    from scipy.sparse.linalg import LinearOperator, eigs

    n = chi ** 6
    dev = u.device
    x = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    ws = api.workspace(api.mera_workspace_size(api.OP_ASCEND, chi, chi, prec), dev)
    ud, wd = u.reshape(-1), w.reshape(-1)

    def matvec(v):
        x.copy_(torch.from_numpy(np.ascontiguousarray(np.real(v), dtype=np.float64)))
        api.mera_ascend(x, ud, wd, chi, chi, y, prec=prec, ws=ws, stream=stream)
        return y.cpu().numpy()

    op = LinearOperator((n, n), matvec=matvec, dtype=np.float64)
    kk = min(k, n - 2)
    lam = eigs(op, k=kk, which="LM", return_eigenvectors=False, tol=tol, v0=np.ones(n) / np.sqrt(n))
    return lam[np.argsort(-np.abs(lam))]


def scaling_dimensions(u, w, chi: int, k: int = 12, prec: int = api.PREC_F64, tol: float = 1e-12):
    """Delta_n = -log2 |lambda_n| for the k largest |lambda| of A_SI, ascending."""
    lam = ascend_eigenvalues(u, w, chi, k, prec, tol)
    return np.sort(-np.log2(np.abs(lam)))
