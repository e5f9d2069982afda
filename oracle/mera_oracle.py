"""Plain FP64 CPU oracle of the scale-invariant binary MERA (arXiv:1906.12030).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
module: only the test-suite, the smoke check of ``__graft_entry__`` and the
``cpu_baseline`` / reference arm of ``bench.py`` use it.  It shares no code
with the CUDA library and imports nothing from it.

Every map is written as the tensor network it is (one ``numpy.einsum`` per
diagram, in float64); numpy picks the pairwise order, which changes the result
only by rounding.  The paper defines its operators through figures that the
text does not carry (Figs. 1c, 4, 5, A1); the leg-level networks below are the
reading fixed from its text, equations and contribution counts:

* Sec. II A, Eq. (iso) and Eq. (unitarity): w[a,b,c] with lower legs a, b and
  upper leg c; u[a,b,m,n] with lower legs a, b and upper legs m, n.  Real
  arithmetic (the Ising Hamiltonian is real), so the overlines drop out.
* Sec. II B, Fig. 4(a): the ascending superoperator maps a 3-site operator one
  layer up.  In a binary MERA layer the disentanglers act on fine sites
  (2k+1, 2k+2) and the isometries on (2k, 2k+1); a 3-site operator has two
  causal-cone positions ("even": it starts on the right leg of a
  disentangler, "odd": on the left leg), and A is their average.
* Fig. 4(b): the descending superoperator D is the Hilbert-Schmidt adjoint of
  A, the same network with rho in place of the output legs.
* Fig. 4(c)/(d), Fig. A1: the environment of w has six contributions and that
  of u four: the three bra-side isometries and the two bra-side
  disentanglers, for each of the two positions.  With symmetric h and rho,
  dE/dw = 2 Gamma_w and dE/du = 2 Gamma_u.
* Fig. 5 and Sec. II C: the update is -U V^T from the SVD of the environment
  (lower legs as rows, upper legs as columns).
* stiefel_step / sweep(eta=...): a Riemannian gradient step on the Stiefel
  manifold, an alternative update (not the paper's), pinned by tangency, the
  retraction and its first-order decrease of the energy.

Pinned against the physics: a chi = 4 MERA that the oracle optimises from a
parity-symmetric start (tests/golden/make_chi4_z2_mera.py) lies within 6e-6
of the exact energy density -4/pi, and the scale-invariant ascending map of
its top layer gives the Ising-CFT scaling dimensions 1/8, 1 and the pair at
9/8 within 1 %.  Higher accuracy would need larger chi and longer runs than
the oracle can afford, so the paper's own figures (5e-10 at chi = 16) pin
nothing here.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------------------
# Hamiltonian (Eq. ham, Sec. II B).  Spins blocked in pairs to local dim 4.
# ---------------------------------------------------------------------------
PAULI_X = np.array([[0.0, 1.0], [1.0, 0.0]])
PAULI_Z = np.array([[1.0, 0.0], [0.0, -1.0]])
EYE2 = np.eye(2)


def ising_bond(hz: float) -> np.ndarray:
    """Two-spin bond -X X - (hz/2)(Z 1 + 1 Z): Eq. (ham) with the field split
    evenly over the two bonds that touch a spin (reading)."""
    return -np.kron(PAULI_X, PAULI_X) - 0.5 * hz * (np.kron(PAULI_Z, EYE2) + np.kron(EYE2, PAULI_Z))


def blocked_two_site(hz: float) -> np.ndarray:
    """h2 between blocked sites j=(s0,s1) and j+1=(s2,s3), 16 x 16.

    The intra-block bonds (s0,s1) and (s2,s3) are each shared by two blocked
    pairs and enter with weight 1/2; the inter-block bond (s1,s2) enters with 1.
    """
    b = ising_bond(hz)
    left = np.kron(b, np.eye(4))                           # spins (0,1)
    middle = np.kron(np.kron(EYE2, b), EYE2)               # spins (1,2)
    right = np.kron(np.eye(4), b)                          # spins (2,3)
    return 0.5 * left + middle + 0.5 * right


def three_site_density(h2: np.ndarray) -> np.ndarray:
    """h^{tau=1}_{n,n+1,n+2} = (h2 (x) 1 + 1 (x) h2)/2 (Sec. II B), 64 x 64."""
    d = int(round(np.sqrt(h2.shape[0])))
    return 0.5 * (np.kron(h2, np.eye(d)) + np.kron(np.eye(d), h2))


def ising_h1(hz: float = 1.0):
    """Shifted first-layer density h1 = h3 - s 1 with s = lambda_max(h3).

    Returns (h1 as a [4]*6 tensor, s).  The shift makes h1 negative
    semidefinite, so that minimising the linearised energy over isometries
    is the -U V^T update (reading of Fig. 5).
    """
    h3 = three_site_density(blocked_two_site(hz))
    s = float(np.linalg.eigvalsh(h3).max())
    h1 = h3 - s * np.eye(h3.shape[0])
    return h1.reshape((4,) * 6), s


def exact_energy_per_spin(hz: float) -> float:
    """Ground-state energy density of the infinite TFI chain (free fermions):
    e0(h) = -(1/pi) int_0^pi sqrt(1 + h^2 - 2 h cos k) dk
          = -(2 (1 + h) / pi) E(4 h / (1 + h)^2),
    E the complete elliptic integral of the second kind; -4/pi at h = 1
    (Sec. III A)."""
    from scipy.special import ellipe

    m = 4.0 * hz / (1.0 + hz) ** 2
    return -2.0 * (1.0 + hz) * float(ellipe(m)) / np.pi


# ---------------------------------------------------------------------------
# The networks (Fig. 4).  Letters are tensor legs, repeated letters summed.
# Ket-side isometries: w[x,a,p] w[b,c,q] w[d,y,r]  (outputs p, q, r)
# Bra-side isometries: w[x,A,s] w[B,C,t] w[D,y,v]  (outputs s, t, v)
# Even position: h on the right leg of the left disentangler and both legs of
#   the right one: u[e,i,a,b] u[j,k,c,d] . h[i,j,k,l,m,n] . u[e,l,A,B] u[m,n,C,D]
# Odd position: h on both legs of the left disentangler and the left leg of
#   the right one:  u[i,j,a,b] u[k,e,c,d] . h[i,j,k,l,m,n] . u[l,m,A,B] u[n,e,C,D]
# ---------------------------------------------------------------------------
_KET_W = ["xap", "bcq", "dyr"]
_BRA_W = ["xAs", "BCt", "Dyv"]
_KET_U = {"even": ["eiab", "jkcd"], "odd": ["ijab", "kecd"]}
_BRA_U = {"even": ["elAB", "mnCD"], "odd": ["lmAB", "neCD"]}
_OP = "ijklmn"       # h (or the hole of D)
_TOP = "pqrstv"      # A's output / rho's legs in D

# numpy chooses the pairwise order greedily; the memory cap is lifted so that
# it never falls back to one multi-operand loop (which would cost chi^12).
_EINSUM_OPT = ("greedy", 1e18)


def _ein(spec: str, *ops):
    return np.einsum(spec, *ops, optimize=_EINSUM_OPT)


def ascend_case(h, u, w, case: str):
    """A_case(h)[p,q,r,s,t,v] for case in {'even','odd'} (Fig. 4a)."""
    kw, bw = _KET_W, _BRA_W
    ku, bu = _KET_U[case], _BRA_U[case]
    spec = ",".join(kw + ku + [_OP] + bu + bw) + "->" + _TOP
    return _ein(spec, w, w, w, u, u, h, u, u, w, w, w)


def ascend(h, u, w):
    """A(h) = (A_even(h) + A_odd(h)) / 2."""
    return 0.5 * (ascend_case(h, u, w, "even") + ascend_case(h, u, w, "odd"))


def ascend_rows(h, u, w, rows):
    """Selected rows of A(h): for each ket triple (p, q, r) in `rows`, the
    chi_t^3 entries A(h)[p, q, r, :, :, :].  The same networks as
    ascend_case with the ket-side isometries' upper legs fixed, so a row
    costs a factor chi_t less than the whole map (used to check full-size
    results entry by entry)."""
    out = []
    for p, q, r in rows:
        acc = 0.0
        for case in ("even", "odd"):
            ku, bu = _KET_U[case], _BRA_U[case]
            spec = ",".join(["xa", "bc", "dy"] + ku + [_OP] + bu + _BRA_W) + "->stv"
            acc = acc + _ein(spec, w[:, :, p], w[:, :, q], w[:, :, r], u, u, h, u, u, w, w, w)
        out.append(0.5 * acc)
    return np.stack(out)


def descend_case(rho, u, w, case: str):
    """D_case(rho)[i,j,k,l,m,n]: the network of A_case with rho on the upper
    legs [p,q,r,s,t,v] and the lower legs open (Fig. 4b)."""
    kw, bw = _KET_W, _BRA_W
    ku, bu = _KET_U[case], _BRA_U[case]
    spec = ",".join(kw + ku + bu + bw + [_TOP]) + "->" + _OP
    return _ein(spec, w, w, w, u, u, u, u, w, w, w, rho)


def descend(rho, u, w):
    """D(rho) = (D_even(rho) + D_odd(rho)) / 2, the adjoint of A."""
    return 0.5 * (descend_case(rho, u, w, "even") + descend_case(rho, u, w, "odd"))


def descend_rows(rho, u, w, rows):
    """Selected rows of D(rho): for each ket triple (i, j, k) in `rows`, the
    chi_b^3 entries D(rho)[i, j, k, :, :, :].  The networks of descend_case
    with the ket legs i, j, k of the lower disentanglers held at one value,
    so a row costs the whole map divided by those legs' dimensions (used to
    check full-size results entry by entry)."""
    out = []
    for i, j, k in rows:
        acc = 0.0
        for case in ("even", "odd"):
            specs = _KET_W + _KET_U[case] + _BRA_U[case] + _BRA_W + [_TOP]
            ops = [w, w, w, u, u, u, u, w, w, w, rho]
            acc = acc + _fixed(specs, ops, _OP, {"i": i, "j": j, "k": k})
        out.append(0.5 * acc)
    return np.stack(out)


def energy(h, rho, u, w) -> float:
    """E(h, rho) = tr(A(h) rho) = sum A[p,q,r,s,t,v] rho[s,t,v,p,q,r]."""
    a = ascend(h, u, w)
    return float(np.einsum("pqrstv,stvpqr->", a, rho))


def _env_network(h, rho, u, w, case: str, hole: tuple[str, int]):
    """One contribution: the network of E_case with one bra-side tensor removed.

    hole = ('w', k) removes bra isometry k in {0,1,2} (left, centre, right);
    hole = ('u', k) removes bra disentangler k in {0,1}.  The open legs come
    out in the removed tensor's own leg order.
    """
    kind, k = hole
    kw, ku = _KET_W, _KET_U[case]
    bu, bw = list(_BRA_U[case]), list(_BRA_W)
    rho_legs = "stvpqr"   # rho[s,t,v,p,q,r] closes tr(A(h) rho)
    if kind == "w":
        out = bw.pop(k)
        ops_bw = [w] * len(bw)
        specs = kw + ku + [_OP] + bu + bw + [rho_legs]
        ops = [w, w, w, u, u, h, u, u] + ops_bw + [rho]
    else:
        out = bu.pop(k)
        specs = kw + ku + [_OP] + bu + bw + [rho_legs]
        ops = [w, w, w, u, u, h, u, w, w, w, rho]
    return _ein(",".join(specs) + "->" + out, *ops)


def env_w(h, rho, u, w):
    """Gamma_w[a,b,c]: half the sum of the 6 bra-isometry holes (Fig. 4c, A1a)."""
    g = np.zeros_like(w)
    for case in ("even", "odd"):
        for k in range(3):
            g += _env_network(h, rho, u, w, case, ("w", k))
    return 0.5 * g


def env_u(h, rho, u, w):
    """Gamma_u[a,b,m,n]: half the sum of the 4 bra-disentangler holes (Fig. 4d, A1b)."""
    g = np.zeros_like(u)
    for case in ("even", "odd"):
        for k in range(2):
            g += _env_network(h, rho, u, w, case, ("u", k))
    return 0.5 * g


def _fixed(specs, ops, out, fixed):
    """The network with the legs in `fixed` (letter -> index) held at one
    value: every operand carrying such a leg is sliced there, and the leg
    leaves the output.  Costs the whole network divided by the fixed legs'
    dimensions."""
    specs2, ops2 = [], []
    for sp, op in zip(specs, ops):
        for letter, idx in fixed.items():
            if letter in sp:
                op = np.take(op, idx, axis=sp.index(letter))
                sp = sp.replace(letter, "")
        specs2.append(sp)
        ops2.append(op)
    out2 = "".join(c for c in out if c not in fixed)
    return _ein(",".join(specs2) + "->" + out2, *ops2)


def env_w_cols(h, rho, u, w, cols):
    """Gamma_w[:, :, c] for each c in `cols`: env_w's six networks with the
    removed isometry's upper leg fixed (used to check full-size results entry
    by entry)."""
    out = []
    for c in cols:
        g = 0.0
        for case in ("even", "odd"):
            for k in range(3):
                bw = list(_BRA_W)
                hole = bw.pop(k)
                specs = _KET_W + _KET_U[case] + [_OP] + list(_BRA_U[case]) + bw + ["stvpqr"]
                ops = [w, w, w, u, u, h, u, u, w, w, rho]
                g = g + _fixed(specs, ops, hole, {hole[2]: c})
        out.append(0.5 * g)
    return np.stack(out)


def env_u_rows(h, rho, u, w, rows):
    """Gamma_u[a, b, :, :] for each (a, b) in `rows`: env_u's four networks
    with the removed disentangler's lower legs fixed."""
    out = []
    for a, b in rows:
        g = 0.0
        for case in ("even", "odd"):
            for k in range(2):
                bu = list(_BRA_U[case])
                hole = bu.pop(k)
                specs = _KET_W + _KET_U[case] + [_OP] + bu + list(_BRA_W) + ["stvpqr"]
                ops = [w, w, w, u, u, h, u, w, w, w, rho]
                g = g + _fixed(specs, ops, hole, {hole[0]: a, hole[1]: b})
        out.append(0.5 * g)
    return np.stack(out)


# ---------------------------------------------------------------------------
# Update (Fig. 5): SVD of the environment, new tensor from U and V.
# ---------------------------------------------------------------------------
def polar_update(env: np.ndarray, n_lower: int) -> np.ndarray:
    """X = -U V^T where env, reshaped (lower legs) x (upper legs), is U S V^T.

    The minus sign is the reading that goes with the negative-semidefinite
    shifted Hamiltonian: -U V^T minimises tr(env^T X) over isometries X.
    """
    shape = env.shape
    rows = int(np.prod(shape[:n_lower]))
    mat = env.reshape(rows, -1)
    uu, _, vt = np.linalg.svd(mat, full_matrices=False)
    return (-(uu @ vt)).reshape(shape)


def stiefel_step(x: np.ndarray, g: np.ndarray, eta: float) -> np.ndarray:
    """One Riemannian gradient step on the Stiefel manifold, embedded metric
    (the update the paper's Fig. A1 caption points to when it mentions
    gradients; not the paper's own SVD update): the Euclidean gradient g is
    projected onto the tangent space at the isometry x,
        r = g - x sym(x^T g),   sym(a) = (a + a^T) / 2,
    and x - eta r is retracted to the manifold by its polar factor (SVD).
    x, g: m x n matrices (m >= n)."""
    a = x.T @ g
    r = g - x @ (0.5 * (a + a.T))
    uu, _, vt = np.linalg.svd(x - eta * r, full_matrices=False)
    return uu @ vt


def update_u(h, rho, u, w):
    return polar_update(env_u(h, rho, u, w), 2)


def update_w(h, rho, u, w):
    return polar_update(env_w(h, rho, u, w), 2)


# ---------------------------------------------------------------------------
# Scale-invariant fixed point (Sec. II B: dominant eigenvector of D_SI).
# ---------------------------------------------------------------------------
def symmetrize_normalize(x: np.ndarray) -> np.ndarray:
    """(X + X^T)/2 with ^T exchanging the ket and bra triples, then / trace."""
    n = int(round(x.size ** 0.5))
    m = x.reshape(n, n)
    m = 0.5 * (m + m.T)
    m = m / np.trace(m)
    return m.reshape(x.shape)


def fixed_point_rho(u, w, rho0, n_iter: int):
    """Power iteration rho <- sym(D(rho)) / tr (reading of 'iterative methods').

    Returns (rho, residual) with residual = ||rho_k - rho_{k-1}||_F of the last
    step (0.0 if n_iter == 0).
    """
    rho = rho0
    resid = 0.0
    for _ in range(n_iter):
        new = symmetrize_normalize(descend(rho, u, w))
        resid = float(np.linalg.norm(new - rho))
        rho = new
    return rho, resid


def identity_density(chi: int) -> np.ndarray:
    n = chi ** 3
    return (np.eye(n) / n).reshape((chi,) * 6)


# ---------------------------------------------------------------------------
# Sweep (Sec. II C).  layers = [(u1, w1), (u2, w2), (u3, w3)], bottom first;
# the last one is the scale-invariant layer.
# ---------------------------------------------------------------------------
def sweep(layers, h1, shift, rho_star, n_pow: int = 20, eta: float | None = None):
    """One optimisation sweep.  Returns (new_layers, rho_star, e_per_spin).
    eta None: the paper's SVD (polar) update of each tensor; eta > 0: a
    Riemannian gradient step of size eta instead (stiefel_step with the
    energy's gradient 2 Gamma, the environments being half the gradient).

    1. ascend h1 through the transitional layers (old tensors),
    2. rho* <- n_pow power iterations of the SI descending map (warm start),
    3. update the SI layer: u from its environment (h_{tau*}, rho*), then w
       with the new u,
    4. transitional layers top-down: u, then w, then descend rho one layer
       (the layer just below the SI layers sees rho* itself),
    5. energy per spin (tr(h1 rho1) + shift) / 2 with the new tensors.
    rho* is not recomputed between the SI update and the descent (reading).
    """
    layers = [(u.copy(), w.copy()) for u, w in layers]
    n = len(layers)
    hs = [h1]
    for tau in range(n - 1):
        u, w = layers[tau]
        hs.append(ascend(hs[tau], u, w))
    u, w = layers[-1]
    rho_star, _ = fixed_point_rho(u, w, rho_star, n_pow)
    rho_above = rho_star
    for tau in range(n - 1, -1, -1):
        u, w = layers[tau]
        if eta is None:
            u = update_u(hs[tau], rho_above, u, w)
            w = update_w(hs[tau], rho_above, u, w)
        else:
            cb, ct = w.shape[0], w.shape[2]
            gu = 2.0 * env_u(hs[tau], rho_above, u, w)
            u = stiefel_step(u.reshape(cb * cb, cb * cb), gu.reshape(cb * cb, cb * cb), eta).reshape(u.shape)
            gw = 2.0 * env_w(hs[tau], rho_above, u, w)
            w = stiefel_step(w.reshape(cb * cb, ct), gw.reshape(cb * cb, ct), eta).reshape(w.shape)
        layers[tau] = (u, w)
        if 0 < tau < n - 1:
            # rho_{tau*} = rho* sits on top of the last transitional layer;
            # it is descended through the transitional layers only.
            rho_above = descend(rho_above, u, w)
    u1, w1 = layers[0]
    e_site = energy(h1, rho_above, u1, w1) + shift
    return layers, rho_star, 0.5 * e_site


def run(layers, hz: float = 1.0, n_sweeps: int = 10, n_pow: int = 20):
    """Repeated sweeps from the given tensors; returns (layers, rho*, energies)."""
    h1, shift = ising_h1(hz)
    chi = layers[-1][1].shape[2]
    rho_star = identity_density(chi)
    energies = []
    for _ in range(n_sweeps):
        layers, rho_star, e = sweep(layers, h1, shift, rho_star, n_pow)
        energies.append(e)
    return layers, rho_star, energies


def energy_per_spin(layers, h1, shift, rho0, n_pow: int = 200):
    """Energy per spin of the MERA as it stands: rho* from n_pow power
    iterations of the SI descending map, descended to the physical lattice,
    then (tr(h1 rho1) + shift) / 2.  A variational upper bound on e0."""
    u, w = layers[-1]
    rho, _ = fixed_point_rho(u, w, rho0, n_pow)
    for tau in range(len(layers) - 2, 0, -1):
        u, w = layers[tau]
        rho = descend(rho, u, w)
    u1, w1 = layers[0]
    return 0.5 * (energy(h1, rho, u1, w1) + shift)


# ---------------------------------------------------------------------------
# Scaling dimensions (Sec. II B, III A): eigenvalues lambda = 2^-Delta of the
# scale-invariant ascending superoperator.
# ---------------------------------------------------------------------------
def ascend_matrix(u, w) -> np.ndarray:
    """Dense chi^6 x chi^6 matrix of A_SI (columns are A(e_k)); small chi only."""
    chi = w.shape[2]
    n = chi ** 6
    cols = np.empty((n, n))
    basis = np.zeros(n)
    for k in range(n):
        basis[:] = 0.0
        basis[k] = 1.0
        cols[:, k] = ascend(basis.reshape((chi,) * 6), u, w).reshape(-1)
    return cols


def scaling_dimensions(u, w, n_dims: int = 12) -> np.ndarray:
    """Delta_n = -log2 |lambda_n| for the n_dims largest |lambda| of A_SI."""
    chi = w.shape[2]
    n = chi ** 6
    if chi <= 3:
        lam = np.linalg.eigvals(ascend_matrix(u, w))
    else:
        from scipy.sparse.linalg import LinearOperator, eigs

        op = LinearOperator((n, n), dtype=np.float64,
                            matvec=lambda v: ascend(v.reshape((chi,) * 6), u, w).reshape(-1))
        lam = eigs(op, k=min(n_dims, n - 2), which="LM", return_eigenvectors=False, tol=1e-12)
    mags = np.sort(np.abs(lam))[::-1][:n_dims]
    return -np.log2(mags)
