"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test uses an independent
construction (dense lattice operators, Kronecker products, finite
differences, closed forms, exact invariants) chosen so that a dropped term,
a wrong sign, a swapped leg or a transposed operand in the oracle fails one
of them.
"""
import json
import os

import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _mat(x):
    n = int(round(x.size ** 0.5))
    return x.reshape(n, n)


def _rng(seed=0):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# Hamiltonian: blocked 3-site densities sum to the dense spin Hamiltonian.
# --------------------------------------------------------------------------
def _embed(op, sites, nsites, d):
    """Dense operator on nsites sites (dim d each) acting as `op` on `sites`."""
    k = len(sites)
    t = op.reshape((d,) * (2 * k))
    rest = [s for s in range(nsites) if s not in sites]
    eye = np.eye(d ** len(rest)).reshape((d,) * (2 * len(rest)))
    full = np.tensordot(t, eye, axes=0)  # legs: op ket, op bra, rest ket, rest bra
    ket_order = list(sites) + rest
    # full legs are [op kets (k), op bras (k), rest kets, rest bras]
    n_rest = len(rest)
    src_ket = list(range(k)) + list(range(2 * k, 2 * k + n_rest))
    src_bra = list(range(k, 2 * k)) + list(range(2 * k + n_rest, 2 * k + 2 * n_rest))
    perm_ket = [src_ket[ket_order.index(s)] for s in range(nsites)]
    perm_bra = [src_bra[ket_order.index(s)] for s in range(nsites)]
    return np.transpose(full, perm_ket + perm_bra).reshape(d ** nsites, d ** nsites)


def _dense_ising_ring(nspins, hz):
    x = np.array([[0.0, 1.0], [1.0, 0.0]])
    z = np.array([[1.0, 0.0], [0.0, -1.0]])
    h = np.zeros((2 ** nspins, 2 ** nspins))
    for n in range(nspins):
        h -= _embed(np.kron(x, x), [n, (n + 1) % nspins], nspins, 2)
        h -= hz * _embed(z, [n], nspins, 2)
    return h


@pytest.mark.parametrize("nblocks", [3, 4])
@pytest.mark.parametrize("hz", [1.0, 0.7])
def test_blocked_density_sums_to_dense_hamiltonian(nblocks, hz):
    h3 = O.three_site_density(O.blocked_two_site(hz))
    total = np.zeros((4 ** nblocks, 4 ** nblocks))
    for j in range(nblocks):
        total += _embed(h3, [j, (j + 1) % nblocks, (j + 2) % nblocks], nblocks, 4)
    dense = _dense_ising_ring(2 * nblocks, hz)  # block j = spins (2j, 2j+1)
    assert np.abs(total - dense).max() < 1e-13


def test_shifted_density_is_negative_semidefinite():
    h1, s = O.ising_h1(1.0)
    ev = np.linalg.eigvalsh(_mat(h1))
    assert ev.max() == pytest.approx(0.0, abs=1e-13)
    h3 = O.three_site_density(O.blocked_two_site(1.0))
    assert np.abs(_mat(h1) + s * np.eye(64) - h3).max() < 1e-15


def test_exact_energy_closed_form():
    gold = json.load(open(GOLDEN))
    assert O.exact_energy_per_spin(1.0) == pytest.approx(gold["e_exact_per_spin"]["value"], abs=1e-15)
    assert O.exact_energy_per_spin(1.0) == pytest.approx(-4.0 / np.pi, abs=1e-15)


def test_exact_energy_off_critical_against_exact_diagonalisation():
    """Gapped chain (h = 3): a 12-spin ring has the infinite-chain energy
    density up to exponentially small finite-size corrections."""
    from scipy.sparse.linalg import eigsh

    hz, n = 3.0, 12
    h = _dense_ising_ring(n, hz)
    e0 = eigsh(h, k=1, which="SA")[0][0] / n
    assert O.exact_energy_per_spin(hz) == pytest.approx(e0, abs=3e-7)


@pytest.mark.parametrize("theta,hz", [(0.0, 1.0), (np.pi / 4, 1.0), (0.3, 0.5), (1.1, 2.0)])
def test_product_state_mera_energy_closed_form(theta, hz):
    """A bond-dimension-1 MERA is a product state: w of the bottom layer maps
    the coarse site to phi (x) phi with phi = (cos t, sin t) per spin, every
    other tensor is 1 (or the identity disentangler).  For such a state
    <Z> = cos 2t and <X> = sin 2t on every spin, so the energy per spin of
    H = -sum X X - h sum Z is -sin^2(2t) - h cos(2t).  This runs the whole
    oracle pipeline -- rho* of the SI layer, descent through chi_t = 1, the
    blocked 3-site density, the shift and the per-spin factor -- against a
    closed form."""
    phi2 = np.array([np.cos(theta), np.sin(theta)])
    phi = np.kron(phi2, phi2)                               # blocked site: two spins
    w1 = np.einsum("a,b->ab", phi, phi).reshape(4, 4, 1)
    u1 = np.eye(16).reshape(4, 4, 4, 4)
    one_u, one_w = np.ones((1, 1, 1, 1)), np.ones((1, 1, 1))
    layers = [(u1, w1), (one_u, one_w), (one_u, one_w)]
    h1, shift = O.ising_h1(hz)
    e = O.energy_per_spin(layers, h1, shift, O.identity_density(1), n_pow=3)
    want = -np.sin(2 * theta) ** 2 - hz * np.cos(2 * theta)
    assert e == pytest.approx(want, abs=1e-13)
    assert e >= O.exact_energy_per_spin(hz) - 1e-13      # variational


# --------------------------------------------------------------------------
# Superoperators: invariants.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("chi_b,chi_t", [(2, 2), (3, 3), (2, 3), (4, 3)])
def test_ascend_identity_is_identity(chi_b, chi_t):
    rng = _rng(1)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    eye_b = np.eye(chi_b ** 3).reshape((chi_b,) * 6)
    a = O.ascend(eye_b, u, w)
    assert np.abs(_mat(a) - np.eye(chi_t ** 3)).max() < 1e-13
    for case in ("even", "odd"):
        assert np.abs(_mat(O.ascend_case(eye_b, u, w, case)) - np.eye(chi_t ** 3)).max() < 1e-13


@pytest.mark.parametrize("chi_b,chi_t", [(2, 2), (3, 3), (2, 3)])
def test_duality_ascend_descend(chi_b, chi_t):
    rng = _rng(2)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b, symmetric=False)
    rho = I.random_operator(rng, chi_t, symmetric=False)
    for case in ("even", "odd"):
        lhs = np.sum(O.ascend_case(h, u, w, case) * rho)
        rhs = np.sum(h * O.descend_case(rho, u, w, case))
        assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


@pytest.mark.parametrize("chi", [2, 3])
def test_descend_preserves_trace_and_positivity(chi):
    rng = _rng(3)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    rho = I.random_density(rng, chi)
    d = _mat(O.descend(rho, u, w))
    assert np.trace(d) == pytest.approx(1.0, abs=1e-14)
    assert np.abs(d - d.T).max() < 1e-14
    assert np.linalg.eigvalsh(d).min() > -1e-14


def test_mirror_symmetry_even_odd():
    """Reflecting the lattice maps the even causal-cone position to the odd one."""
    rng = _rng(4)
    chi = 3
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h = I.random_operator(rng, chi, symmetric=False)
    um = np.transpose(u, (1, 0, 3, 2))
    wm = np.transpose(w, (1, 0, 2))
    rev = (2, 1, 0, 5, 4, 3)
    lhs = O.ascend_case(h, u, w, "odd")
    rhs = np.transpose(O.ascend_case(np.transpose(h, rev), um, wm, "even"), rev)
    assert np.abs(lhs - rhs).max() < 1e-13


# --------------------------------------------------------------------------
# Dense brute force on a 6-site periodic chain.
# --------------------------------------------------------------------------
def _layer_matrix(u, w):
    """M = (u_12 u_34 u_50)(w_01 w_23 w_45): fine 6-site space <- coarse 3 sites."""
    chi_b, chi_t = w.shape[0], w.shape[2]
    # U[f0..f5, m0..m5] with disentanglers on fine pairs (1,2), (3,4), (5,0)
    U = np.einsum("bcBC,deDE,faFA->abcdefABCDEF", u, u, u)
    W = np.einsum("ABx,CDy,EFz->ABCDEFxyz", w, w, w)
    M = np.tensordot(U, W, axes=([6, 7, 8, 9, 10, 11], [0, 1, 2, 3, 4, 5]))
    return M.reshape(chi_b ** 6, chi_t ** 3)


@pytest.mark.parametrize("chi_b,chi_t", [(2, 2), (2, 3)])
def test_brute_force_six_site_ring(chi_b, chi_t):
    rng = _rng(5)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    M = _layer_matrix(u, w)
    assert np.abs(M.T @ M - np.eye(chi_t ** 3)).max() < 1e-13
    h = I.random_operator(rng, chi_b, symmetric=False)
    hm = _mat(h)
    for case, sites, coarse_order in (("even", [0, 1, 2], (2, 0, 1)), ("odd", [1, 2, 3], (0, 1, 2))):
        dense = M.T @ _embed(hm, sites, 6, chi_b) @ M
        t = dense.reshape((chi_t,) * 6)
        perm = list(coarse_order) + [3 + c for c in coarse_order]
        want = np.transpose(t, perm)
        got = O.ascend_case(h, u, w, case)
        assert np.abs(got - want).max() < 1e-13, case
        # descending: the 3 fine sites' reduced density of M rho M^T
        rho = I.random_operator(rng, chi_t, symmetric=False)
        inv = np.argsort(perm)
        rho_nat = np.transpose(rho, inv).reshape(chi_t ** 3, chi_t ** 3)
        fine = (M @ rho_nat @ M.T).reshape((chi_b,) * 12)
        rest = [s for s in range(6) if s not in sites]
        # partial trace over the other three fine sites
        letters = "abcdefghijkl"
        ket = list(letters[:6])
        bra = list(letters[6:])
        for s in rest:
            bra[s] = ket[s]
        spec = "".join(ket + bra) + "->" + "".join(ket[s] for s in sites) + "".join(bra[s] for s in sites)
        want_d = np.einsum(spec, fine)
        got_d = O.descend_case(rho, u, w, case)
        assert np.abs(got_d - want_d).max() < 1e-13, case


def test_ttn_special_case_identity_disentanglers():
    """u = 1 turns the MERA layer into a binary-tree layer (Fig. 1a)."""
    rng = _rng(6)
    chi_b, chi_t = 2, 3
    w = I.random_w(rng, chi_b, chi_t)
    u = np.einsum("am,bn->abmn", np.eye(chi_b), np.eye(chi_b))
    h = I.random_operator(rng, chi_b, symmetric=False)
    wm = w.reshape(chi_b ** 2, chi_t)
    w2 = np.kron(wm, wm)
    x = w2.T @ np.kron(_mat(h), np.eye(chi_b)) @ w2
    want_even = np.kron(np.eye(chi_t), x).reshape((chi_t,) * 6)
    assert np.abs(O.ascend_case(h, u, w, "even") - want_even).max() < 1e-13
    # odd position: h on the right leg under the first isometry and both
    # legs under the second one; the third coarse site sees the identity
    xo = w2.T @ np.kron(np.eye(chi_b), _mat(h)) @ w2
    want_odd = np.kron(xo, np.eye(chi_t)).reshape((chi_t,) * 6)
    assert np.abs(O.ascend_case(h, u, w, "odd") - want_odd).max() < 1e-13


# --------------------------------------------------------------------------
# Environments are the energy gradient; the paper's contribution counts.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("chi_b,chi_t", [(2, 2), (3, 2), (2, 3)])
def test_environments_are_half_the_gradient(chi_b, chi_t):
    rng = _rng(7)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b)
    rho = I.random_operator(rng, chi_t)
    gw = O.env_w(h, rho, u, w)
    gu = O.env_u(h, rho, u, w)
    eps = 1e-5
    xw = rng.standard_normal(w.shape)
    xu = rng.standard_normal(u.shape)
    fd_w = (O.energy(h, rho, u, w + eps * xw) - O.energy(h, rho, u, w - eps * xw)) / (2 * eps)
    fd_u = (O.energy(h, rho, u + eps * xu, w) - O.energy(h, rho, u - eps * xu, w)) / (2 * eps)
    assert fd_w == pytest.approx(2 * np.sum(gw * xw), rel=1e-8, abs=1e-10)
    assert fd_u == pytest.approx(2 * np.sum(gu * xu), rel=1e-8, abs=1e-10)


def test_environment_contraction_closes_to_energy():
    """Each hole, closed again with the removed tensor, gives E_case; so
    <Gamma_w, w> = 3 E and <Gamma_u, u> = 2 E (6 and 4 terms, halved)."""
    gold = json.load(open(GOLDEN))["env_contributions"]
    rng = _rng(8)
    chi = 2
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h = I.random_operator(rng, chi)
    rho = I.random_density(rng, chi)
    e = O.energy(h, rho, u, w)
    assert np.sum(O.env_w(h, rho, u, w) * w) == pytest.approx(gold["w"] / 2 * e, rel=1e-12)
    assert np.sum(O.env_u(h, rho, u, w) * u) == pytest.approx(gold["u"] / 2 * e, rel=1e-12)


# --------------------------------------------------------------------------
# Update (Fig. 5).
# --------------------------------------------------------------------------
def test_polar_update_closed_forms():
    # env = R diag(3, 2): -U V^T = -R
    th = 0.3
    r = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    env = (r @ np.diag([3.0, 2.0])).reshape(2, 1, 2)
    x = O.polar_update(env, 2).reshape(2, 2)
    assert np.abs(x + r).max() < 1e-15
    # rectangular: rows = lower legs, columns = upper leg
    env = np.array([[2.0, 0.0], [0.0, 0.0], [0.0, 5.0], [0.0, 0.0]]).reshape(2, 2, 2)
    x = O.polar_update(env, 2).reshape(4, 2)
    want = -np.array([[1.0, 0.0], [0.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    assert np.abs(x - want).max() < 1e-15


@pytest.mark.parametrize("chi_b,chi_t", [(2, 2), (3, 2)])
def test_update_fixed_by_minus_identity_hamiltonian(chi_b, chi_t):
    """With h = -1 every isometric tensor is optimal: the update returns it."""
    rng = _rng(9)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = -np.eye(chi_b ** 3).reshape((chi_b,) * 6)
    rho = I.random_density(rng, chi_t)
    assert np.abs(O.update_u(h, rho, u, w) - u).max() < 1e-12
    assert np.abs(O.update_w(h, rho, u, w) - w).max() < 1e-12


def test_updates_satisfy_constraints():
    rng = _rng(10)
    chi_b, chi_t = 3, 2
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b)
    rho = I.random_density(rng, chi_t)
    un = O.update_u(h, rho, u, w).reshape(chi_b ** 2, chi_b ** 2)
    wn = O.update_w(h, rho, u, w).reshape(chi_b ** 2, chi_t)
    assert np.abs(un.T @ un - np.eye(chi_b ** 2)).max() < 1e-13   # Eq. (unitarity)
    assert np.abs(wn.T @ wn - np.eye(chi_t)).max() < 1e-13       # Eq. (iso)


# --------------------------------------------------------------------------
# Fixed point and scaling dimensions.
# --------------------------------------------------------------------------
def test_fixed_point_is_a_fixed_point():
    rng = _rng(11)
    chi = 2
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    rho, resid = O.fixed_point_rho(u, w, O.identity_density(chi), 300)
    assert resid < 1e-12
    again = O.symmetrize_normalize(O.descend(rho, u, w))
    assert np.abs(again - rho).max() < 1e-12
    # dominant eigenvalue of D_SI is 1: the unnormalised map preserves the trace
    assert np.trace(_mat(O.descend(rho, u, w))) == pytest.approx(1.0, abs=1e-14)


def test_scaling_dimension_of_identity_is_zero():
    gold = json.load(open(GOLDEN))["ising_cft_scaling_dims"]["value"]
    rng = _rng(12)
    u, w = I.random_u(rng, 2), I.random_w(rng, 2, 2)
    dims = O.scaling_dimensions(u, w, 6)
    assert dims[0] == pytest.approx(gold[0], abs=1e-12)
    assert np.all(dims >= -1e-12)


# --------------------------------------------------------------------------
# Physics: the sweep lowers the energy towards -4/pi and stays above it.
# --------------------------------------------------------------------------
def test_sweeps_lower_energy_and_respect_variational_bound():
    layers = I.init_mera(0, 4)
    h1, shift = O.ising_h1(1.0)
    layers, rho, es = O.run(layers, 1.0, n_sweeps=40, n_pow=20)
    e_true = O.energy_per_spin(layers, h1, shift, rho, n_pow=200)
    exact = O.exact_energy_per_spin(1.0)
    assert e_true >= exact
    assert es[-1] < es[0]
    assert np.all(np.diff(es[5:]) < 1e-9)
    assert (e_true - exact) / abs(exact) < 0.25
    for u, w in layers:
        um = u.reshape(u.shape[0] ** 2, -1)
        wm = w.reshape(w.shape[0] ** 2, -1)
        assert np.abs(um.T @ um - np.eye(um.shape[1])).max() < 1e-12
        assert np.abs(wm.T @ wm - np.eye(wm.shape[1])).max() < 1e-12


# ---------------------------------------------------------------------------
# Riemannian (Stiefel) gradient step: pinned by properties, not a retyping.
# ---------------------------------------------------------------------------
def test_stiefel_step_stays_on_the_manifold_and_fixes_zero_steps():
    rng = np.random.default_rng(41)
    x = I.random_isometry(rng, 9, 4)
    g = rng.standard_normal((9, 4))
    y = O.stiefel_step(x, g, 0.3)
    assert np.abs(y.T @ y - np.eye(4)).max() < 1e-13
    assert np.abs(O.stiefel_step(x, g, 0.0) - x).max() < 1e-13


def test_stiefel_direction_is_tangent():
    """The step direction (y(-eta) - y(eta)) / (2 eta) -> the projected
    gradient r as eta -> 0, and r must lie in the tangent space:
    x^T r + r^T x = 0."""
    rng = np.random.default_rng(42)
    x = I.random_isometry(rng, 16, 5)
    g = rng.standard_normal((16, 5))
    eta = 1e-5
    r = (O.stiefel_step(x, g, -eta) - O.stiefel_step(x, g, eta)) / (2 * eta)
    assert np.abs(x.T @ r + r.T @ x).max() < 1e-8
    # and it is the gradient's tangent part: <g - r, t> = 0 for tangent t
    k = rng.standard_normal((5, 5))
    t = x @ (k - k.T) + (np.eye(16) - x @ x.T) @ rng.standard_normal((16, 5))
    assert abs(np.sum((g - r) * t)) < 1e-5 * np.abs(g).sum()


def test_stiefel_step_descends_the_mera_energy_at_the_predicted_rate():
    """f(w) = tr(A(h) rho) with symmetric h, rho has gradient 2 Gamma_w; a step
    of size eta along the Riemannian gradient changes f by -eta |r|^2 to
    first order (central difference), r the projected gradient."""
    rng = np.random.default_rng(43)
    chi = 2
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h, rho = I.random_operator(rng, chi), I.random_density(rng, chi)
    x = w.reshape(chi * chi, chi)
    g = (2.0 * O.env_w(h, rho, u, w)).reshape(chi * chi, chi)
    a = x.T @ g
    r = g - x @ (0.5 * (a + a.T))
    eta = 1e-5

    def f(xx):
        return O.energy(h, rho, u, xx.reshape(w.shape))

    slope = (f(O.stiefel_step(x, g, eta)) - f(O.stiefel_step(x, g, -eta))) / (2 * eta)
    assert slope == pytest.approx(-np.sum(r * r), rel=1e-6)


def test_riemannian_sweeps_lower_the_energy():
    """Small Riemannian steps: the energy per spin decreases sweep by sweep
    (after the first few, while rho* settles) and stays above -4/pi."""
    h1, shift = O.ising_h1(1.0)
    layers = I.init_mera(0, 2)
    rho = O.identity_density(2)
    es = []
    for _ in range(12):
        layers, rho, e = O.sweep(layers, h1, shift, rho, 20, eta=0.1)
        es.append(e)
    assert all(b <= a + 1e-12 for a, b in zip(es[4:], es[5:]))
    assert es[-1] >= -4.0 / np.pi


def test_z2_symmetric_start_is_kept_by_the_sweep():
    """Tensors that commute with the Ising chain's Z2 parity stay so under the
    sweep (the Hamiltonian commutes with prod Z, so every environment is
    block diagonal in the charges): the odd-charge blocks stay zero."""
    chi = 4
    layers = I.init_mera(1, chi, z2=True)
    h1, shift = O.ising_h1(1.0)
    layers, rho, _ = O.run(layers, 1.0, 3, 20)
    pb = I.parity_labels(4, physical=True)
    for u, w in layers:
        cb, ct = w.shape[0], w.shape[2]
        pt = I.parity_labels(ct)
        pair = (pb[:, None] ^ pb[None, :]).reshape(-1)
        W = w.reshape(cb * cb, ct)
        U = u.reshape(cb * cb, cb * cb)
        assert np.abs(W[pair[:, None] != pt[None, :]]).max() < 1e-12
        assert np.abs(U[pair[:, None] != pair[None, :]]).max() < 1e-12
        pb = pt


# --------------------------------------------------------------------------
# Physics near convergence: a chi = 4 MERA optimised by the oracle alone
# (tests/golden/make_chi4_z2_mera.py: parity-symmetric start, 8900 sweeps)
# reproduces the Ising CFT read off the scale-invariant ascending map
# (Sec. II B: Delta_sigma = 1/8, Delta_eps = 1, the sigma descendants at
# 9/8) and the exact energy density -4/pi (Sec. III A).  The stored state
# only saves the CPU time of the first sweeps; the test sweeps on from it.
# --------------------------------------------------------------------------
CHI4 = os.path.join(os.path.dirname(__file__), "golden", "mera_chi4_z2.json")


def test_converged_chi4_mera_reproduces_the_ising_cft():
    gold = json.load(open(GOLDEN))
    doc = json.load(open(CHI4))
    layers = [(np.array(x["u"]).reshape((x["chi_b"],) * 4),
               np.array(x["w"]).reshape(x["chi_b"], x["chi_b"], x["chi_t"])) for x in doc["layers"]]
    rho = np.array(doc["rho_star"]).reshape((doc["chi"],) * 6)
    h1, shift = O.ising_h1(1.0)
    exact = gold["e_exact_per_spin"]["value"]
    e_start = O.energy_per_spin(layers, h1, shift, rho, 100)
    assert e_start == pytest.approx(doc["energy_per_spin"], abs=1e-12)
    for _ in range(100):
        layers, rho, _ = O.sweep(layers, h1, shift, rho, 20)
    e = O.energy_per_spin(layers, h1, shift, rho, 100)
    # 100 more sweeps keep lowering the energy, which stays above -4/pi
    assert exact < e < e_start
    assert (e - exact) / abs(exact) < 6.5e-6
    for u, w in layers:
        um, wm = u.reshape(u.shape[0] ** 2, -1), w.reshape(w.shape[0] ** 2, -1)
        assert np.abs(um.T @ um - np.eye(um.shape[1])).max() < 1e-12
        assert np.abs(wm.T @ wm - np.eye(wm.shape[1])).max() < 1e-12
    dims = O.scaling_dimensions(*layers[-1], 6)
    d_id, d_sigma, d_eps = gold["ising_cft_scaling_dims"]["value"]
    assert dims[0] == pytest.approx(d_id, abs=1e-9)
    assert abs(dims[1] - d_sigma) < 0.003
    assert abs(dims[2] - d_eps) < 0.002
    assert np.all(np.abs(dims[3:5] - gold["sigma_descendant"]["value"]) < 0.005)
    assert dims[5] > 1.5      # then a gap: no other primary or descendant below 3/2


# --------------------------------------------------------------------------
# Entry-wise helpers for full-size checks: ascend_rows, descend_rows,
# env_w_cols and env_u_rows compute parts of the (pinned) maps with some legs
# held fixed.
# They must equal the corresponding parts of the whole maps.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("chi_b,chi_t", [(3, 3), (2, 3), (4, 5), (3, 2)])
def test_row_and_column_helpers_equal_the_whole_maps(chi_b, chi_t):
    rng = _rng(100 + 10 * chi_b + chi_t)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b, symmetric=False)
    rho = I.random_operator(rng, chi_t, symmetric=False)
    a, gw, gu = O.ascend(h, u, w), O.env_w(h, rho, u, w), O.env_u(h, rho, u, w)
    rows3 = [(0, 0, 0), (chi_t - 1, 0, chi_t - 1)]
    for k, (p, q, r) in enumerate(rows3):
        assert np.abs(O.ascend_rows(h, u, w, rows3)[k] - a[p, q, r]).max() < 1e-12
    cols = [0, chi_t - 1]
    for k, c in enumerate(O.env_w_cols(h, rho, u, w, cols)):
        assert np.abs(c - gw[:, :, cols[k]]).max() < 1e-12
    rows2 = [(0, 0), (chi_b - 1, 0), (1, chi_b - 1)]
    for k, r in enumerate(O.env_u_rows(h, rho, u, w, rows2)):
        assert np.abs(r - gu[rows2[k]]).max() < 1e-12
    d = O.descend(rho, u, w)
    rows_d = [(0, 0, 0), (chi_b - 1, 0, 1), (1, chi_b - 1, chi_b - 1)]
    for k, r in enumerate(O.descend_rows(rho, u, w, rows_d)):
        assert np.abs(r - d[rows_d[k]]).max() < 1e-12
