"""Differentiation (energy adjoint): hand-written backward of mera_energy
against central finite differences (FP64, step 1e-6) and against the
environments, which are exactly half the energy gradient for symmetric h
and rho (Fig. 4c/d, A1)."""
import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu


def _t(x, grad=False):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda().requires_grad_(grad)


@pytest.mark.parametrize("chi_b,chi_t", [(3, 3), (4, 6), (5, 5)])
def test_energy_gradient_matches_finite_differences(chi_b, chi_t):
    from paper_1906_12030_gb300.autograd import mera_energy

    rng = np.random.default_rng(60 + chi_b)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b, symmetric=False)   # general operators: both hole sides matter
    rho = I.random_operator(rng, chi_t, symmetric=False)
    ht, rt, ut, wt = _t(h, True), _t(rho, True), _t(u, True), _t(w, True)
    e = mera_energy(ht, rt, ut, wt, chi_b, chi_t)
    e.backward()
    assert e.item() == pytest.approx(O.energy(h, rho, u, w), rel=1e-12)
    eps = 1e-6
    for x, grad, name in ((h, ht.grad, "h"), (rho, rt.grad, "rho"), (u, ut.grad, "u"), (w, wt.grad, "w")):
        d = rng.standard_normal(x.shape)
        args = {"h": h, "rho": rho, "u": u, "w": w}
        plus, minus = dict(args), dict(args)
        plus[name] = x + eps * d
        minus[name] = x - eps * d
        fd = (O.energy(plus["h"], plus["rho"], plus["u"], plus["w"])
              - O.energy(minus["h"], minus["rho"], minus["u"], minus["w"])) / (2 * eps)
        an = float((grad.cpu().numpy() * d).sum())
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9), name


def test_symmetric_gradient_is_twice_the_environment():
    from paper_1906_12030_gb300.autograd import mera_energy

    chi = 4
    rng = np.random.default_rng(70)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h, rho = I.random_operator(rng, chi), I.random_density(rng, chi)
    ut, wt = _t(u, True), _t(w, True)
    mera_energy(_t(h), _t(rho), ut, wt, chi, chi).backward()
    np.testing.assert_allclose(ut.grad.cpu().numpy(), 2 * O.env_u(h, rho, u, w), rtol=0, atol=1e-11)
    np.testing.assert_allclose(wt.grad.cpu().numpy(), 2 * O.env_w(h, rho, u, w), rtol=0, atol=1e-11)


def test_operator_transpose():
    d = 3
    x = np.random.default_rng(71).standard_normal((d,) * 6)
    out = torch.empty(d ** 6, dtype=torch.float64, device="cuda")
    m.mera_op_transpose(_t(x).reshape(-1), d, out)
    want = np.transpose(x, (3, 4, 5, 0, 1, 2))
    assert np.array_equal(out.cpu().numpy().reshape(want.shape), want)


# Tolerances of the tensor-core modes (relative to the largest FP64 entry):
# the map parity tests' bounds for each mode (TF32 5e-3, BF16X3 8e-5), and
# twice that for BF16X3, whose u and w gradients sum two environments; the
# fixed-point split mode OZ4 at its map tolerance (1.2e-7), doubled likewise.
_MODE_TOL = {m.PREC_TF32: 5e-3, m.PREC_BF16X3: 1.6e-4, m.PREC_OZ4: 2.4e-7}


def _grads(h, rho, u, w, chi_b, chi_t, prec):
    """Energy and its four gradients through MeraEnergy (forward + backward)."""
    from paper_1906_12030_gb300.autograd import mera_energy

    ts = [_t(x, True) for x in (h, rho, u, w)]
    e = mera_energy(*ts, chi_b, chi_t, prec)
    e.backward()
    return e.item(), [t.grad.cpu().numpy() for t in ts]


def test_adjoint_against_central_differences_chi12():
    """FP64 adjoint at chi = 12 against central differences (step 1e-6) of the
    oracle's energy, one random direction per input; general (non-symmetric)
    h and rho so that the ket-side and bra-side holes both enter."""
    chi = 12
    rng = np.random.default_rng(80)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h = I.random_operator(rng, chi, symmetric=False)
    rho = I.random_operator(rng, chi, symmetric=False)
    e, grads = _grads(h, rho, u, w, chi, chi, m.PREC_F64)
    args = {"h": h, "rho": rho, "u": u, "w": w}
    assert e == pytest.approx(O.energy(h, rho, u, w), rel=1e-10)
    eps = 1e-6
    for (name, x), g in zip(args.items(), grads):
        d = rng.standard_normal(x.shape)
        plus, minus = dict(args), dict(args)
        plus[name], minus[name] = x + eps * d, x - eps * d
        fd = (O.energy(**plus) - O.energy(**minus)) / (2 * eps)
        assert float((g * d).sum()) == pytest.approx(fd, rel=1e-6), name


@pytest.mark.parametrize("chi", [12, 16])
def test_mixed_precision_adjoint_against_fp64(chi):
    """The adjoint with TF32, split-BF16 and fixed-point split contractions
    matches the FP64 adjoint entry by entry within each mode's tolerance."""
    rng = np.random.default_rng(81 + chi)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h = I.random_operator(rng, chi, symmetric=False)
    rho = I.random_operator(rng, chi, symmetric=False)
    e64, g64 = _grads(h, rho, u, w, chi, chi, m.PREC_F64)
    for prec, tol in _MODE_TOL.items():
        e, gs = _grads(h, rho, u, w, chi, chi, prec)
        errs = {name: float(np.abs(g - want).max() / np.abs(want).max())
                for name, g, want in zip(("h", "rho", "u", "w"), gs, g64)}
        print(f"prec={prec} chi={chi} adjoint errors {errs}")
        for name, err in errs.items():
            assert err <= tol, (prec, name, err)


@pytest.mark.parametrize("prec", [m.PREC_TF32, m.PREC_BF16X3])
def test_adjoint_at_chi24_recomputes_and_satisfies_euler_identities(prec):
    """chi = 24, too large for an FP64 comparison: the forward keeps no
    intermediate (only the inputs are saved; the backward recomputes every
    rank-6 contraction), and the gradients obey Euler's identity for the
    homogeneous polynomial E: degree 1 in h and rho, 4 in u (two ket- and two
    bra-side disentanglers per diagram), 6 in w.  h is a rank-16 density and
    rho a full-rank diagonal density: every final pairing (tr(A(h) rho) over
    the positive diagonal, <D(rho), h> with D(rho) near the identity, and the
    environments against u and w) is free of cancellation, so each identity
    holds to the mode's relative map error."""
    from paper_1906_12030_gb300.autograd import mera_energy

    chi = 24
    rng = np.random.default_rng(90)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h = I.random_low_rank_density(rng, chi, 16)
    rho = I.random_diagonal_density(rng, chi)
    ts = [_t(x, True) for x in (h, rho, u, w)]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    e = mera_energy(*ts, chi, chi, prec)
    torch.cuda.synchronize()
    kept = torch.cuda.memory_allocated() - before
    assert kept < 1 << 20, kept          # a chi^6 intermediate would be 1.5 GB
    e.backward()
    ev = e.item()
    assert ev > 0
    degree = {"h": 1, "rho": 1, "u": 4, "w": 6}
    # at K = chi^3 = 13824 the FP32 accumulation dominates: the derived map
    # bound 10 u + K 2^-24 (TF32 5e-3; BF16X3 1.05e-3, measured 5e-4)
    tol = {m.PREC_TF32: 5e-3, m.PREC_BF16X3: 10 * 1.5 * 2.0 ** -16 + chi ** 3 * 2.0 ** -24}[prec]
    for (name, k), x, t in zip(degree.items(), (h, rho, u, w), ts):
        lhs = float(torch.sum(t.grad * t.detach()))
        assert lhs == pytest.approx(k * ev, rel=tol), (name, lhs, k * ev)
