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
