"""GPU parity: every C-ABI map against the FP64 oracle on seeded inputs.

FP64 mode: |gpu - oracle| <= 1e-10 * max|oracle| element by element (the
relative-to-max-norm reading of "within 1e-10 relative").  Sizes span
several GEMM tiles with ragged tails (chi = 5: 625-row operands) and uneven
layer dimensions (chi_b != chi_t) as in the first two MERA layers.
"""
import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10
# (1, 1) and (2, 1): the degenerate bond dimensions (every leg trivial, a
# one-state coarse leg); the rest span several tiles with ragged edges.
# the last five are layers of the bond-dimension ladder chi = 6, 10, 14, whose
# chi^2 is not a multiple of 8 (padded operand rows)
DIMS = [(1, 1), (2, 1), (2, 2), (3, 3), (4, 4), (5, 5), (2, 3), (4, 6), (4, 16), (3, 8), (8, 8),
        (6, 6), (4, 10), (10, 10), (4, 14), (14, 14)]


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _err(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _inputs(chi_b, chi_t, seed=0):
    rng = np.random.default_rng(seed)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b)
    rho = I.random_density(rng, chi_t)
    return u, w, h, rho


@pytest.mark.parametrize("chi_b,chi_t", DIMS)
def test_ascend_descend_f64(chi_b, chi_t):
    u, w, h, rho = _inputs(chi_b, chi_t, 1)
    hn = I.random_operator(np.random.default_rng(7), chi_b, symmetric=False)
    out = torch.empty(chi_t ** 6, dtype=torch.float64, device="cuda")
    m.mera_ascend(_cuda(hn).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1), chi_b, chi_t, out)
    assert _err(out.cpu().numpy().reshape((chi_t,) * 6), O.ascend(hn, u, w)) < TOL_F64
    out_d = torch.empty(chi_b ** 6, dtype=torch.float64, device="cuda")
    m.mera_descend(_cuda(rho).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1), chi_b, chi_t, out_d)
    assert _err(out_d.cpu().numpy().reshape((chi_b,) * 6), O.descend(rho, u, w)) < TOL_F64


@pytest.mark.parametrize("chi_b,chi_t", DIMS)
def test_environments_f64(chi_b, chi_t):
    u, w, h, rho = _inputs(chi_b, chi_t, 2)
    gu = torch.empty(chi_b ** 4, dtype=torch.float64, device="cuda")
    gw = torch.empty(chi_b ** 2 * chi_t, dtype=torch.float64, device="cuda")
    args = (_cuda(h).reshape(-1), _cuda(rho).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1), chi_b, chi_t)
    m.mera_env_u(*args, gu)
    m.mera_env_w(*args, gw)
    assert _err(gu.cpu().numpy().reshape(u.shape), O.env_u(h, rho, u, w)) < TOL_F64
    assert _err(gw.cpu().numpy().reshape(w.shape), O.env_w(h, rho, u, w)) < TOL_F64


@pytest.mark.parametrize("chi_b,chi_t", [(3, 3), (4, 6), (5, 5)])
def test_energy_f64(chi_b, chi_t):
    u, w, h, rho = _inputs(chi_b, chi_t, 3)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    m.mera_energy(_cuda(h).reshape(-1), _cuda(rho).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1),
                  chi_b, chi_t, e)
    want = O.energy(h, rho, u, w)
    assert abs(e.item() - want) <= TOL_F64 * max(1.0, abs(want))


@pytest.mark.parametrize("chi", [2, 4, 5])
def test_fixed_point_f64(chi):
    u, w, _, _ = _inputs(chi, chi, 4)
    rho0 = O.identity_density(chi)
    want, resid_want = O.fixed_point_rho(u, w, rho0, 20)
    rho = _cuda(rho0).reshape(-1).clone()
    resid = torch.empty(1, dtype=torch.float64, device="cuda")
    m.mera_fixed_point_rho(_cuda(u).reshape(-1), _cuda(w).reshape(-1), chi, rho, 20, resid)
    assert _err(rho.cpu().numpy().reshape(want.shape), want) < TOL_F64
    assert resid.item() == pytest.approx(resid_want, rel=1e-6, abs=1e-14)


def test_fixed_point_zero_iterations_is_identity_map():
    chi = 3
    u, w, _, rho0 = _inputs(chi, chi, 5)
    rho = _cuda(rho0).reshape(-1).clone()
    resid = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    m.mera_fixed_point_rho(_cuda(u).reshape(-1), _cuda(w).reshape(-1), chi, rho, 0, resid)
    assert np.array_equal(rho.cpu().numpy(), rho0.reshape(-1))
    assert resid.item() == 0.0


@pytest.mark.parametrize("mm,nn", [(16, 16), (16, 4), (64, 64), (256, 256), (256, 16), (100, 37)])
def test_polar_update_f64(mm, nn):
    rng = np.random.default_rng(mm * 1000 + nn)
    env = rng.standard_normal((mm, nn))
    out = torch.empty(mm * nn, dtype=torch.float64, device="cuda")
    m.mera_polar_update(_cuda(env).reshape(-1), mm, nn, out)
    want = O.polar_update(env.reshape(mm, 1, nn), 1).reshape(mm, nn)
    got = out.cpu().numpy().reshape(mm, nn)
    assert np.abs(got - want).max() < 1e-10
    assert np.abs(got.T @ got - np.eye(nn)).max() < 1e-12


def test_polar_update_converges_over_thirty_decades():
    """env is a signed permutation of diag(s), s from 1 down to 1e-30, so
    its polar factor is the signed permutation itself.  The quintic step
    grows each singular value 2.5-fold until it nears 1 (81 steps from
    1e-30), within the default 100; the cubic (3 x - x^3) / 2 grows it
    1.5-fold and would still be at 1e-9 after 100 steps."""
    mm, nn = 24, 12
    rng = np.random.default_rng(5)
    s = 10.0 ** -np.linspace(0.0, 30.0, nn)
    rows, cols = rng.permutation(mm)[:nn], rng.permutation(nn)
    signs = rng.choice([-1.0, 1.0], nn)
    env = np.zeros((mm, nn))
    env[rows, cols] = signs * s
    want = np.zeros((mm, nn))
    want[rows, cols] = -signs  # the update is -polar(env)
    out = torch.empty(mm * nn, dtype=torch.float64, device="cuda")
    m.mera_device_status(clear=True)
    m.mera_polar_update(_cuda(env).reshape(-1), mm, nn, out)
    got = out.cpu().numpy().reshape(mm, nn)
    assert m.mera_device_status(clear=True) == 0
    assert np.abs(got - want).max() < 1e-14


def test_polar_reports_nonconvergence_for_rank_deficient_input():
    """The polar update is asynchronous: non-convergence within max_iter
    steps is reported through the device status word, not a return code."""
    mm, nn = 16, 4
    env = np.zeros((mm, nn))
    env[0, 0] = 1.0  # rank 1: no unique polar factor
    out = torch.empty(mm * nn, dtype=torch.float64, device="cuda")
    m.mera_device_status(clear=True)
    m.mera_polar_update(_cuda(env).reshape(-1), mm, nn, out, max_iter=30)
    torch.cuda.synchronize()
    assert m.mera_device_status(clear=True) == 1 << 4  # MERA_ENOTCONV
    # a converging update leaves the word clear
    rng = np.random.default_rng(3)
    m.mera_polar_update(_cuda(rng.standard_normal((mm, nn))).reshape(-1), mm, nn, out)
    assert m.mera_device_status(clear=True) == 0


def test_sweep_returns_before_its_stream_completes():
    """Every compute call is asynchronous on its stream, the polar updates
    of the direct sweep included: at chi = 16 a sweep runs ~60 ms on the GPU,
    and the call returns while its stream is still busy."""
    chi = 16
    layers = I.init_mera(0, chi)
    h1, shift = O.ising_h1(1.0)
    st = m.MeraState([_cuda(u).reshape(-1).clone() for u, _ in layers], [_cuda(w).clone() for _, w in layers],
                     _cuda(O.identity_density(chi)).reshape(-1).clone())
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    h1d = _cuda(h1).reshape(-1)
    stream = torch.cuda.Stream()
    ws = m.workspace(m.mera_sweep_workspace_size(st.chi_b, st.chi_t, m.PREC_BF16X3))
    m.mera_sweep(st, h1d, shift, 20, e, prec=m.PREC_BF16X3, ws=ws, stream=stream)  # plans, recordings
    torch.cuda.synchronize()
    busy = []
    for _ in range(3):
        m.mera_sweep(st, h1d, shift, 20, e, prec=m.PREC_BF16X3, ws=ws, stream=stream)
        busy.append(not stream.query())
        stream.synchronize()
    assert all(busy)
    assert m.mera_device_status(clear=True) == 0


def test_argument_errors_do_not_launch():
    chi = 3
    u, w, h, _ = _inputs(chi, chi, 6)
    out = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.MeraError) as ei:
        m.mera_ascend(_cuda(h).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1), chi, chi, out, ws=small)
    assert ei.value.status == 2  # MERA_ENOMEM
    with pytest.raises(m.MeraError):
        m.mera_ascend(_cuda(h).reshape(-1), _cuda(u).reshape(-1), _cuda(w).reshape(-1), chi, chi, out, prec=9)


def test_sweeps_match_oracle_chi4():
    chi, n_sweeps = 4, 4
    layers = I.init_mera(0, chi)
    h1, shift = O.ising_h1(1.0)
    ol, orho, oes = O.run([(u.copy(), w.copy()) for u, w in layers], 1.0, n_sweeps, 20)
    us = [_cuda(u).reshape(-1).clone() for u, _ in layers]
    ws = [_cuda(w).clone() for _, w in layers]
    rho = _cuda(O.identity_density(chi)).reshape(-1).clone()
    st = m.MeraState(us, ws, rho)
    st.chi_b = [w.shape[0] for _, w in layers]
    st.chi_t = [w.shape[2] for _, w in layers]
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    h1d = _cuda(h1).reshape(-1)
    es = []
    for _ in range(n_sweeps):
        m.mera_sweep(st, h1d, shift, 20, e)
        es.append(e.item())
    np.testing.assert_allclose(es, oes, rtol=1e-10, atol=0)
    for (ou, ow), u, w in zip(ol, us, ws):
        assert np.abs(u.cpu().numpy().reshape(ou.shape) - ou).max() < 1e-9
        assert np.abs(w.cpu().numpy().reshape(ow.shape) - ow).max() < 1e-9
    assert _err(rho.cpu().numpy().reshape(orho.shape), orho) < 1e-9


@pytest.mark.parametrize("mm,nn", [(16, 16), (64, 8), (256, 16), (300, 7)])
def test_stiefel_step_f64(mm, nn):
    rng = np.random.default_rng(mm + 7 * nn)
    x = I.random_isometry(rng, mm, nn)
    g = rng.standard_normal((mm, nn))
    out = torch.empty(mm * nn, dtype=torch.float64, device="cuda")
    m.mera_stiefel_step(_cuda(x).reshape(-1), _cuda(g).reshape(-1), mm, nn, 0.2, out)
    want = O.stiefel_step(x, g, 0.2)
    got = out.cpu().numpy().reshape(mm, nn)
    assert np.abs(got - want).max() < 1e-10
    # in place (out aliases X) gives the same
    xd = _cuda(x).reshape(-1).clone()
    m.mera_stiefel_step(xd, _cuda(g).reshape(-1), mm, nn, 0.2, xd)
    assert np.abs(xd.cpu().numpy().reshape(mm, nn) - want).max() < 1e-10


def test_riemannian_sweeps_match_oracle_chi3():
    chi, n_sweeps, eta = 3, 3, 0.1
    layers = I.init_mera(2, chi)
    h1, shift = O.ising_h1(1.0)
    ol = [(u.copy(), w.copy()) for u, w in layers]
    orho = O.identity_density(chi)
    oes = []
    for _ in range(n_sweeps):
        ol, orho, e_ = O.sweep(ol, h1, shift, orho, 20, eta=eta)
        oes.append(e_)
    us = [_cuda(u).reshape(-1).clone() for u, _ in layers]
    ws = [_cuda(w).clone() for _, w in layers]
    rho = _cuda(O.identity_density(chi)).reshape(-1).clone()
    st = m.MeraState(us, ws, rho)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    h1d = _cuda(h1).reshape(-1)
    es = []
    for _ in range(n_sweeps):
        m.mera_sweep_riemannian(st, h1d, shift, 20, eta, e)
        es.append(e.item())
    np.testing.assert_allclose(es, oes, rtol=1e-10, atol=0)
    for (ou, ow), u, w in zip(ol, us, ws):
        assert np.abs(u.cpu().numpy().reshape(ou.shape) - ou).max() < 1e-9
        assert np.abs(w.cpu().numpy().reshape(ow.shape) - ow).max() < 1e-9


# --------------------------------------------------------------------------
# Full size (chi = 16, the benchmarked workload): sampled rows and properties.
# --------------------------------------------------------------------------
def test_ascend_chi16_sampled_rows_and_identity():
    chi = 16
    u, w, h, rho = _inputs(chi, chi, 8)
    ud, wd = _cuda(u).reshape(-1), _cuda(w).reshape(-1)
    out = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")
    m.mera_ascend(_cuda(h).reshape(-1), ud, wd, chi, chi, out)
    got = out.cpu().numpy().reshape((chi,) * 6)
    rows = [(0, 0, 0), (3, 15, 7), (15, 1, 9)]
    want = O.ascend_rows(h, u, w, rows)
    for k, (p, q, r) in enumerate(rows):
        assert _err(got[p, q, r], want[k]) < TOL_F64
    # A(1) = 1 (Eq. iso / unitarity) at full size
    eye = torch.eye(chi ** 3, dtype=torch.float64, device="cuda").reshape(-1)
    m.mera_ascend(eye, ud, wd, chi, chi, out)
    a1 = out.reshape(chi ** 3, chi ** 3)
    assert (a1 - torch.eye(chi ** 3, dtype=torch.float64, device="cuda")).abs().max().item() < 1e-12


# --------------------------------------------------------------------------
# Scaling dimensions (Sec. II B, Fig. 7): Arnoldi with the GPU ascend as
# matvec against the oracle's eigen-solve of the same map.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("chi", [2, 3, 4])
def test_scaling_dimensions_match_oracle(chi):
    from paper_1906_12030_gb300 import scaling

    rng = np.random.default_rng(40 + chi)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    # Ask both for 10 eigenvalues and compare the leading 4: near the cut-off
    # of a random map |lambda| is nearly degenerate and either solver may
    # keep a different member of a close pair.
    got = scaling.scaling_dimensions(_cuda(u), _cuda(w), chi, k=10)[:4]
    want = O.scaling_dimensions(u, w, 10)[:4]
    assert got[0] == pytest.approx(0.0, abs=1e-9)  # A(1) = 1
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-8)


def test_scaling_dimensions_of_the_optimised_chi4_mera():
    """The stored chi = 4 MERA that the oracle optimised (tests/golden): the
    GPU Arnoldi gives the oracle's leading dimensions of its scale-invariant
    layer and, with them, the Ising CFT values (Sec. II B): 0, 1/8, 1 and the
    two sigma descendants at 9/8, before a gap."""
    import json
    import os

    from paper_1906_12030_gb300 import scaling

    golden = os.path.join(os.path.dirname(__file__), "golden")
    doc = json.load(open(os.path.join(golden, "mera_chi4_z2.json")))
    cft = json.load(open(os.path.join(golden, "paper_values.json")))
    top = doc["layers"][-1]
    chi = top["chi_t"]
    u = np.array(top["u"]).reshape((chi,) * 4)
    w = np.array(top["w"]).reshape(chi, chi, chi)
    got = scaling.scaling_dimensions(_cuda(u), _cuda(w), chi, k=8)[:6]
    want = O.scaling_dimensions(u, w, 8)[:6]
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-8)
    d_id, d_sigma, d_eps = cft["ising_cft_scaling_dims"]["value"]
    assert got[0] == pytest.approx(d_id, abs=1e-9)
    assert abs(got[1] - d_sigma) < 0.003 and abs(got[2] - d_eps) < 0.002
    assert np.all(np.abs(got[3:5] - cft["sigma_descendant"]["value"]) < 0.005) and got[5] > 1.5


def test_fp64_sweeps_replayed_by_the_oracle_from_checkpoints():
    """The plain FP64 GPU run compared with the oracle from its own
    checkpoints: the GPU state after sweeps 1, 2 and 40 of a chi = 8 run is
    copied out, the oracle runs the next sweep from it, and the GPU's next
    sweep matches (energy to 1e-10 relative, u, w and rho* to 1e-9)."""
    chi, last = 8, 41
    checkpoints = {1, 2, 40}
    layers = I.init_mera(0, chi)
    h1, shift = O.ising_h1(1.0)
    st = m.MeraState([_cuda(u).reshape(-1).clone() for u, _ in layers], [_cuda(w).clone() for _, w in layers],
                     _cuda(O.identity_density(chi)).reshape(-1).clone())
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    h1d = _cuda(h1).reshape(-1)
    ws = m.workspace(m.mera_sweep_workspace_size(st.chi_b, st.chi_t, m.PREC_F64))
    shapes = [(u.shape, w.shape) for u, w in layers]
    snap = None
    n_checked = 0
    for k in range(1, last + 1):
        m.mera_sweep(st, h1d, shift, 20, e, ws=ws)
        if snap is not None:  # k = checkpoint + 1: the oracle's sweep from the snapshot
            ol, orho, oe = O.sweep(snap[0], h1, shift, snap[1], 20)
            assert e.item() == pytest.approx(oe, rel=1e-10, abs=0)
            for (ou, ow), u, w in zip(ol, st.us, st.ws):
                assert np.abs(u.cpu().numpy().reshape(ou.shape) - ou).max() < 1e-9
                assert np.abs(w.cpu().numpy().reshape(ow.shape) - ow).max() < 1e-9
            assert np.abs(st.rho_star.cpu().numpy().reshape(orho.shape) - orho).max() < 1e-9
            n_checked += 1
            snap = None
        if k in checkpoints:
            snap = ([(u.cpu().numpy().reshape(su), w.cpu().numpy().reshape(sw))
                     for (su, sw), u, w in zip(shapes, st.us, st.ws)],
                    st.rho_star.cpu().numpy().reshape((chi,) * 6))
    assert n_checked == len(checkpoints)
    assert m.mera_device_status(clear=True) == 0
