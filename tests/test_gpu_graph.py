"""A sweep recorded once as a CUDA graph and replayed (mera_sweep_graph_create
/ mera_graph_launch) must give exactly what mera_sweep gives on the same
state: the recorded polar updates run the same device-gated Newton-Schulz
steps, only without the host's convergence checks."""
import numpy as np
import pytest

import mera_inputs as I

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu


def _state(seed, chi):
    layers = I.init_mera(seed, chi)
    us = [torch.from_numpy(u).cuda().reshape(-1).contiguous() for u, _ in layers]
    ws = [torch.from_numpy(w).cuda().contiguous() for _, w in layers]
    rho = (torch.eye(chi ** 3, dtype=torch.float64, device="cuda") / chi ** 3).reshape(-1).contiguous()
    return m.MeraState(us, ws, rho), us, ws, rho


@pytest.mark.parametrize("prec,chi", [(m.PREC_F64, 4), (m.PREC_BF16X3, 8), (m.PREC_BF16X3, 16)])
def test_graph_replays_equal_direct_sweeps(prec, chi):
    h1_host, shift = m.mera_ising_h1(1.0)
    h1 = torch.from_numpy(h1_host.reshape(-1)).cuda()
    s_dir, u_dir, w_dir, r_dir = _state(3, chi)
    s_gr, u_gr, w_gr, r_gr = _state(3, chi)
    stream = torch.cuda.Stream()
    e_dir = torch.empty(1, dtype=torch.float64, device="cuda")
    e_gr = torch.empty(1, dtype=torch.float64, device="cuda")
    ws_dir = m.workspace(m.mera_sweep_workspace_size(s_dir.chi_b, s_dir.chi_t, prec))
    ws_gr = m.workspace(m.mera_sweep_workspace_size(s_gr.chi_b, s_gr.chi_t, prec))
    torch.cuda.synchronize()
    m.mera_device_status(clear=True)
    graph = m.mera_sweep_graph(s_gr, h1, shift, 20, e_gr, prec=prec, ws=ws_gr, stream=stream)
    try:
        # recording computes nothing: the state is still the initial one
        torch.cuda.synchronize()
        assert torch.equal(r_gr, r_dir) and all(torch.equal(a, b) for a, b in zip(u_gr, u_dir))
        for _ in range(3):
            try:
                m.mera_sweep(s_dir, h1, shift, 20, e_dir, prec=prec, ws=ws_dir, stream=stream)
            except m.MeraNotConverged:
                pass
            graph.launch(stream)
            stream.synchronize()
            assert e_gr.item() == e_dir.item()
        for a, b in zip(u_gr + w_gr + [r_gr], u_dir + w_dir + [r_dir]):
            assert torch.equal(a, b)
        assert m.mera_device_status(clear=True) == 0
    finally:
        graph.close()


def test_graph_needs_a_stream():
    h1_host, shift = m.mera_ising_h1(1.0)
    h1 = torch.from_numpy(h1_host.reshape(-1)).cuda()
    st, *_ = _state(0, 4)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MeraError):
        m.mera_sweep_graph(st, h1, shift, 20, e, prec=m.PREC_F64, stream=None)


def test_grown_mera_contains_the_smaller_one():
    """chi = 4 -> 6 growth: the new tensors are isometric / unitary to binary64
    accuracy, their leading blocks are the old tensors up to the perturbation,
    and the grown MERA's energy after one sweep is no higher than the old
    one's."""
    from paper_1906_12030_gb300 import grow

    h1_host, shift = m.mera_ising_h1(1.0)
    h1 = torch.from_numpy(h1_host.reshape(-1)).cuda()
    st, *_ = _state(5, 4)
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(30):
        try:
            m.mera_sweep(st, h1, shift, 20, e, prec=m.PREC_F64)
        except m.MeraNotConverged:
            pass
    e_small = e.item()
    big = grow.grow_state(st, I.layer_dims(6), seed=1, eps=1e-4)
    for (cb, ct), (nb, nt), u, w, u2, w2 in zip(zip(st.chi_b, st.chi_t), zip(big.chi_b, big.chi_t), st.us, st.ws,
                                               big.us, big.ws):
        U = u2.reshape(nb * nb, nb * nb)
        W = w2.reshape(nb * nb, nt)
        eye_u = torch.eye(nb * nb, dtype=torch.float64, device="cuda")
        eye_w = torch.eye(nt, dtype=torch.float64, device="cuda")
        assert float((U.T @ U - eye_u).abs().max()) < 1e-12
        assert float((W.T @ W - eye_w).abs().max()) < 1e-12
        old_u = u.reshape((cb,) * 4)
        old_w = w.reshape(cb, cb, ct)
        assert float((u2.reshape((nb,) * 4)[:cb, :cb, :cb, :cb] - old_u).abs().max()) < 1e-2
        assert float((w2.reshape(nb, nb, nt)[:cb, :cb, :ct] - old_w).abs().max()) < 1e-2
    try:
        m.mera_sweep(big, h1, shift, 20, e, prec=m.PREC_F64)
    except m.MeraNotConverged:
        pass
    e_big = e.item()
    # variational: above the exact energy, and the warm start loses nothing
    # (one more sweep with more freedom lowers it further)
    assert -4.0 / np.pi - 1e-9 <= e_big <= e_small + 1e-4



@pytest.mark.parametrize("use_graph", [False, True])
def test_sweep_from_host_buffers_equals_the_device_sweep(use_graph):
    """mera_sweep_host (the state copied in from pinned host memory, the
    sweep, the energy copied out) gives bit for bit the device sweep of the
    same state."""
    chi, prec = 4, m.PREC_BF16X3
    layers = I.init_mera(3, chi)
    h1n, shift = m.mera_ising_h1(1.0)

    def state():
        us = [torch.from_numpy(u).cuda().reshape(-1).contiguous() for u, _ in layers]
        ws = [torch.from_numpy(w).cuda().contiguous() for _, w in layers]
        rho = (torch.eye(chi ** 3, dtype=torch.float64, device="cuda") / chi ** 3).reshape(-1).contiguous()
        return m.MeraState(us, ws, rho)

    ref = state()
    h1 = torch.from_numpy(h1n.reshape(-1)).cuda()
    e_ref = torch.empty(1, dtype=torch.float64, device="cuda")
    m.mera_sweep(ref, h1, shift, 20, e_ref, prec=prec)
    # host copies of the initial state, then the same sweep through host buffers
    hu = [torch.from_numpy(u.reshape(-1).copy()).pin_memory() for u, _ in layers]
    hw = [torch.from_numpy(w.reshape(-1).copy()).pin_memory() for _, w in layers]
    hrho = (torch.eye(chi ** 3, dtype=torch.float64) / chi ** 3).reshape(-1).contiguous().pin_memory()
    hh1 = torch.from_numpy(h1n.reshape(-1).copy()).pin_memory()
    dev = state()
    for t in dev.us + dev.ws + [dev.rho_star]:
        t.zero_()  # the copies must bring the whole state in
    h1d = torch.zeros_like(h1)
    e_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    e_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream()
    ws = m.workspace(m.mera_sweep_workspace_size(dev.chi_b, dev.chi_t, prec))
    graph = m.mera_sweep_graph(dev, h1d, shift, 20, e_dev, prec=prec, ws=ws, stream=stream) if use_graph else None
    m.mera_sweep_host(dev, hu, hw, hrho, hh1, h1d, shift, 20, e_dev, e_host, prec=prec, ws=ws, graph=graph,
                      stream=stream)
    stream.synchronize()
    assert float(e_host[0]) == e_ref.item()
    for a, b in zip(ref.us + ref.ws + [ref.rho_star], dev.us + dev.ws + [dev.rho_star]):
        assert torch.equal(a, b)
    if graph is not None:
        graph.close()


def test_parity_symmetric_growth_keeps_the_symmetry():
    """grow_state(z2=True): a parity-symmetric chi = 4 MERA grown to chi = 6
    stays isometric, keeps every tensor block-diagonal in the parity charges,
    and holds the old tensors at their charge-preserving positions (up to the
    small perturbation and the polar step)."""
    from paper_1906_12030_gb300 import grow

    chi0, chi1 = 4, 6
    layers = I.init_mera(5, chi0, z2=True)
    st = m.MeraState([torch.from_numpy(u).cuda().reshape(-1).contiguous() for u, _ in layers],
                     [torch.from_numpy(w).cuda().contiguous() for _, w in layers],
                     (torch.eye(chi0 ** 3, dtype=torch.float64, device="cuda") / chi0 ** 3).reshape(-1))
    dims = I.layer_dims(chi1)
    g = grow.grow_state(st, dims, seed=1, eps=1e-3, z2=True, bottom_parity=I.parity_labels(4, physical=True))
    pb = I.parity_labels(4, physical=True)
    for k, ((cb, ct), u, w) in enumerate(zip(dims, g.us, g.ws)):
        u = u.cpu().numpy().reshape((cb,) * 4)
        w = w.cpu().numpy().reshape(cb, cb, ct)
        pt = I.parity_labels(ct)
        pair = pb[:, None] ^ pb[None, :]
        assert np.abs(u.reshape(cb * cb, -1).T @ u.reshape(cb * cb, -1) - np.eye(cb * cb)).max() < 1e-12
        assert np.abs(w.reshape(cb * cb, -1).T @ w.reshape(cb * cb, -1) - np.eye(ct)).max() < 1e-12
        assert np.abs(u[pair[:, :, None, None] != pair[None, None, :, :]]).max() < 1e-14
        assert np.abs(w[pair[:, :, None] != pt[None, None, :]]).max() < 1e-14
        pb = pt
    # the old top-layer isometry at its charge-preserving positions
    mb = grow._leg_map(chi0, chi1, True)
    w_old = layers[-1][1]
    w_new = g.ws[-1].cpu().numpy().reshape(chi1, chi1, chi1)[np.ix_(mb, mb, mb)]
    assert np.abs(w_new - w_old).max() < 1e-2
