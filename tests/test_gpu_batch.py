"""Batched sweeps of independent MERAs (different transverse fields h and
bond dimensions): each result must be exactly what a lone sweep gives, and
every MERA's variational energy stays above the exact ground-state energy
e0(h) of the infinite chain (closed form, Sec. III A)."""
import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu


def _mera(seed, chi, hz):
    layers = I.init_mera(seed, chi)
    us = [torch.from_numpy(u).cuda().reshape(-1).contiguous() for u, _ in layers]
    ws = [torch.from_numpy(w).cuda().contiguous() for _, w in layers]
    rho = (torch.eye(chi ** 3, dtype=torch.float64, device="cuda") / chi ** 3).reshape(-1).contiguous()
    h1, shift = m.mera_ising_h1(hz)
    return m.MeraState(us, ws, rho), torch.from_numpy(h1.reshape(-1)).cuda(), shift


def _sweep(st, h1, shift, e, prec):
    try:
        m.mera_sweep(st, h1, shift, 20, e, prec=prec)
    except m.MeraNotConverged:
        pass


@pytest.mark.parametrize("prec", [m.PREC_F64, m.PREC_BF16X3])
def test_batched_sweeps_equal_lone_sweeps(prec):
    rng = np.random.default_rng(80)
    specs = [(s, int(rng.choice([4, 6, 8])), float(rng.uniform(0.9, 1.1))) for s in range(6)]
    batch = [_mera(*sp) for sp in specs]
    alone = [_mera(*sp) for sp in specs]
    eb = torch.empty(len(specs), dtype=torch.float64, device="cuda")
    ea = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(3):
        try:
            m.mera_sweep_batch([b[0] for b in batch], [b[1] for b in batch], [b[2] for b in batch], 20, eb,
                               prec=prec, n_threads=6)
        except m.MeraNotConverged:
            pass
        energies = []
        for st, h1, shift in alone:
            _sweep(st, h1, shift, ea, prec)
            energies.append(ea.item())
        torch.cuda.synchronize()
        assert eb.cpu().tolist() == energies
    for (sb, _, _), (sa, _, _) in zip(batch, alone):
        for x, y in zip(sb.us + sb.ws + [sb.rho_star], sa.us + sa.ws + [sa.rho_star]):
            assert torch.equal(x, y)


def test_batched_energies_respect_exact_bound():
    rng = np.random.default_rng(81)
    specs = [(10 + s, 4, float(rng.uniform(0.9, 1.1))) for s in range(4)]
    batch = [_mera(*sp) for sp in specs]
    eb = torch.empty(len(specs), dtype=torch.float64, device="cuda")
    for _ in range(20):
        try:
            m.mera_sweep_batch([b[0] for b in batch], [b[1] for b in batch], [b[2] for b in batch], 20, eb,
                               n_threads=4)
        except m.MeraNotConverged:
            pass
    for (st, h1, shift), (_, chi, hz) in zip(batch, specs):
        # variational energy of the MERA as it stands: converged rho*, then down to the lattice
        rho = st.rho_star.clone()
        m.mera_fixed_point_rho(st.us[-1], st.ws[-1], chi, rho, 300)
        for t in range(len(st.us) - 2, 0, -1):
            out = torch.empty(st.chi_b[t] ** 6, dtype=torch.float64, device="cuda")
            m.mera_descend(rho, st.us[t], st.ws[t], st.chi_b[t], st.chi_t[t], out)
            rho = out
        e = torch.empty(1, dtype=torch.float64, device="cuda")
        m.mera_energy(h1, rho, st.us[0], st.ws[0], st.chi_b[0], st.chi_t[0], e)
        e_site = 0.5 * (e.item() + shift)
        e0 = O.exact_energy_per_spin(hz)
        assert e_site >= e0 - 1e-12
        assert e_site < 0.6 * e0  # well down from the random start (about 0.05 e0)


def test_lanes_share_scratch_and_match_lone_sweeps():
    """A budget of twice the largest scratch forces lanes: MERAs of one lane
    share a buffer and a stream, and every result is still exactly the lone
    sweep's."""
    prec = m.PREC_BF16X3
    rng = np.random.default_rng(82)
    specs = [(20 + s, int(rng.choice([4, 6, 8])), float(rng.uniform(0.9, 1.1))) for s in range(6)]
    batch = [_mera(*sp) for sp in specs]
    alone = [_mera(*sp) for sp in specs]
    states = [b[0] for b in batch]
    need = [m.mera_sweep_workspace_size(st.chi_b, st.chi_t, prec) for st in states]
    wss, streams = m.batch_resources(states, prec, budget_bytes=2 * max(need))
    assert 1 < len({id(s) for s in streams}) < len(states)
    eb = torch.empty(len(specs), dtype=torch.float64, device="cuda")
    ea = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        try:
            m.mera_sweep_batch(states, [b[1] for b in batch], [b[2] for b in batch], 20, eb, prec=prec, wss=wss,
                               streams=streams, n_threads=4)
        except m.MeraNotConverged:
            pass
        energies = []
        for st, h1, shift in alone:
            _sweep(st, h1, shift, ea, prec)
            energies.append(ea.item())
        torch.cuda.synchronize()
        assert eb.cpu().tolist() == energies
    for sb, (sa, _, _) in zip(states, alone):
        for x, y in zip(sb.us + sb.ws + [sb.rho_star], sa.us + sa.ws + [sa.rho_star]):
            assert torch.equal(x, y)


def test_scratch_shared_across_streams_is_rejected():
    batch = [_mera(30 + s, 4, 1.0) for s in range(2)]
    st0 = batch[0][0]
    ws = m.workspace(m.mera_sweep_workspace_size(st0.chi_b, st0.chi_t, m.PREC_F64))
    e = torch.zeros(2, dtype=torch.float64, device="cuda")
    n0 = m.mera_launch_count()
    with pytest.raises(m.MeraError, match="another stream"):
        m.mera_sweep_batch([b[0] for b in batch], [b[1] for b in batch], [b[2] for b in batch], 20, e,
                           wss=[ws, ws], streams=[torch.cuda.Stream(), torch.cuda.Stream()])
    assert m.mera_launch_count() == n0


@pytest.mark.parametrize("prec,tol,tol_x", [(m.PREC_F64, 1e-11, 1e-8), (m.PREC_OZ4, 1e-8, 1e-5)])
def test_batched_meras_match_the_oracle(prec, tol, tol_x):
    """Every member of a batch (different h and chi) against the FP64
    oracle's sweeps of the same MERA: energies per spin after each of three
    sweeps (to tol), and the tensors after the last (to tol_x)."""
    specs = [(30, 3, 0.93), (31, 4, 1.0), (32, 4, 1.07), (33, 5, 0.97)]
    batch = [_mera(*sp) for sp in specs]
    eb = torch.empty(len(specs), dtype=torch.float64, device="cuda")
    oracle = []
    for seed, chi, hz in specs:
        h1, shift = O.ising_h1(hz)
        oracle.append(([(u.copy(), w.copy()) for u, w in I.init_mera(seed, chi)], h1, shift,
                       O.identity_density(chi)))
    for _ in range(3):
        m.mera_sweep_batch([b[0] for b in batch], [b[1] for b in batch], [b[2] for b in batch], 20, eb,
                           prec=prec, n_threads=4)
        got = eb.cpu().numpy()
        for i, (layers, h1, shift, rho) in enumerate(oracle):
            layers, rho, e = O.sweep(layers, h1, shift, rho, 20)
            oracle[i] = (layers, h1, shift, rho)
            assert abs(got[i] - e) <= tol, (i, got[i], e)
    for (st, _, _), (layers, _, _, _) in zip(batch, oracle):
        for (ou, ow), u, w in zip(layers, st.us, st.ws):
            assert np.abs(u.cpu().numpy().reshape(ou.shape) - ou).max() < tol_x
            assert np.abs(w.cpu().numpy().reshape(ow.shape) - ow).max() < tol_x
    assert m.mera_device_status(clear=True) == 0
