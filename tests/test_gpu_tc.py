"""Tensor-core (tcgen05) paths: the GEMM kernel and the maps in TF32, BF16
and split-BF16 (BF16X3) against the FP64 oracle.

GEMM bound (elementwise, rigorous): with operand unit roundoff u and FP32
accumulation over K terms,
    |C - A B^T| <= (2 u + u^2 + K 2^-24) (|A| |B|^T),
u = 2^-11 + 2^-24 for TF32 (11 significant bits after the binary64 -> FP32
rounding), 2^-8 for BF16 (8 significant bits), and 1.5 * 2^-16 for the BF16
pair: hi + lo represents x to 2^-16 |x| and the dropped lo*lo product is at
most 2^-16 |a b|, so 2u >= 3 * 2^-16.
Map tolerances (relative to the largest oracle entry): a diagram is ~10
chained contractions, each rounding its result to the operand precision
once (~10 u in a random walk, x2 for the even + odd / 4-6 hole sums) and
accumulating up to K = chi_t^3 products in FP32.  TF32: 10 u = 5e-3.
BF16: 10 u = 4e-2 (3e-2 kept, 3x the measured 9e-3).  BF16X3: the random
walk of ~10 roundings to the 16-bit pair, sqrt(10) * 2^-17 = 2.4e-5, plus
the FP32 accumulation over K <= 4096; measured at most 2.9e-5 over these
shapes and the chi = 16 rows, so 8e-5 (about 3x; the bound 10 u + K 2^-24
= 5e-4 would let a tenfold regression pass).  The error grows with K: at
chi = 32 (K up to 32768) a descending map is ~2.4e-4 from the fixed-point
split mode OZ4 (bench.py's accuracy block).
BF16X6: the binary64 -> FP32 conversion (2^-24), the three-part split of
the FP32 value (2^-25) and the dropped products (mid*lo, lo*mid, lo*lo,
below 2^-23 |a b| together) fit in 2u with u = 2^-22; its maps are
limited by FP32 accumulation: 10 u + 10 sqrt(K) 2^-24 (random walk over
K <= 4096 in ~10 chained GEMMs) = 4e-5.
"""
import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu

U_OPERAND = {m.PREC_TF32: 2.0 ** -11 + 2.0 ** -24, m.PREC_BF16: 2.0 ** -8, m.PREC_BF16X3: 1.5 * 2.0 ** -16,
             m.PREC_BF16X6: 2.0 ** -22}
MAP_TOL = {m.PREC_TF32: 5e-3, m.PREC_BF16: 3e-2, m.PREC_BF16X3: 8e-5, m.PREC_BF16X6: 4e-5}
TC_PRECS = [m.PREC_TF32, m.PREC_BF16, m.PREC_BF16X3, m.PREC_BF16X6]


def bf16x3_tol(chi):
    """BF16X3 map tolerance at bond dimension chi: MAP_TOL (measured) while
    the contractions have K = chi^3 <= 4096, the derived bound 10 u + K 2^-24
    beyond, where the FP32 accumulation over K grows (measured 2.0e-4 at
    chi = 32 and 4.1e-4 at chi = 40 against bounds of 2.2e-3 and 4.0e-3)."""
    k = chi ** 3
    return MAP_TOL[m.PREC_BF16X3] if k <= 4096 else 10 * U_OPERAND[m.PREC_BF16X3] + k * 2.0 ** -24


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(autouse=True)
def _device_status_clean():
    m.mera_device_status(clear=True)
    yield
    assert m.mera_device_status(clear=True) == 0, "a bounded device wait timed out"


@pytest.mark.parametrize("prec", TC_PRECS + [m.PREC_F64])
# the planner's widths for these N: 256, 16, 160 (300), 192 (576), 64, 64, 256, 160 (129), 256
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (16, 16, 16), (200, 300, 100), (300, 576, 200), (130, 17, 7),
                                   (1000, 64, 520), (4096, 256, 512), (257, 129, 33), (64, 512, 2048)])
def test_gemm_bound(prec, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C = torch.empty(M * N, dtype=torch.float64, device="cuda")
    m.mera_gemm_test(prec, _cuda(A), _cuda(B), C)
    got = C.cpu().numpy().reshape(M, N)
    exact = A @ B.T
    mag = np.abs(A) @ np.abs(B).T
    if prec == m.PREC_F64:
        assert np.all(np.abs(got - exact) <= 1e-14 * K * mag + 1e-300)
        return
    u = U_OPERAND[prec]
    bound = (2 * u + u * u + K * 2.0 ** -24) * mag
    assert np.all(np.abs(got - exact) <= bound), float(np.max(np.abs(got - exact) / bound))


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 70, 40)])
def test_gemm_exact_on_small_integers(prec, M, N, K):
    """Small-integer operands are exact in every operand format and their
    products and sums (|c| <= 64 * K) are exact in the FP32 accumulator, so
    the caller's binary64 output must equal A B^T bit for bit: this pins the
    epilogue's binary32 -> binary64 conversion, including signs and zeros."""
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    A[0, :] = 0.0  # a zero row: signed zeros in the output
    C = torch.empty(M * N, dtype=torch.float64, device="cuda")
    m.mera_gemm_test(prec, _cuda(A), _cuda(B), C)
    got = C.cpu().numpy().reshape(M, N)
    assert np.array_equal(got, A @ B.T)


def _maps(prec, chi_b, chi_t, seed):
    rng = np.random.default_rng(seed)
    u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
    h = I.random_operator(rng, chi_b)
    rho = I.random_density(rng, chi_t)
    d = lambda x: _cuda(x).reshape(-1)  # noqa: E731
    hd, rd, ud, wd = d(h), d(rho), d(u), d(w)
    res = {}
    a = torch.empty(chi_t ** 6, dtype=torch.float64, device="cuda")
    m.mera_ascend(hd, ud, wd, chi_b, chi_t, a, prec=prec)
    res["ascend"] = (a, O.ascend(h, u, w))
    dd = torch.empty(chi_b ** 6, dtype=torch.float64, device="cuda")
    m.mera_descend(rd, ud, wd, chi_b, chi_t, dd, prec=prec)
    res["descend"] = (dd, O.descend(rho, u, w))
    gu = torch.empty(chi_b ** 4, dtype=torch.float64, device="cuda")
    m.mera_env_u(hd, rd, ud, wd, chi_b, chi_t, gu, prec=prec)
    res["env_u"] = (gu, O.env_u(h, rho, u, w))
    gw = torch.empty(chi_b ** 2 * chi_t, dtype=torch.float64, device="cuda")
    m.mera_env_w(hd, rd, ud, wd, chi_b, chi_t, gw, prec=prec)
    res["env_w"] = (gw, O.env_w(h, rho, u, w))
    return res


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("chi_b,chi_t", [(1, 1), (2, 1), (2, 2), (3, 3), (4, 4), (5, 5), (4, 16), (8, 8), (3, 8), (6, 6),
                                           (10, 10), (4, 14), (4, 12), (12, 12)])
def test_maps_mixed_precision(prec, chi_b, chi_t):
    res = _maps(prec, chi_b, chi_t, 11)
    errs = {}
    for name, (got, want) in res.items():
        g = got.cpu().numpy().reshape(want.shape)
        errs[name] = float(np.abs(g - want).max() / np.abs(want).max())
    print(f"prec={prec} chi=({chi_b},{chi_t}) errors {errs}")
    for name, e in errs.items():
        assert e < MAP_TOL[prec], (name, e)


@pytest.mark.parametrize("prec", [m.PREC_F64, m.PREC_BF16X3, m.PREC_BF16])
@pytest.mark.parametrize("chi_b,chi_t,block", [(4, 4, False), (8, 8, False), (4, 16, False), (8, 8, True)])
def test_sliced_maps(prec, chi_b, chi_t, block):
    """Rank-7 intermediates computed one slice at a time (forced here at
    small chi; by default only above 16 GiB) give the oracle's maps within
    the mode's tolerance, and agree with the unsliced program.  block: a
    threshold of half the chi = 8 intermediate, so each slice covers four
    values of the sliced leg."""
    whole = _maps(prec, chi_b, chi_t, 5)
    eb = {m.PREC_F64: 8, m.PREC_BF16X3: 4, m.PREC_BF16: 2}[prec]
    m.mera_set_slice_bytes(8 ** 7 * eb // 2 if block else 0)
    try:
        plan = m.mera_plan_json(m.OP_ENV_W, chi_b, chi_t, prec)
        assert any("=" in st["label"] for dg in plan["diagrams"] for st in dg["steps"] if st["kind"] == "gemm")
        res = _maps(prec, chi_b, chi_t, 5)
        torch.cuda.synchronize()
    finally:
        m.mera_set_slice_bytes(16 << 30)
    tol = 1e-10 if prec == m.PREC_F64 else MAP_TOL[prec]
    for name, (got, want) in res.items():
        g = got.cpu().numpy().reshape(want.shape)
        w0 = whole[name][0].cpu().numpy().reshape(want.shape)
        scale = np.abs(want).max()
        assert np.abs(g - want).max() / scale < tol, name
        assert np.abs(g - w0).max() / scale < tol, name


@pytest.mark.parametrize("prec", TC_PRECS)
def test_fixed_point_and_energy_mixed(prec):
    chi = 4
    rng = np.random.default_rng(12)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    want, _ = O.fixed_point_rho(u, w, O.identity_density(chi), 20)
    rho = _cuda(O.identity_density(chi)).reshape(-1).clone()
    m.mera_fixed_point_rho(_cuda(u).reshape(-1), _cuda(w).reshape(-1), chi, rho, 20, prec=prec)
    r = rho.cpu().numpy().reshape(want.shape)
    assert np.abs(r - want).max() / np.abs(want).max() < MAP_TOL[prec]
    # normalisation and symmetry are FP64 in every mode
    rm = r.reshape(chi ** 3, -1)
    assert abs(np.trace(rm) - 1.0) < 1e-14
    assert np.abs(rm - rm.T).max() == 0.0


# --------------------------------------------------------------------------
# The benchmarked configuration: chi = 16 in BF16X3 (bench.py's default).
# Sampled rows against the oracle's row-by-row contraction, and properties
# that hold at any size.
# --------------------------------------------------------------------------
def test_chi16_bf16x3_sampled_rows_and_properties():
    chi, prec = 16, m.PREC_BF16X3
    rng = np.random.default_rng(90)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h, rho = I.random_operator(rng, chi), I.random_density(rng, chi)
    d = lambda x: _cuda(x).reshape(-1)  # noqa: E731
    ud, wd, hd, rd = d(u), d(w), d(h), d(rho)
    a = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")
    m.mera_ascend(hd, ud, wd, chi, chi, a, prec=prec)
    got = a.cpu().numpy().reshape((chi,) * 6)
    rows = [(0, 0, 0), (5, 11, 2), (15, 15, 15)]
    want = O.ascend_rows(h, u, w, rows)
    scale = np.abs(want).max()
    for k, (p, q, r) in enumerate(rows):
        assert np.abs(got[p, q, r] - want[k]).max() <= MAP_TOL[prec] * scale
    # duality of the GPU maps themselves, and trace preservation of D
    dd = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")
    m.mera_descend(rd, ud, wd, chi, chi, dd, prec=prec)
    lhs = float(torch.dot(a, rd))
    rhs = float(torch.dot(hd, dd))
    assert abs(lhs - rhs) <= MAP_TOL[prec] * (abs(lhs) + 1e-30) * 10
    tr = float(torch.trace(dd.reshape(chi ** 3, chi ** 3)))
    assert tr == pytest.approx(1.0, abs=MAP_TOL[prec])
    # A(1) = 1 (Eq. iso, Eq. unitarity)
    eye = torch.eye(chi ** 3, dtype=torch.float64, device="cuda").reshape(-1)
    m.mera_ascend(eye, ud, wd, chi, chi, a, prec=prec)
    err = (a.reshape(chi ** 3, chi ** 3) - torch.eye(chi ** 3, dtype=torch.float64, device="cuda")).abs().max()
    assert float(err) < MAP_TOL[prec]


@pytest.mark.parametrize("prec,tol", [(m.PREC_F64, 1e-10), (m.PREC_BF16X3, None), (m.PREC_OZ4, 1e-8)])
def test_descend_chi16_sampled_rows(prec, tol):
    """The descending map at the benchmarked size (chi = 16; the rho* power
    iteration applies it 20 times per sweep) against the oracle's rows with
    the ket legs held fixed (oracle.descend_rows), entry by entry."""
    chi = 16
    tol = MAP_TOL[prec] if tol is None else tol
    rng = np.random.default_rng(91)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    rho = I.random_density(rng, chi)
    d = lambda x: _cuda(x).reshape(-1)  # noqa: E731
    out = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")
    m.mera_descend(d(rho), d(u), d(w), chi, chi, out, prec=prec)
    got = out.cpu().numpy().reshape((chi,) * 6)
    rows = [(0, 0, 0), (7, 2, 13), (15, 15, 15), (9, 9, 4)]
    want = O.descend_rows(rho, u, w, rows)
    scale = np.abs(want).max()
    errs = [float(np.abs(got[i, j, k] - want[n]).max() / scale) for n, (i, j, k) in enumerate(rows)]
    print(f"prec={prec} chi=16 descend rows: max rel err {max(errs):.3e}")
    assert max(errs) <= tol


def _dot(a, b, chunk=1 << 30):
    """Dot product of long vectors (the BLAS dot takes at most 2^31 - 1)."""
    return sum(float(torch.dot(a[i:i + chunk], b[i:i + chunk])) for i in range(0, a.numel(), chunk))


@pytest.mark.parametrize("chi", [32, 40])
def test_full_size_properties(chi):
    """chi = 32 and 40 (the precision workload's largest sizes; chi = 40 runs
    the sliced chi^9 pairs), where the oracle cannot run: properties that hold
    at any size, on seeded operators drawn on the device.
    - A(1) = 1 (Eq. iso, Eq. unitarity);
    - tr D(rho) = tr rho;
    - duality <A(h), rho> = <h, D(rho)> (D is the adjoint of A)."""
    prec = m.PREC_BF16X3
    tol = bf16x3_tol(chi)
    rng = np.random.default_rng(chi)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    ud, wd = _cuda(u).reshape(-1), _cuda(w).reshape(-1)
    n3 = chi ** 3
    g = torch.Generator(device="cuda")
    g.manual_seed(chi)
    ws = m.workspace(max(m.mera_workspace_size(op, chi, chi, prec) for op in (m.OP_ASCEND, m.OP_DESCEND)))
    out = torch.empty(n3 * n3, dtype=torch.float64, device="cuda")
    x = torch.eye(n3, dtype=torch.float64, device="cuda").reshape(-1)
    m.mera_ascend(x, ud, wd, chi, chi, out, prec=prec, ws=ws)
    err = float((out.reshape(n3, n3).diagonal() - 1.0).abs().max())
    out.reshape(n3, n3).diagonal().zero_()
    err = max(err, float(out.abs().max()))
    assert err < tol, err
    # duality and trace with random (non-symmetric) h and rho
    x.normal_(generator=g)  # h
    rho = torch.empty_like(x).normal_(generator=g)
    m.mera_ascend(x, ud, wd, chi, chi, out, prec=prec, ws=ws)
    lhs = _dot(out, rho)
    hn, rn = float(x.norm()), float(rho.norm())
    m.mera_descend(rho, ud, wd, chi, chi, out, prec=prec, ws=ws)
    rhs = _dot(x, out)
    # both sides carry the maps' error relative to |h| |rho|
    assert abs(lhs - rhs) <= tol * hn * rn, (lhs, rhs)
    tr_in = float(rho.reshape(n3, n3).diagonal().sum())
    tr_out = float(out.reshape(n3, n3).diagonal().sum())
    assert abs(tr_out - tr_in) <= tol * float(rho.reshape(n3, n3).diagonal().abs().sum()) + 1e-9
    torch.cuda.synchronize()


def test_autotuned_widths_keep_the_maps():
    """The tile-width autotuner records a width for the large GEMM shapes of
    the chi = 8 programs; the maps built afterwards use those widths (the
    plan says so) and still match the oracle within the mode's tolerance."""
    prec, chi = m.PREC_BF16X3, 8
    m.mera_autotune_reset()
    try:
        n = m.mera_autotune(m.OP_ASCEND, chi, chi, prec) + m.mera_autotune(m.OP_ENV_W, chi, chi, prec)
        assert n > 0
        widths = {st["bn"] for dg in m.mera_plan_json(m.OP_ENV_W, chi, chi, prec)["diagrams"]
                  for st in dg["steps"] if st["kind"] == "gemm"}
        assert widths <= {16, 64, 128, 256}
        res = _maps(prec, chi, chi, 21)
        for name, (got, want) in res.items():
            g = got.cpu().numpy().reshape(want.shape)
            assert np.abs(g - want).max() / np.abs(want).max() < MAP_TOL[prec], name
    finally:
        m.mera_autotune_reset()


def test_autotuned_widths_are_bit_identical_at_full_size():
    """chi = 16, the benchmarked size: the widths the autotuner picks change
    the tiling, not the order in which each output element sums its K range
    (no step gains a K split here), so the maps come out bit for bit the same
    as with the planner's widths."""
    prec, chi = m.PREC_BF16X3, 16
    rng = np.random.default_rng(16)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    ud, wd = _cuda(u).reshape(-1), _cuda(w).reshape(-1)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    h = torch.randn(chi ** 6, dtype=torch.float64, device="cuda", generator=g)
    m.mera_autotune_reset()
    try:
        a0 = torch.empty_like(h)
        d0 = torch.empty_like(h)
        m.mera_ascend(h, ud, wd, chi, chi, a0, prec=prec)
        m.mera_descend(h, ud, wd, chi, chi, d0, prec=prec)
        m.mera_autotune(m.OP_ASCEND, chi, chi, prec)
        m.mera_autotune(m.OP_DESCEND, chi, chi, prec)
        plans = [m.mera_plan_json(op, chi, chi, prec) for op in (m.OP_ASCEND, m.OP_DESCEND)]
        split_steps = [st for p in plans for dg in p["diagrams"] for st in dg["steps"]
                       if st["kind"] == "gemm" and st["split"] > 1]
        a1 = torch.empty_like(h)
        d1 = torch.empty_like(h)
        m.mera_ascend(h, ud, wd, chi, chi, a1, prec=prec)
        m.mera_descend(h, ud, wd, chi, chi, d1, prec=prec)
        if not split_steps:
            assert torch.equal(a0, a1) and torch.equal(d0, d1)
        else:
            assert float((a0 - a1).abs().max()) <= MAP_TOL[prec] * float(a0.abs().max())
    finally:
        m.mera_autotune_reset()


def test_chi16_sampled_environments():
    """chi = 16, the benchmarked size: rows of Gamma_u and a column of Gamma_w
    from the library (FP64 and BF16X3, the environments of every sweep) against
    the oracle's entry-wise helpers (the whole maps cost minutes on the CPU).
    Tolerances are relative to the largest sampled oracle entry."""
    chi = 16
    rng = np.random.default_rng(91)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    h, rho = I.random_operator(rng, chi), I.random_density(rng, chi)
    rows, cols = [(0, 0), (7, 12)], [5]
    want_u = O.env_u_rows(h, rho, u, w, rows)
    want_w = O.env_w_cols(h, rho, u, w, cols)
    su, sw = np.abs(want_u).max(), np.abs(want_w).max()
    d = lambda x: _cuda(x).reshape(-1)  # noqa: E731
    ud, wd, hd, rd = d(u), d(w), d(h), d(rho)
    for prec, tol in ((m.PREC_F64, 1e-10), (m.PREC_BF16X3, MAP_TOL[m.PREC_BF16X3])):
        gu = torch.empty(chi ** 4, dtype=torch.float64, device="cuda")
        gw = torch.empty(chi ** 3, dtype=torch.float64, device="cuda")
        m.mera_env_u(hd, rd, ud, wd, chi, chi, gu, prec=prec)
        m.mera_env_w(hd, rd, ud, wd, chi, chi, gw, prec=prec)
        gu = gu.cpu().numpy().reshape((chi,) * 4)
        gw = gw.cpu().numpy().reshape(chi, chi, chi)
        for k, (a, b) in enumerate(rows):
            assert np.abs(gu[a, b] - want_u[k]).max() <= tol * su, (prec, a, b)
        for k, c in enumerate(cols):
            assert np.abs(gw[:, :, c] - want_w[k]).max() <= tol * sw, (prec, c)
