"""Fixed-point split modes (MERA_PREC_OZ3 / MERA_PREC_OZ4) against the FP64
oracle and against the error model of the split.

Error model, per 256-element block of K with MA and MB the largest |entry|
of the A row and the B row in that block:
- representation: each entry is kept to EPS_S * MA (half the last slice's
  grid: OZ3 2^-26, OZ4 2^-35);
- dropped slice products (orders summing to S or more): at most DROP_S * MA
  * MB per term (OZ3 (1,2), (2,1): 2 * 2^-25; OZ4 (1,3), (3,1), (2,2):
  3 * 2^-34);
- the leading products of a block sum exactly; the other kept products
  (P1 of them per K step: 5 for OZ3, 9 for OZ4, each at most ~2^-7 MA MB)
  are accumulated in FP32, one rounding of at most 2^-24 of the partial sum
  per MMA over 16 terms: at most ceil(n/16) P1 2^-24 (n 2^-6 MA MB) in a
  block of n terms (a worst case; the rounding errors have random signs);
- blocks are summed as a binary32 pair (~2^-48).
The rigorous bound below adds these up; the statistical one checks the
typical size: the largest error over all outputs stays within
C_S sqrt(K) max|A| max|B|, C_S = 6 (2 EPS_S + DROP_S) for OZ3 (limited by
the dropped products) and 6 * 2^-27 for OZ4 (limited by the FP32 rounding
of the second accumulator; measured ~2^-28.5 per term).  A map chains ~10
such products, intermediates kept as binary32 pairs and split again.
"""
import numpy as np
import pytest

import mera_inputs as I
from oracle import mera_oracle as O

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu

OZ = [m.PREC_OZ3, m.PREC_OZ4]
EPS = {m.PREC_OZ3: 2.0 ** -26, m.PREC_OZ4: 2.0 ** -35}
DROP = {m.PREC_OZ3: 2 * 2.0 ** -25 + 2.0 ** -34, m.PREC_OZ4: 3 * 2.0 ** -34 + 2.0 ** -42}
P1 = {m.PREC_OZ3: 5, m.PREC_OZ4: 9}
STAT = {m.PREC_OZ3: 6 * (2 * 2.0 ** -26 + 2 * 2.0 ** -25), m.PREC_OZ4: 6 * 2.0 ** -27}
# map tolerances relative to the largest oracle entry: about 3x the largest
# error measured over the test's shapes (OZ3 2.6e-7, OZ4 4.0e-8)
MAP_TOL = {m.PREC_OZ3: 8e-7, m.PREC_OZ4: 1.2e-7}


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(autouse=True)
def _device_status_clean():
    m.mera_device_status(clear=True)
    yield
    assert m.mera_device_status(clear=True) == 0, "a bounded device wait timed out"


def _gemm(prec, A, B):
    C = torch.empty(A.shape[0], B.shape[0], dtype=torch.float64, device="cuda")
    m.mera_gemm_test(prec, _cuda(A), _cuda(B), C)
    return C.cpu().numpy()


def _bound(prec, A, B):
    """The rigorous elementwise error bound of the model above."""
    K = A.shape[1]
    out = np.zeros((A.shape[0], B.shape[0]))
    for k0 in range(0, K, 256):
        n = min(256, K - k0)
        a = np.abs(A[:, k0:k0 + 256]).max(axis=1)
        b = np.abs(B[:, k0:k0 + 256]).max(axis=1)
        per_block = n * (2 * EPS[prec] + DROP[prec]) + -(-n // 16) * P1[prec] * n * 1.1 * 2.0 ** -30
        out += per_block * np.outer(a, b)
    return out + 2.0 ** -45 * (np.abs(A) @ np.abs(B).T)


@pytest.mark.parametrize("prec", OZ)
@pytest.mark.parametrize("M,N,K", [(128, 128, 256), (16, 16, 16), (200, 300, 100), (130, 17, 7), (1000, 64, 520),
                                   (4096, 256, 4096), (257, 129, 33), (64, 512, 8192)])
def test_gemm_error_model(prec, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 13 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    got = _gemm(prec, A, B)
    exact = A @ B.T
    err = np.abs(got - exact)
    assert np.all(err <= _bound(prec, A, B) + 1e-300)
    amax, bmax = np.abs(A).max(), np.abs(B).max()
    print(f"prec={prec} K={K}: max err / (sqrt(K) max|A| max|B|) = {err.max() / (np.sqrt(K) * amax * bmax):.3e}")
    assert err.max() <= STAT[prec] * np.sqrt(K) * amax * bmax, err.max()


@pytest.mark.parametrize("K", [2048, 8192])
def test_oz4_is_far_more_accurate_than_fp32_accumulation(K):
    """The point of the mode: with exact block sums, OZ4's error does not
    grow with the FP32 accumulation over K that bounds BF16X6 (24-bit
    operands, FP32 accumulation)."""
    rng = np.random.default_rng(K)
    A = rng.standard_normal((512, K))
    B = rng.standard_normal((256, K))
    exact = A @ B.T
    e6 = np.abs(_gemm(m.PREC_BF16X6, A, B) - exact).max()
    e4 = np.abs(_gemm(m.PREC_OZ4, A, B) - exact).max()
    print(f"K={K}: BF16X6 {e6:.3e}  OZ4 {e4:.3e}")
    assert e4 * 100 < e6


@pytest.mark.parametrize("prec", OZ)
def test_blocks_carry_their_own_exponent(prec):
    """K = 512: block 0 of every A row is ~1e6 and its B partner ~1e-6,
    block 1 is O(1) on both sides, so both blocks contribute O(1) terms.
    One exponent per row would leave block 1 some 40 bits below the row's
    largest entry; one per block keeps it at full accuracy."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((256, 512))
    B = rng.standard_normal((128, 512))
    A[:, :256] *= 1e6
    B[:, :256] *= 1e-6
    got = _gemm(prec, A, B)
    exact = A @ B.T
    assert np.all(np.abs(got - exact) <= _bound(prec, A, B) + 1e-300)


@pytest.mark.parametrize("prec", OZ)
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 70, 40), (256, 128, 600)])
def test_gemm_exact_on_small_integers(prec, M, N, K):
    """Small integers are their own leading slice: products and sums are
    exact, so the binary64 output equals A B^T bit for bit."""
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    A[0, :] = 0.0
    got = _gemm(prec, A, B)
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


@pytest.mark.parametrize("prec", OZ)
@pytest.mark.parametrize("chi_b,chi_t", [(1, 1), (2, 1), (2, 2), (3, 3), (4, 4), (5, 5), (4, 16), (8, 8), (3, 8), (6, 6),
                                           (10, 10), (4, 14)])
def test_maps(prec, chi_b, chi_t):
    res = _maps(prec, chi_b, chi_t, 11)
    errs = {}
    for name, (got, want) in res.items():
        g = got.cpu().numpy().reshape(want.shape)
        errs[name] = float(np.abs(g - want).max() / np.abs(want).max())
    print(f"prec={prec} chi=({chi_b},{chi_t}) errors {errs}")
    for name, e in errs.items():
        assert e < MAP_TOL[prec], (name, e)


@pytest.mark.parametrize("prec,chi,tol", [(m.PREC_OZ4, 4, 1e-8), (m.PREC_OZ4, 8, 1e-8), (m.PREC_OZ3, 4, 1e-6)])
def test_sweeps_track_the_oracle(prec, chi, tol):
    """20 optimisation sweeps from the seeded QR start in the split mode
    track the FP64 oracle's sweep energies to `tol` per spin (the mixed-
    precision target is 1e-6 per site)."""
    n_sweeps = 20
    layers = I.init_mera(0, chi)
    h1, shift = O.ising_h1(1.0)
    _, _, oes = O.run([(u.copy(), w.copy()) for u, w in layers], 1.0, n_sweeps, 20)
    us = [_cuda(u).reshape(-1).clone() for u, _ in layers]
    ws = [_cuda(w).clone() for _, w in layers]
    rho = _cuda(O.identity_density(chi)).reshape(-1).clone()
    st = m.MeraState(us, ws, rho)
    e = torch.empty(n_sweeps, dtype=torch.float64, device="cuda")
    h1d = _cuda(h1).reshape(-1)
    for i in range(n_sweeps):
        m.mera_sweep(st, h1d, shift, 20, e[i:i + 1], prec=prec)
    es = e.cpu().numpy()
    gap = np.abs(es - np.asarray(oes))
    print(f"prec={prec} chi={chi}: max |dE| per spin over {n_sweeps} sweeps {gap.max():.3e}")
    assert gap.max() < tol
