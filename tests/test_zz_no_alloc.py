"""The allocation-free ascending map (mera_ascend_noalloc).

This entry point is for callers that cannot hand the library scratch memory
(an application whose own pool allocator owns all device memory, or a loop
that cannot afford a cudaMalloc); it keeps its scratch in a static device
array.  Its result must equal mera_ascend's, within the FP64 tolerance the
parity tests use, on two calls in a row (the second call finds the first
call's leftovers in the shared array).  The file sorts last so that a run
stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import mera_inputs as I

torch = pytest.importorskip("torch")
m = pytest.importorskip("paper_1906_12030_gb300")

pytestmark = pytest.mark.gpu

TOL = {m.PREC_F64: 1e-10, m.PREC_BF16X3: 5e-4}


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(-1)


def _call_noalloc(h, u, w, chi_b, chi_t, out, prec):
    """Straight through the C ABI (ctypes), no workspace argument."""
    lib = m.library()
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.mera_ascend_noalloc(ptr(h), ptr(u), ptr(w), chi_b, chi_t, ptr(out), prec, stream)


@pytest.mark.parametrize("prec,chi_b,chi_t", [(m.PREC_F64, 4, 4), (m.PREC_F64, 5, 5), (m.PREC_F64, 4, 16),
                                              (m.PREC_F64, 8, 8), (m.PREC_BF16X3, 8, 8)])
def test_noalloc_matches_workspace_entry_point_twice(prec, chi_b, chi_t):
    outs = []
    for seed in (31, 32):  # two calls in a row, different inputs
        rng = np.random.default_rng(seed)
        u, w = I.random_u(rng, chi_b), I.random_w(rng, chi_b, chi_t)
        h = I.random_operator(rng, chi_b)
        hd, ud, wd = _cuda(h), _cuda(u), _cuda(w)
        ref = torch.empty(chi_t ** 6, dtype=torch.float64, device="cuda")
        m.mera_ascend(hd, ud, wd, chi_b, chi_t, ref, prec=prec)
        got = torch.full((chi_t ** 6,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call_noalloc(hd, ud, wd, chi_b, chi_t, got, prec) == 0, m.library().mera_last_error()
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - r).max() <= TOL[prec] * np.abs(r).max()
        outs.append(g)
    assert not np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_the_static_array():
    chi = 10  # needs ~92 MiB of FP64 scratch > 32 MiB
    assert m.mera_workspace_size(m.OP_ASCEND, chi, chi, m.PREC_F64) > m.NOALLOC_SCRATCH_BYTES
    z = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")  # noqa: E731
    status = _call_noalloc(z(chi ** 6), z(chi ** 4), z(chi ** 3), chi, chi, z(chi ** 6), m.PREC_F64)
    assert status == 1  # MERA_EINVAL
    assert b"static array" in m.library().mera_last_error()
