"""ctypes binding of ``include/mera.h``: argument marshalling only.

Each function has the name of its C entry point and forwards PyTorch
tensors as raw device pointers.  Errors come back as :class:`MeraError`
(carrying the C status and message); a missing library raises at import
time of the first call, never falls back to another implementation.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

__all__ = [
    "MeraError", "MeraNotConverged", "PREC_F64", "PREC_TF32", "PREC_BF16", "PREC_BF16X3", "PREC_BF16X6",
    "PREC_OZ3", "PREC_OZ4", "PRECS",
    "OP_ASCEND", "OP_DESCEND", "OP_ENV_U", "OP_ENV_W", "OP_ENERGY", "OP_FIXED_POINT",
    "library", "library_path", "mera_version", "mera_workspace_size", "mera_ascend", "mera_descend",
    "mera_fixed_point_rho", "mera_env_u", "mera_env_w", "mera_polar_update", "mera_polar_workspace_size",
    "mera_energy", "mera_ising_h1", "mera_sweep", "mera_sweep_workspace_size", "mera_plan_json", "mera_flops",
    "workspace", "MeraState", "mera_launch_count", "mera_profile_enable", "mera_profile_read",
    "PROF_GEMM", "PROF_GEMM_DOMINANT", "PROF_PERMUTE", "mera_device_status", "mera_gemm_test",
    "mera_ascend_noalloc", "NOALLOC_SCRATCH_BYTES", "mera_op_transpose", "mera_energy_adjoint", "mera_sweep_host", "mera_sweep_batch", "mera_set_slice_bytes",
    "MeraGraph", "mera_sweep_graph", "mera_stiefel_step",
    "mera_stiefel_workspace_size", "mera_sweep_riemannian", "mera_autotune", "mera_autotune_reset",
    "mera_batch_lanes", "batch_resources", "mera_set_tile_width", "mera_tile_widths",
]

PREC_F64, PREC_TF32, PREC_BF16, PREC_BF16X3, PREC_BF16X6, PREC_OZ3, PREC_OZ4 = 0, 1, 2, 3, 4, 5, 6
PRECS = {"f64": PREC_F64, "tf32": PREC_TF32, "bf16": PREC_BF16, "bf16x3": PREC_BF16X3, "bf16x6": PREC_BF16X6,
         "oz3": PREC_OZ3, "oz4": PREC_OZ4}
OP_ASCEND, OP_DESCEND, OP_ENV_U, OP_ENV_W, OP_ENERGY, OP_FIXED_POINT, OP_ENERGY_ADJOINT = 0, 1, 2, 3, 4, 5, 6
MAX_LAYERS = 8
PROF_GEMM, PROF_GEMM_DOMINANT, PROF_PERMUTE = 0, 1, 2
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

_OK, _EINVAL, _ENOMEM, _ECUDA, _ENOTCONV, _ETIMEOUT = 0, 1, 2, 3, 4, 5


class MeraError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mera status {status}: {message}")
        self.status = status


class MeraNotConverged(MeraError):
    pass


class _State(ctypes.Structure):
    _fields_ = [
        ("n_layers", ctypes.c_int),
        ("chi_b", ctypes.c_int * MAX_LAYERS),
        ("chi_t", ctypes.c_int * MAX_LAYERS),
        ("u", ctypes.c_void_p * MAX_LAYERS),
        ("w", ctypes.c_void_p * MAX_LAYERS),
        ("rho_star", ctypes.c_void_p),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    from . import build as _build

    return _build.LIB


def library():
    """Load (building in-tree if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        path = _build.build()  # no-op when the in-tree build is up to date
        lib = ctypes.CDLL(path)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        psz, pd = ctypes.POINTER(sz), ctypes.POINTER(d)
        sig = {
            "mera_version": ([], ctypes.c_char_p),
            "mera_last_error": ([], ctypes.c_char_p),
            "mera_workspace_size": ([i, i, i, i, psz], i),
            "mera_ascend": ([vp, vp, vp, i, i, vp, i, vp, sz, vp], i),
            "mera_descend": ([vp, vp, vp, i, i, vp, i, vp, sz, vp], i),
            "mera_fixed_point_rho": ([vp, vp, i, vp, i, vp, i, vp, sz, vp], i),
            "mera_env_u": ([vp, vp, vp, vp, i, i, vp, i, vp, sz, vp], i),
            "mera_env_w": ([vp, vp, vp, vp, i, i, vp, i, vp, sz, vp], i),
            "mera_polar_update": ([vp, i, i, vp, i, d, vp, sz, vp], i),
            "mera_polar_workspace_size": ([i, i, psz], i),
            "mera_energy": ([vp, vp, vp, vp, i, i, vp, i, vp, sz, vp], i),
            "mera_ising_h1": ([d, vp, pd], i),
            "mera_sweep": ([ctypes.POINTER(_State), vp, d, i, i, vp, sz, vp, vp], i),
            "mera_sweep_workspace_size": ([i, ctypes.POINTER(i), ctypes.POINTER(i), i, psz], i),
            "mera_plan_json": ([i, i, i, i, ctypes.c_char_p, sz, psz], i),
            "mera_flops": ([i, i, i, pd], i),
            "mera_launch_count": ([], ctypes.c_longlong),
            "mera_device_status": ([ctypes.POINTER(i), i], i),
            "mera_gemm_test": ([i, vp, vp, i, i, i, vp, vp, sz, vp], i),
            "mera_ascend_noalloc": ([vp, vp, vp, i, i, vp, i, vp], i),
            "mera_op_transpose": ([vp, i, vp, vp], i),
            "mera_energy_adjoint": ([vp, vp, vp, vp, i, i, vp, vp, vp, vp, vp, i, vp, sz, vp], i),
            "mera_set_slice_bytes": ([sz], i),
            "mera_sweep_graph_create": ([ctypes.POINTER(_State), vp, d, i, i, vp, sz, vp, vp, ctypes.POINTER(vp)], i),
            "mera_graph_launch": ([vp, vp], i),
            "mera_sweep_host": ([ctypes.POINTER(_State), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp, d, i, i,
                                 vp, sz, vp, vp, vp, vp], i),
            "mera_graph_destroy": ([vp], i),
            "mera_stiefel_workspace_size": ([i, i, ctypes.POINTER(sz)], i),
            "mera_stiefel_step": ([vp, vp, i, i, d, vp, vp, sz, vp], i),
            "mera_sweep_riemannian": ([ctypes.POINTER(_State), vp, d, i, i, d, vp, sz, vp, vp], i),
            "mera_autotune": ([i, i, i, i, vp, sz, vp, sz, vp, ctypes.POINTER(i)], i),
            "mera_autotune_reset": ([], i),
            "mera_set_tile_width": ([i, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, i, i], i),
            "mera_tile_widths": ([ctypes.POINTER(ctypes.c_longlong), i, ctypes.POINTER(i)], i),
            "mera_sweep_batch": ([ctypes.POINTER(_State), i, ctypes.POINTER(vp), ctypes.POINTER(d), i, i,
                                  ctypes.POINTER(vp), ctypes.POINTER(sz), vp, ctypes.POINTER(vp), i], i),
            "mera_batch_lanes": ([i, i, ctypes.POINTER(i), ctypes.POINTER(i), i, i, sz, i, ctypes.POINTER(i),
                                  ctypes.POINTER(i), psz], i),
            "mera_profile_enable": ([i], i),
            "mera_profile_read": ([i, ctypes.POINTER(ctypes.c_longlong), pd, pd], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int):
    if status == _OK:
        return
    msg = library().mera_last_error().decode(errors="replace")
    if status == _ENOTCONV:
        raise MeraNotConverged(status, msg)
    raise MeraError(status, msg)


def _dev(t, numel=None, name="tensor"):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t, numel, name):
    import torch

    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    return _dev(t, numel, name)


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream))


def _ws(ws):
    if ws is None:
        return ctypes.c_void_p(0), 0
    return ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size()


def mera_version() -> str:
    return library().mera_version().decode()


def mera_workspace_size(op: int, chi_b: int, chi_t: int, prec: int) -> int:
    n = ctypes.c_size_t(0)
    _check(library().mera_workspace_size(op, chi_b, chi_t, prec, ctypes.byref(n)))
    return n.value


def workspace(nbytes: int, device=None):
    """A 256-byte aligned device scratch buffer of at least nbytes."""
    import torch

    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def _auto_ws(ws, op, chi_b, chi_t, prec, device):
    if ws is not None:
        return ws
    return workspace(mera_workspace_size(op, chi_b, chi_t, prec), device)


def mera_ascend(h, u, w, chi_b, chi_t, out, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_ASCEND, chi_b, chi_t, prec, h.device)
    p, n = _ws(ws)
    _check(library().mera_ascend(_f64(h, chi_b ** 6, "h"), _f64(u, chi_b ** 4, "u"), _f64(w, chi_b ** 2 * chi_t, "w"),
                                 chi_b, chi_t, _f64(out, chi_t ** 6, "out"), prec, p, n, _stream(stream)))
    return out


def mera_descend(rho, u, w, chi_b, chi_t, out, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_DESCEND, chi_b, chi_t, prec, rho.device)
    p, n = _ws(ws)
    _check(library().mera_descend(_f64(rho, chi_t ** 6, "rho"), _f64(u, chi_b ** 4, "u"),
                                  _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t, _f64(out, chi_b ** 6, "out"), prec,
                                  p, n, _stream(stream)))
    return out


def mera_fixed_point_rho(u, w, chi, rho_inout, n_iter, resid=None, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_FIXED_POINT, chi, chi, prec, u.device)
    p, n = _ws(ws)
    _check(library().mera_fixed_point_rho(_f64(u, chi ** 4, "u"), _f64(w, chi ** 3, "w"), chi,
                                          _f64(rho_inout, chi ** 6, "rho"), n_iter,
                                          _f64(resid, 1, "resid") if resid is not None else None, prec, p, n,
                                          _stream(stream)))
    return rho_inout


def mera_env_u(h, rho, u, w, chi_b, chi_t, out, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_ENV_U, chi_b, chi_t, prec, h.device)
    p, n = _ws(ws)
    _check(library().mera_env_u(_f64(h, chi_b ** 6, "h"), _f64(rho, chi_t ** 6, "rho"), _f64(u, chi_b ** 4, "u"),
                                _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t, _f64(out, chi_b ** 4, "out"), prec, p,
                                n, _stream(stream)))
    return out


def mera_env_w(h, rho, u, w, chi_b, chi_t, out, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_ENV_W, chi_b, chi_t, prec, h.device)
    p, n = _ws(ws)
    _check(library().mera_env_w(_f64(h, chi_b ** 6, "h"), _f64(rho, chi_t ** 6, "rho"), _f64(u, chi_b ** 4, "u"),
                                _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t, _f64(out, chi_b ** 2 * chi_t, "out"),
                                prec, p, n, _stream(stream)))
    return out


def mera_polar_workspace_size(m: int, n: int) -> int:
    b = ctypes.c_size_t(0)
    _check(library().mera_polar_workspace_size(m, n, ctypes.byref(b)))
    return b.value


def mera_polar_update(env, m, n, out, max_iter=0, tol=0.0, ws=None, stream=None):
    if ws is None:
        ws = workspace(mera_polar_workspace_size(m, n), env.device)
    p, nb = _ws(ws)
    _check(library().mera_polar_update(_f64(env, m * n, "env"), m, n, _f64(out, m * n, "out"), max_iter, tol, p, nb,
                                       _stream(stream)))
    return out


def mera_energy(h, rho, u, w, chi_b, chi_t, e_out, prec=PREC_F64, ws=None, stream=None):
    ws = _auto_ws(ws, OP_ENERGY, chi_b, chi_t, prec, h.device)
    p, n = _ws(ws)
    _check(library().mera_energy(_f64(h, chi_b ** 6, "h"), _f64(rho, chi_t ** 6, "rho"), _f64(u, chi_b ** 4, "u"),
                                 _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t, _f64(e_out, 1, "e_out"), prec, p, n,
                                 _stream(stream)))
    return e_out


def mera_ising_h1(hz: float = 1.0):
    """Host (numpy) [4]*6 shifted blocked Ising density and its shift."""
    import numpy as np

    h1 = np.zeros(4 ** 6, dtype=np.float64)
    s = ctypes.c_double(0.0)
    _check(library().mera_ising_h1(float(hz), h1.ctypes.data_as(ctypes.c_void_p), ctypes.byref(s)))
    return h1.reshape((4,) * 6), s.value


def mera_plan_json(op: int, chi_b: int, chi_t: int, prec: int = PREC_F64) -> dict:
    lib = library()
    n = ctypes.c_size_t(0)
    _check(lib.mera_plan_json(op, chi_b, chi_t, prec, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib.mera_plan_json(op, chi_b, chi_t, prec, buf, n.value + 1, ctypes.byref(n)))
    return json.loads(buf.value.decode())


def mera_flops(op: int, chi_b: int, chi_t: int) -> float:
    f = ctypes.c_double(0.0)
    _check(library().mera_flops(op, chi_b, chi_t, ctypes.byref(f)))
    return f.value


class MeraState:
    """Device tensors of one MERA (layers bottom first) for :func:`mera_sweep`."""

    def __init__(self, us, ws, rho_star):
        self.us, self.ws, self.rho_star = list(us), list(ws), rho_star
        self.chi_b = [int(round(w.shape[0])) for w in self.ws]
        self.chi_t = [int(w.shape[2]) for w in self.ws]

    def _c(self):
        st = _State()
        st.n_layers = len(self.us)
        for k, (u, w) in enumerate(zip(self.us, self.ws)):
            st.chi_b[k] = self.chi_b[k]
            st.chi_t[k] = self.chi_t[k]
            st.u[k] = _f64(u, self.chi_b[k] ** 4, "u").value
            st.w[k] = _f64(w, self.chi_b[k] ** 2 * self.chi_t[k], "w").value
        st.rho_star = _f64(self.rho_star, self.chi_t[-1] ** 6, "rho_star").value
        return st


def mera_sweep_workspace_size(chi_b, chi_t, prec) -> int:
    n = len(chi_b)
    cb = (ctypes.c_int * n)(*chi_b)
    ct = (ctypes.c_int * n)(*chi_t)
    b = ctypes.c_size_t(0)
    _check(library().mera_sweep_workspace_size(n, cb, ct, prec, ctypes.byref(b)))
    return b.value


def mera_sweep(state: MeraState, h1, shift, n_pow, e_out, prec=PREC_F64, ws=None, stream=None):
    if ws is None:
        ws = workspace(mera_sweep_workspace_size(state.chi_b, state.chi_t, prec), h1.device)
    p, n = _ws(ws)
    st = state._c()
    _check(library().mera_sweep(ctypes.byref(st), _f64(h1, state.chi_b[0] ** 6, "h1"), float(shift), n_pow, prec, p,
                                n, _f64(e_out, 1, "e_out"), _stream(stream)))
    return e_out


def mera_sweep_host(state: MeraState, us_host, ws_host, rho_host, h1_host, h1, shift, n_pow, e_dev, e_host,
                    prec=PREC_F64, ws=None, graph=None, stream=None):
    """One sweep with the inputs taken from host tensors (pinned CPU float64
    tensors: u and w of every layer, rho*, h1) copied into `state` and `h1`
    (device) on the stream, the energy copied back into e_host (a pinned
    one-element CPU tensor).  graph: a MeraGraph recorded on these device
    buffers, replayed instead of a direct sweep."""
    if graph is None and ws is None:
        ws = workspace(mera_sweep_workspace_size(state.chi_b, state.chi_t, prec), h1.device)
    p, n = _ws(ws) if ws is not None else (None, 0)
    st = state._c()

    def host_ptr(t, numel, name):
        if t.element_size() != 8 or t.is_cuda or not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name}: a contiguous CPU float64 tensor of {numel} elements is needed")
        return ctypes.c_void_p(t.data_ptr())

    nl = len(state.us)
    ups = (ctypes.c_void_p * nl)(*[host_ptr(t, state.chi_b[k] ** 4, f"u[{k}]") for k, t in enumerate(us_host)])
    wps = (ctypes.c_void_p * nl)(*[host_ptr(t, state.chi_b[k] ** 2 * state.chi_t[k], f"w[{k}]")
                                   for k, t in enumerate(ws_host)])
    _check(library().mera_sweep_host(
        ctypes.byref(st), ups, wps, host_ptr(rho_host, state.chi_t[-1] ** 6, "rho"),
        host_ptr(h1_host, state.chi_b[0] ** 6, "h1"), _f64(h1, state.chi_b[0] ** 6, "h1_dev"), float(shift), n_pow,
        prec, p, n, _f64(e_dev, 1, "e_dev"), host_ptr(e_host, 1, "e_host"),
        graph._h if graph is not None else None, _stream(stream)))


class MeraGraph:
    """A sweep recorded as a CUDA graph (mera_sweep_graph_create).  Keeps the
    recorded buffers alive; launch() replays the sweep on any stream."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        if self._h is None:
            raise MeraError(1, "graph destroyed")
        _check(library().mera_graph_launch(self._h, _stream(stream)))

    def close(self):
        if self._h is not None:
            library().mera_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mera_sweep_graph(state: MeraState, h1, shift, n_pow, e_out, prec=PREC_F64, ws=None, stream=None) -> MeraGraph:
    """Record one mera_sweep into a CUDA graph (nothing is computed).  `stream`
    must be a torch.cuda.Stream other than the legacy default stream."""
    if stream is None:
        raise MeraError(1, "graph capture needs a non-default stream")
    if ws is None:
        ws = workspace(mera_sweep_workspace_size(state.chi_b, state.chi_t, prec), h1.device)
    p, n = _ws(ws)
    st = state._c()
    h = ctypes.c_void_p()
    _check(library().mera_sweep_graph_create(ctypes.byref(st), _f64(h1, state.chi_b[0] ** 6, "h1"), float(shift),
                                             n_pow, prec, p, n, _f64(e_out, 1, "e_out"), _stream(stream),
                                             ctypes.byref(h)))
    return MeraGraph(h, (state, h1, e_out, ws))


def mera_stiefel_workspace_size(m: int, n: int) -> int:
    out = ctypes.c_size_t()
    _check(library().mera_stiefel_workspace_size(m, n, ctypes.byref(out)))
    return out.value


def mera_stiefel_step(x, g, m, n, eta, out, ws=None, stream=None):
    """out = polar(X - eta (G - X sym(X^T G))) for an m x n isometry X."""
    if ws is None:
        ws = workspace(mera_stiefel_workspace_size(m, n), x.device)
    p, nb = _ws(ws)
    _check(library().mera_stiefel_step(_f64(x, m * n, "x"), _f64(g, m * n, "g"), m, n, float(eta),
                                       _f64(out, m * n, "out"), p, nb, _stream(stream)))
    return out


def mera_sweep_riemannian(state: MeraState, h1, shift, n_pow, eta, e_out, prec=PREC_F64, ws=None, stream=None):
    """mera_sweep with Riemannian gradient steps of size eta instead of polar updates."""
    if ws is None:
        ws = workspace(mera_sweep_workspace_size(state.chi_b, state.chi_t, prec), h1.device)
    p, n = _ws(ws)
    st = state._c()
    _check(library().mera_sweep_riemannian(ctypes.byref(st), _f64(h1, state.chi_b[0] ** 6, "h1"), float(shift), n_pow,
                                           prec, float(eta), p, n, _f64(e_out, 1, "e_out"), _stream(stream)))
    return e_out


def mera_autotune(op: int, chi_b: int, chi_t: int, prec: int, device=None, stream=None) -> int:
    """Time the tile widths of op's GEMM steps and record the fastest
    (mera_autotune); returns the number of step shapes recorded."""
    import torch

    dev = device if device is not None else torch.device("cuda")
    ws = workspace(mera_workspace_size(op, chi_b, chi_t, prec), dev)
    n_out = {OP_ASCEND: chi_t ** 6, OP_DESCEND: chi_b ** 6, OP_ENV_U: chi_b ** 4, OP_ENV_W: chi_b ** 2 * chi_t}[op]
    out = torch.empty(n_out, dtype=torch.float64, device=dev)
    p, nb = _ws(ws)
    n = ctypes.c_int(0)
    _check(library().mera_autotune(op, chi_b, chi_t, prec, _f64(out, n_out, "out"), n_out, p, nb, _stream(stream),
                                   ctypes.byref(n)))
    return n.value


def mera_autotune_reset() -> None:
    _check(library().mera_autotune_reset())


def mera_set_tile_width(prec: int, M: int, N: int, K: int, c_final: bool, bn: int) -> None:
    """Record tile width bn for a GEMM shape without timing (0 forgets it)."""
    _check(library().mera_set_tile_width(prec, M, N, K, int(bool(c_final)), bn))


def mera_tile_widths() -> list:
    """Every recorded width as (prec, M, N, K, c_final, width)."""
    n = ctypes.c_int(0)
    _check(library().mera_tile_widths(None, 0, ctypes.byref(n)))
    buf = (ctypes.c_longlong * (6 * max(n.value, 1)))()
    _check(library().mera_tile_widths(buf, n.value, ctypes.byref(n)))
    return [tuple(int(x) for x in buf[6 * k:6 * k + 6]) for k in range(n.value)]


def mera_launch_count() -> int:
    return int(library().mera_launch_count())


def mera_profile_enable(on: bool = True) -> None:
    _check(library().mera_profile_enable(1 if on else 0))


def mera_profile_read(kind: int = PROF_GEMM):
    """(launches, device ms, algorithmic flops) since profiling was enabled."""
    n, ms, fl = ctypes.c_longlong(0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(library().mera_profile_read(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl)))
    return n.value, ms.value, fl.value


def mera_device_status(clear: bool = True) -> int:
    """Device failure bits: 1 << MERA_ETIMEOUT (a bounded wait timed out),
    1 << MERA_ENOTCONV (a polar update recorded in a graph did not converge).
    Synchronises with the device."""
    st = ctypes.c_int(0)
    _check(library().mera_device_status(ctypes.byref(st), 1 if clear else 0))
    return st.value


def mera_gemm_test(prec, A, B, C, stream=None):
    """C = A @ B.T through the library's GEMM kernel of mode prec (test hook)."""
    M, K = A.shape
    N = B.shape[0]
    eb = 8 if prec == PREC_F64 else (4 if prec == PREC_TF32 else 2)
    ld = (K * eb + 15) // 16 * 16 // eb
    pad = lambda x: (x + 255) // 256 * 256  # noqa: E731
    planes = {PREC_BF16X3: 2, PREC_BF16X6: 3, PREC_OZ3: 3, PREC_OZ4: 4}.get(prec, 1)
    raw = 2 * (pad(M * ld * 4) + pad(N * ld * 4)) if prec in (PREC_OZ3, PREC_OZ4) else 0
    ws = workspace(planes * (pad(M * ld * eb) + pad(N * ld * eb)) + raw, A.device)
    p, n = _ws(ws)
    _check(library().mera_gemm_test(prec, _f64(A, M * K, "A"), _f64(B, N * K, "B"), M, N, K, _f64(C, M * N, "C"),
                                    p, n, _stream(stream)))
    return C


def mera_ascend_noalloc(h, u, w, chi_b, chi_t, out, prec=PREC_F64, stream=None):
    """mera_ascend with the library's static device scratch (no workspace).

    For callers that cannot allocate scratch memory; sizes needing more than
    NOALLOC_SCRATCH_BYTES of scratch raise MeraError.  Calls share the
    scratch, so calls that overlap on the GPU must not be issued."""
    _check(library().mera_ascend_noalloc(_f64(h, chi_b ** 6, "h"), _f64(u, chi_b ** 4, "u"),
                                         _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t,
                                         _f64(out, chi_t ** 6, "out"), prec, _stream(stream)))
    return out


def mera_op_transpose(x, d, out, stream=None):
    """out[I, J] = x[J, I] for a 3-site operator of local dimension d."""
    _check(library().mera_op_transpose(_f64(x, d ** 6, "x"), d, _f64(out, d ** 6, "out"), _stream(stream)))
    return out


def mera_energy_adjoint(h, rho, u, w, chi_b, chi_t, g, dh=None, drho=None, du=None, dw=None, prec=PREC_F64,
                        ws=None, stream=None):
    """Gradients of tr(A(h) rho) times the upstream gradient g (a one-element
    device tensor): any of dh [chi_b^6], drho [chi_t^6], du [chi_b^4],
    dw [chi_b^2 chi_t] that is given is written."""
    ws = _auto_ws(ws, OP_ENERGY_ADJOINT, chi_b, chi_t, prec, h.device)
    p, n = _ws(ws)
    opt = lambda t, k, name: None if t is None else _f64(t, k, name)  # noqa: E731
    _check(library().mera_energy_adjoint(
        _f64(h, chi_b ** 6, "h"), _f64(rho, chi_t ** 6, "rho"), _f64(u, chi_b ** 4, "u"),
        _f64(w, chi_b ** 2 * chi_t, "w"), chi_b, chi_t, _f64(g, 1, "g"), opt(dh, chi_b ** 6, "dh"),
        opt(drho, chi_t ** 6, "drho"), opt(du, chi_b ** 4, "du"), opt(dw, chi_b ** 2 * chi_t, "dw"), prec, p, n,
        _stream(stream)))


def mera_sweep_batch(states, h1s, shifts, n_pow, e_out, prec=PREC_F64, wss=None, streams=None, n_threads=8):
    """One sweep of each of several independent MERAs, run concurrently.

    states: list of MeraState; h1s: device h1 per MERA; shifts: floats;
    e_out: device float64 tensor with one slot per MERA; wss: scratch per
    MERA (allocated when None); streams: a torch.cuda.Stream per MERA.  MERAs
    given the same stream run one after another and may share scratch
    (batch_resources makes such lanes under a memory budget)."""
    import torch

    n = len(states)
    if wss is None:
        wss = [workspace(mera_sweep_workspace_size(s.chi_b, s.chi_t, prec), e_out.device) for s in states]
    if streams is None:
        streams = [torch.cuda.Stream(device=e_out.device) for _ in range(n)]
    arr = (_State * n)(*[s._c() for s in states])
    h_arr = (ctypes.c_void_p * n)(*[_f64(h, s.chi_b[0] ** 6, "h1").value for h, s in zip(h1s, states)])
    sh_arr = (ctypes.c_double * n)(*[float(x) for x in shifts])
    ws_arr = (ctypes.c_void_p * n)(*[w.data_ptr() for w in wss])
    wb_arr = (ctypes.c_size_t * n)(*[w.numel() * w.element_size() for w in wss])
    st_arr = (ctypes.c_void_p * n)(*[int(s.cuda_stream) for s in streams])
    # the batch's streams must see the caller's pending work on the inputs
    cur = torch.cuda.current_stream(e_out.device)
    for s in streams:
        s.wait_stream(cur)
    _check(library().mera_sweep_batch(arr, n, h_arr, sh_arr, n_pow, prec, ws_arr, wb_arr,
                                      _f64(e_out, n, "e_out"), st_arr, n_threads))
    for s in streams:
        cur.wait_stream(s)
    return e_out


def mera_batch_lanes(dims, prec, budget_bytes, max_lanes=32, n_pow=20):
    """Lanes of a batch under a scratch budget (mera_batch_lanes).

    dims: one (chi_b list, chi_t list) per MERA, all with the same number of
    layers.  Returns (lane of each MERA, scratch bytes of each lane)."""
    n = len(dims)
    n_layers = len(dims[0][0])
    if any(len(b) != n_layers or len(t) != n_layers for b, t in dims):
        raise ValueError("every MERA of a batch needs the same number of layers")
    cb = (ctypes.c_int * (n * n_layers))(*[x for b, _ in dims for x in b])
    ct = (ctypes.c_int * (n * n_layers))(*[x for _, t in dims for x in t])
    lane = (ctypes.c_int * n)()
    lane_bytes = (ctypes.c_size_t * n)()
    n_lanes = ctypes.c_int(0)
    _check(library().mera_batch_lanes(n, n_layers, cb, ct, prec, n_pow, int(budget_bytes), max_lanes, lane,
                                      ctypes.byref(n_lanes), lane_bytes))
    return list(lane), [int(lane_bytes[k]) for k in range(n_lanes.value)]


def batch_resources(states, prec, budget_bytes, max_lanes=32, n_pow=20, device=None):
    """Scratch and streams for mera_sweep_batch under a memory budget: one
    buffer and one stream per lane of mera_batch_lanes, shared by the lane's
    MERAs.  Returns (wss, streams), one entry per MERA."""
    import torch

    dev = device if device is not None else torch.device("cuda")
    lanes, lane_bytes = mera_batch_lanes([(s.chi_b, s.chi_t) for s in states], prec, budget_bytes, max_lanes, n_pow)
    bufs = [workspace(b, dev) for b in lane_bytes]
    strs = [torch.cuda.Stream(device=dev) for _ in lane_bytes]
    return [bufs[k] for k in lanes], [strs[k] for k in lanes]


def mera_set_slice_bytes(nbytes: int) -> None:
    """Slice rank-7 intermediates larger than nbytes (default 16 GiB)."""
    _check(library().mera_set_slice_bytes(int(nbytes)))
