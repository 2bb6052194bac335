"""GB300-native stage-1 tables of the Gaussian boson sampling emulator of
arXiv:2511.14923: vacuum probabilities, click moments and click cumulants of a
zero-mean Gaussian state over every mode subset of size <= kmax <= 5.

This module is a thin ctypes binding over ``libgbs.so`` (C ABI in
``include/gbs.h``): it checks tensor arguments, allocates outputs and the
workspace through PyTorch (device memory and streams only) and calls the
library. Every step of the computation runs in the library's CUDA kernels; if
the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from math import comb

import torch

__all__ = [
    "GbsError", "lib", "build", "table_size", "order_offset", "rank", "unrank", "workspace_bytes",
    "Workspace", "vacuum_probs", "click_moments", "cumulants", "PRECISIONS", "cumulants_backward",
    "spin_correlators", "spin_cumulants",
    "covariance", "covariance_backward", "CumulantFn", "CovarianceFn", "fit_weights", "Batch",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgbs.so")
_lib = None

PRECISIONS = {"fp64": 0, "fp32r": 1}
STATUS = {0: "GBS_OK", 1: "GBS_ERR_INVALID_ARG", 2: "GBS_ERR_NOT_POSDEF", 3: "GBS_ERR_CUDA",
          4: "GBS_ERR_TIMEOUT", 5: "GBS_ERR_WORKSPACE"}


class GbsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


class _Instance(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("kappa_out", ctypes.c_void_p), ("M", ctypes.c_int), ("kmax", ctypes.c_int)]


def lib() -> ctypes.CDLL:
    """The loaded libgbs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2511_14923_gb300.build() "
                          "(nvcc, sm_103a); there is no fallback implementation")
    L = ctypes.CDLL(_LIB_PATH)
    u64, i32, vp, sz = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    L.gbs_table_size.argtypes = [i32, i32]; L.gbs_table_size.restype = u64
    L.gbs_order_offset.argtypes = [i32, i32]; L.gbs_order_offset.restype = u64
    L.gbs_rank.argtypes = [ctypes.POINTER(i32), i32]; L.gbs_rank.restype = u64
    L.gbs_unrank.argtypes = [u64, i32, ctypes.POINTER(i32)]; L.gbs_unrank.restype = i32
    L.gbs_workspace_bytes.argtypes = [i32, i32, i32]; L.gbs_workspace_bytes.restype = sz
    L.gbs_last_error.argtypes = []; L.gbs_last_error.restype = ctypes.c_char_p
    L.gbs_stream_status.argtypes = [vp, vp]; L.gbs_stream_status.restype = i32
    L.gbs_status_code.argtypes = [ctypes.c_uint]; L.gbs_status_code.restype = i32
    L.gbs_autotune.argtypes = [vp, i32, i32, vp, i32, vp, sz, vp, ctypes.POINTER(ctypes.c_float)]
    L.gbs_autotune.restype = i32
    L.gbs_schedule.argtypes = [i32, i32, i32, ctypes.POINTER(i32)]; L.gbs_schedule.restype = i32
    L.gbs_timing.argtypes = [i32]; L.gbs_timing.restype = i32
    L.gbs_timing_read.argtypes = [ctypes.POINTER(ctypes.c_float)]; L.gbs_timing_read.restype = i32
    L.gbs_timing_read_backward.argtypes = [ctypes.POINTER(ctypes.c_float)]
    L.gbs_timing_read_backward.restype = i32
    L.gbs_pipe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), vp, vp]; L.gbs_pipe_peaks.restype = i32
    L.gbs_backward_workspace_bytes.argtypes = [i32, i32]; L.gbs_backward_workspace_bytes.restype = sz
    L.gbs_cumulants_backward.argtypes = [vp, i32, i32, vp, vp, vp, sz, vp]; L.gbs_cumulants_backward.restype = i32
    L.gbs_covariance.argtypes = [vp, vp, vp, vp, i32, vp, vp]; L.gbs_covariance.restype = i32
    L.gbs_covariance_backward.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.gbs_covariance_backward.restype = i32
    L.gbs_batched_workspace_bytes.argtypes = [ctypes.POINTER(_Instance), i32, i32]
    L.gbs_batched_workspace_bytes.restype = sz
    L.gbs_batched_plan.argtypes = [ctypes.POINTER(_Instance), i32, i32, vp, sz, vp]; L.gbs_batched_plan.restype = i32
    L.gbs_cumulants_batched.argtypes = [i32, vp, vp]; L.gbs_cumulants_batched.restype = i32
    L.gbs_batched_autotune.argtypes = [ctypes.POINTER(_Instance), i32, i32, vp, sz, vp, ctypes.POINTER(ctypes.c_float)]
    L.gbs_batched_autotune.restype = i32
    L.gbs_batched_schedule.argtypes = [vp, ctypes.POINTER(i32)]; L.gbs_batched_schedule.restype = i32
    for name in ("gbs_vacuum_probs", "gbs_click_moments", "gbs_cumulants", "gbs_spin_correlators",
                 "gbs_spin_cumulants"):
        f = getattr(L, name)
        f.argtypes = [vp, i32, i32, vp, i32, vp, sz, vp]
        f.restype = i32
    L.gbs_sampler_workspace_bytes.argtypes = [i32, i32, i32, i32]; L.gbs_sampler_workspace_bytes.restype = sz
    L.gbs_sample.argtypes = [vp, i32, i32, ctypes.POINTER(i32), i32, vp, vp, vp, vp, vp, i32, i32, vp, sz, vp]
    L.gbs_sample.restype = i32
    L.gbs_displaced_tables.argtypes = [vp, vp, i32, i32, i32, vp, vp, sz, vp]
    L.gbs_displaced_tables.restype = i32
    L.gbs_range_workspace_bytes.argtypes = [i32, i32, i32]; L.gbs_range_workspace_bytes.restype = sz
    L.gbs_range_entries.argtypes = [i32, i32, i32, i32]; L.gbs_range_entries.restype = u64
    L.gbs_range_split.argtypes = [i32, i32, i32, ctypes.POINTER(i32)]; L.gbs_range_split.restype = i32
    L.gbs_table_range.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp, sz, vp]
    L.gbs_table_range.restype = i32
    L.gbs_noalloc_status.argtypes = [vp]; L.gbs_noalloc_status.restype = i32
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise GbsError(rc, lib().gbs_last_error().decode())


# Deferred device-status checks (check="defer"): the call's status word is copied
# to pinned host memory on its stream (no synchronisation) and read once that
# copy has completed -- at the next library call from this process, or in
# check_pending(). Entries: (event after the copy, pinned int32[1], call name).
_pending: list = []


def _defer_status(ws: torch.Tensor, stream, what: str):
    """Queue the status word (first 4 bytes of the workspace tensor ws) for a
    deferred check, after raising for any earlier deferred call that failed."""
    check_pending(wait=False)
    word = ws.reshape(-1).view(torch.uint8)[:4].view(torch.int32)
    host = torch.empty(1, dtype=torch.int32, pin_memory=True)
    with torch.cuda.stream(stream):
        host.copy_(word, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(stream)
    _pending.append((ev, host, what))


def check_pending(wait: bool = True):
    """Raise GbsError for the first failed call among those queued with
    check="defer" whose status word has arrived (with wait=True, after waiting
    for every queued copy). Calls whose status has been read are dropped."""
    global _pending
    keep, failed = [], None
    for ev, host, what in _pending:
        if wait:
            ev.synchronize()
        if not ev.query():
            keep.append((ev, host, what))
            continue
        if failed is None:
            rc = int(lib().gbs_status_code(ctypes.c_uint(int(host.item()) & 0xFFFFFFFF)))
            if rc != 0:
                failed = GbsError(rc, f"{what}: " + lib().gbs_last_error().decode())
    _pending = keep
    if failed is not None:
        raise failed


def table_size(M: int, kmax: int) -> int:
    return int(lib().gbs_table_size(M, kmax))


def order_offset(M: int, d: int) -> int:
    return int(lib().gbs_order_offset(M, d))


def rank(modes) -> int:
    arr = (ctypes.c_int * len(modes))(*[int(m) for m in modes])
    return int(lib().gbs_rank(arr, len(modes)))


def unrank(r: int, d: int) -> list[int]:
    arr = (ctypes.c_int * d)()
    _check(lib().gbs_unrank(r, d, arr))
    return list(arr)


def workspace_bytes(M: int, kmax: int, precision: str = "fp64") -> int:
    return int(lib().gbs_workspace_bytes(M, kmax, PRECISIONS[precision]))


class Workspace:
    """Device workspace sized for (M, kmax, precision); reusable across calls on one stream."""

    def __init__(self, M: int, kmax: int, precision: str = "fp64", device=None):
        n = workspace_bytes(M, kmax, precision)
        if n == 0:
            raise GbsError(1, f"invalid (M={M}, kmax={kmax}, precision={precision})")
        dev = torch.device(device or "cuda")
        if dev.type != "cuda":
            raise TypeError("the workspace lives in device memory (a CUDA device)")
        self.buf = torch.empty(n, dtype=torch.uint8, device=dev)
        self.nbytes = n

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def status(self, stream=None) -> int:
        st = stream or torch.cuda.current_stream(self.buf.device)
        return int(lib().gbs_stream_status(ctypes.c_void_p(self.ptr), ctypes.c_void_p(st.cuda_stream)))


def _workspace_for(workspace, M: int, kmax: int, precision: str, device) -> Workspace:
    """The caller's Workspace after checking that it sits on the inputs' device and
    is large enough for (M, kmax, precision), or a new one."""
    if workspace is None:
        return Workspace(M, kmax, precision, device=device)
    if not isinstance(workspace, Workspace):
        raise TypeError("workspace must be a Workspace")
    if workspace.buf.device != torch.device(device):
        raise ValueError(f"workspace is on {workspace.buf.device}, the inputs on {device}")
    need = workspace_bytes(M, kmax, precision)
    if workspace.nbytes < need:
        raise GbsError(5, f"workspace holds {workspace.nbytes} bytes, (M={M}, kmax={kmax}, {precision}) needs {need}")
    return workspace


def _workspace_tensor(workspace, need: int, device) -> torch.Tensor:
    """A raw device workspace: the caller's contiguous CUDA tensor on the inputs'
    device with at least need bytes, or a new uint8 tensor."""
    if workspace is None:
        return torch.empty(need, dtype=torch.uint8, device=device)
    if not isinstance(workspace, torch.Tensor) or not workspace.is_cuda:
        raise TypeError("workspace must be a CUDA tensor")
    if workspace.device != torch.device(device):
        raise ValueError(f"workspace is on {workspace.device}, the inputs on {device}")
    if not workspace.is_contiguous():
        raise ValueError("workspace must be contiguous")
    if _nbytes(workspace) < need:
        raise GbsError(5, f"workspace holds {_nbytes(workspace)} bytes, {need} needed")
    return workspace


def _on(t: torch.Tensor, device, name: str) -> torch.Tensor:
    if t.device != torch.device(device):
        raise ValueError(f"{name} is on {t.device}, the other inputs on {device}")
    return t


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def _prep(V: torch.Tensor):
    if not isinstance(V, torch.Tensor) or V.dtype != torch.float64 or not V.is_cuda:
        raise TypeError("V must be a CUDA float64 tensor")
    if V.dim() != 2 or V.shape[0] != V.shape[1] or V.shape[0] % 2:
        raise ValueError("V must be 2M x 2M")
    return V.contiguous(), V.shape[0] // 2


def _forward(fname: str, V: torch.Tensor, kmax: int, precision: str, out, workspace, check):
    """check: True = synchronise and raise on a device error; "defer" = queue the
    status for check_pending(); False = leave it in the workspace."""
    V, M = _prep(V)
    n = table_size(M, kmax)
    if n == 0:
        raise GbsError(1, f"invalid (M={M}, kmax={kmax})")
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=V.device)
    elif out.numel() != n or out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous CUDA float64 tensor of {n} entries")
    _on(out, V.device, "out")
    ws = _workspace_for(workspace, M, kmax, precision, V.device)
    st = torch.cuda.current_stream(V.device)
    f = getattr(lib(), fname)
    _check(f(ctypes.c_void_p(V.data_ptr()), M, kmax, ctypes.c_void_p(out.data_ptr()), PRECISIONS[precision],
             ctypes.c_void_p(ws.ptr), ws.nbytes, ctypes.c_void_p(st.cuda_stream)))
    if check == "defer":
        _defer_status(ws.buf, st, fname)
    elif check:
        _check(ws.status(st))
    return out


def vacuum_probs(V, kmax, precision="fp64", out=None, workspace=None, check=True):
    """P0(S) = det[(V_S + I)/2]^{-1/2} for every 1 <= |S| <= kmax (table layout of gbs.h)."""
    return _forward("gbs_vacuum_probs", V, kmax, precision, out, workspace, check)


def click_moments(V, kmax, precision="fp64", out=None, workspace=None, check=True):
    """mu(S) = probability that every mode of S clicks, for every 1 <= |S| <= kmax."""
    return _forward("gbs_click_moments", V, kmax, precision, out, workspace, check)


def cumulants(V, kmax, precision="fp64", out=None, workspace=None, check=True):
    """Joint click cumulants kt(S) for every 1 <= |S| <= kmax."""
    return _forward("gbs_cumulants", V, kmax, precision, out, workspace, check)


def spin_correlators(V, kmax, precision="fp64", out=None, workspace=None, check=True):
    """Spin correlators c(S) = E[prod (-1)^{x_k}] for every 1 <= |S| <= kmax."""
    return _forward("gbs_spin_correlators", V, kmax, precision, out, workspace, check)


def spin_cumulants(V, kmax, precision="fp64", out=None, workspace=None, check=True):
    """Spin cumulants kappa(S) (the sampler's input table) for every 1 <= |S| <= kmax."""
    return _forward("gbs_spin_cumulants", V, kmax, precision, out, workspace, check)


TABLES = {"p0": 0, "mu": 1, "kappa": 2, "spin_c": 3, "spin_kappa": 4}


def displaced_tables(V, mean, kmax, table="kappa", out=None, workspace=None, check=True):
    """One table ("p0", "mu", "kappa", "spin_c" or "spin_kappa") of a displaced
    Gaussian state with first moments mean (2M, xxpp, hbar = 2), in FP64."""
    V, M = _prep(V)
    if table not in TABLES:
        raise ValueError(f"table must be one of {sorted(TABLES)}")
    mean = _on(_dev64(mean, "mean"), V.device, "mean")
    if mean.numel() != 2 * M:
        raise ValueError(f"mean must have 2M = {2 * M} entries")
    n = table_size(M, kmax)
    if n == 0:
        raise GbsError(1, f"invalid (M={M}, kmax={kmax})")
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=V.device)
    elif out.numel() != n or out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous CUDA float64 tensor of {n} entries")
    _on(out, V.device, "out")
    ws = _workspace_for(workspace, M, kmax, "fp64", V.device)
    st = torch.cuda.current_stream(V.device)
    _check(lib().gbs_displaced_tables(_vp(V), _vp(mean), M, kmax, TABLES[table], _vp(out), ctypes.c_void_p(ws.ptr),
                                      ws.nbytes, ctypes.c_void_p(st.cuda_stream)))
    if check:
        _check(ws.status(st))
    return out


def range_split(M: int, kmax: int, n_parts: int) -> list[int]:
    """Cost-balanced top-element bounds [0 = b_0 <= .. <= b_n = M] of n_parts slices
    of the order-kmax group (gbs_range_split)."""
    arr = (ctypes.c_int * (n_parts + 1))()
    _check(lib().gbs_range_split(M, kmax, n_parts, arr))
    return list(arr)


def range_entries(M: int, kmax: int, c_lo: int, c_hi: int) -> int:
    return int(lib().gbs_range_entries(M, kmax, c_lo, c_hi))


def table_range(V, kmax, c_lo, c_hi, table="kappa", precision="fp64", out=None, workspace=None, check=True):
    """The order-kmax entries of one table ("p0", "mu", "kappa", "spin_c",
    "spin_kappa") whose largest mode lies in [c_lo, c_hi), in colex order
    (gbs_table_range): a contiguous slice of the order-kmax group."""
    V, M = _prep(V)
    if table not in TABLES:
        raise ValueError(f"table must be one of {sorted(TABLES)}")
    if not (0 <= c_lo <= c_hi <= M):
        raise ValueError(f"need 0 <= c_lo <= c_hi <= M = {M}")
    n = range_entries(M, kmax, c_lo, c_hi)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=V.device)
    elif out.numel() < n or out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous CUDA float64 tensor of at least {n} entries")
    _on(out, V.device, "out")
    nb = int(lib().gbs_range_workspace_bytes(M, kmax, PRECISIONS[precision]))
    if nb == 0:
        raise GbsError(1, f"invalid (M={M}, kmax={kmax}, precision={precision})")
    ws = _workspace_tensor(workspace, nb, V.device)
    st = torch.cuda.current_stream(V.device)
    _check(lib().gbs_table_range(_vp(V), M, kmax, TABLES[table], c_lo, c_hi, _vp(out), PRECISIONS[precision], _vp(ws),
                                 _nbytes(ws), ctypes.c_void_p(st.cuda_stream)))
    if check:
        _check(lib().gbs_stream_status(_vp(ws), ctypes.c_void_p(st.cuda_stream)))
    return out[:n]


SAMPLE_PRECISIONS = {"fp64": 0, "fp32": 1}


def sampler_workspace_bytes(M: int, K: int, batch: int, precision: str = "fp32") -> int:
    return int(lib().gbs_sampler_workspace_bytes(M, K, batch, SAMPLE_PRECISIONS[precision]))


def sample(kappa, M: int, K: int, u=None, force=None, orders=None, batch: int = 1024, precision: str = "fp32",
           want_q0: bool = False, workspace=None, check: bool = True):
    """Chain-rule sampler (gbs_sample): bitstrings drawn from the spin-cumulant table
    kappa (CUDA float64, orders 1..K). u: (n, M) CUDA float64 uniforms, or force:
    (n, M) CUDA uint8 bits to score. Returns (bits (n, M) uint8, logp (n,) float64 =
    natural log of each bitstring's estimated probability, q0 (n, M) float64 or
    None)."""
    kappa = _dev64(kappa, "kappa")
    if kappa.numel() != table_size(M, K):
        raise ValueError(f"kappa must hold table_size(M, K) = {table_size(M, K)} entries")
    src = force if force is not None else u
    if src is None:
        raise ValueError("give u or force")
    n = src.shape[0]
    dev = kappa.device
    if u is not None:
        u = _on(_dev64(u, "u"), dev, "u")
        if tuple(u.shape) != (n, M):
            raise ValueError("u must be (n, M)")
    if force is not None:
        if not isinstance(force, torch.Tensor) or not force.is_cuda or force.dtype != torch.uint8:
            raise TypeError("force must be a CUDA uint8 tensor")
        if tuple(force.shape) != (n, M):
            raise ValueError("force must be (n, M)")
        force = _on(force, dev, "force").contiguous()
    bits = torch.empty((n, M), dtype=torch.uint8, device=dev)
    prob = torch.empty(n, dtype=torch.float64, device=dev)
    q0 = torch.empty((n, M), dtype=torch.float64, device=dev) if want_q0 else None
    nb = sampler_workspace_bytes(M, K, batch, precision)
    if nb == 0:
        raise GbsError(1, f"invalid sampler shape (M={M}, K={K}, batch={batch}, precision={precision})")
    ws = _workspace_tensor(workspace, nb, dev)
    ordv = None if orders is None else (ctypes.c_int * 3)(*[int(o) for o in orders])
    st = torch.cuda.current_stream(dev)
    _check(lib().gbs_sample(_vp(kappa), M, K, ordv, n, None if u is None else _vp(u),
                            None if force is None else _vp(force), _vp(bits), _vp(prob),
                            None if q0 is None else _vp(q0), batch, SAMPLE_PRECISIONS[precision], _vp(ws),
                            _nbytes(ws), ctypes.c_void_p(st.cuda_stream)))
    if check:
        _check(lib().gbs_stream_status(_vp(ws), ctypes.c_void_p(st.cuda_stream)))
    return bits, prob, q0


def _vp(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _dev64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    return t.contiguous()


def cumulants_backward(V, kmax, grad_kappa, workspace: torch.Tensor | None = None, check=True):
    """dL/dV (2M x 2M, symmetric) from dL/dkt (table layout); FP64 sums, refined P0
    and double-float inverses (see gbs_cumulants_backward in gbs.h)."""
    V, M = _prep(V)
    g = _on(_dev64(grad_kappa, "grad_kappa"), V.device, "grad_kappa")
    n = table_size(M, kmax)
    if g.numel() != n:
        raise ValueError(f"grad_kappa must have {n} entries")
    nb = int(lib().gbs_backward_workspace_bytes(M, kmax))
    ws = _workspace_tensor(workspace, nb, V.device)
    out = torch.empty_like(V)
    st = torch.cuda.current_stream(V.device)
    _check(lib().gbs_cumulants_backward(_vp(V), M, kmax, _vp(g), _vp(out), _vp(ws), _nbytes(ws),
                                        ctypes.c_void_p(st.cuda_stream)))
    if check == "defer":
        _defer_status(ws, st, "gbs_cumulants_backward")
    elif check:
        _check(lib().gbs_stream_status(_vp(ws), ctypes.c_void_p(st.cuda_stream)))
    return out


def covariance(U: torch.Tensor, r: torch.Tensor, eta: torch.Tensor) -> torch.Tensor:
    """V = D S Q S^T D + I - D^2 for squeezers r, interferometer U (complex M x M)
    and per-mode transmissions eta (all CUDA tensors)."""
    Ur, Ui = U.real.to(torch.float64).contiguous(), U.imag.to(torch.float64).contiguous()
    r, eta = _dev64(r, "r"), _dev64(eta, "eta")
    M = Ur.shape[0]
    V = torch.empty(2 * M, 2 * M, dtype=torch.float64, device=r.device)
    st = torch.cuda.current_stream(r.device)
    _check(lib().gbs_covariance(_vp(Ur), _vp(Ui), _vp(r), _vp(eta), M, _vp(V), ctypes.c_void_p(st.cuda_stream)))
    return V


def covariance_backward(U, r, eta, V, grad_V):
    Ur, Ui = U.real.to(torch.float64).contiguous(), U.imag.to(torch.float64).contiguous()
    r, eta, V, G = _dev64(r, "r"), _dev64(eta, "eta"), _dev64(V, "V"), _dev64(grad_V, "grad_V")
    M = Ur.shape[0]
    dr, de = torch.empty_like(r), torch.empty_like(eta)
    st = torch.cuda.current_stream(r.device)
    _check(lib().gbs_covariance_backward(_vp(Ur), _vp(Ui), _vp(r), _vp(eta), M, _vp(V), _vp(G), _vp(dr), _vp(de),
                                         ctypes.c_void_p(st.cuda_stream)))
    return dr, de


class CumulantFn(torch.autograd.Function):
    """kt = cumulants(V); backward through gbs_cumulants_backward.

    Neither pass synchronises the stream: device errors (a reduced covariance that
    is not positive definite) are checked with check="defer" and raise GbsError at
    a later library call or in check_pending(); the affected entries are NaN."""

    @staticmethod
    def forward(ctx, V, kmax, precision="fp64"):
        ctx.save_for_backward(V)
        ctx.kmax = kmax
        return cumulants(V, kmax, precision, check="defer")

    @staticmethod
    def backward(ctx, g):
        (V,) = ctx.saved_tensors
        return cumulants_backward(V, ctx.kmax, g.contiguous(), check="defer"), None, None


class CovarianceFn(torch.autograd.Function):
    """V = covariance(U, r, eta); gradients flow to r and eta (U is fixed)."""

    @staticmethod
    def forward(ctx, r, eta, U):
        V = covariance(U, r, eta)
        ctx.save_for_backward(r, eta, V)
        ctx.U = U
        return V

    @staticmethod
    def backward(ctx, G):
        r, eta, V = ctx.saved_tensors
        dr, de = covariance_backward(ctx.U, r, eta, V, G.contiguous())
        return dr, de, None


def fit_weights(M: int, kmax: int, device=None) -> torch.Tensor:
    """Per-entry loss weights 1 / C(M, d) (each order weighs the same in total)."""
    return torch.cat([torch.full((comb(M, d),), 1.0 / comb(M, d), dtype=torch.float64, device=device)
                      for d in range(1, kmax + 1)])


class Batch:
    """Ragged batch of click-cumulant tables computed by one persistent launch.

    Vs: list of CUDA float64 2M x 2M covariances (kept by reference: update them
    in place and call run() again, or replay the captured graph); kmaxes: list of
    orders. outputs[i] receives instance i's table. autotune=True times the
    candidate schedules of the batched kernel on this batch (gbs_batched_autotune)
    and keeps the fastest; tune_ms then holds its time."""

    def __init__(self, Vs, kmaxes, precision="fp32r", autotune=False):
        self.Vs = [_prep(V)[0] for V in Vs]
        self.kmaxes = [int(k) for k in kmaxes]
        self.precision = precision
        dev = self.Vs[0].device
        self.outputs = []
        arr = (_Instance * len(self.Vs))()
        for i, (V, k) in enumerate(zip(self.Vs, self.kmaxes)):
            M = V.shape[0] // 2
            n = table_size(M, k)
            if n == 0:
                raise GbsError(1, f"instance {i}: invalid (M={M}, kmax={k})")
            out = torch.empty(n, dtype=torch.float64, device=dev)
            self.outputs.append(out)
            arr[i] = _Instance(V.data_ptr(), out.data_ptr(), M, k)
        self._arr = arr
        nb = int(lib().gbs_batched_workspace_bytes(arr, len(arr), PRECISIONS[precision]))
        if nb == 0:
            raise GbsError(1, lib().gbs_last_error().decode())
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        st = torch.cuda.current_stream(dev)
        _check(lib().gbs_batched_plan(arr, len(arr), PRECISIONS[precision], _vp(self.ws), nb,
                                      ctypes.c_void_p(st.cuda_stream)))
        self.graph = None
        self.tune_ms = None
        if autotune:
            self.autotune()

    def autotune(self) -> float:
        """Pick the batched kernel's schedule for this batch by timing the candidates
        (outputs are overwritten); the plan in the workspace then uses it."""
        st = torch.cuda.current_stream(self.ws.device)
        ms = ctypes.c_float(0.0)
        _check(lib().gbs_batched_autotune(self._arr, len(self._arr), PRECISIONS[self.precision], _vp(self.ws),
                                          _nbytes(self.ws), ctypes.c_void_p(st.cuda_stream), ctypes.byref(ms)))
        self.graph = None
        self.tune_ms = float(ms.value)
        return self.tune_ms

    def schedule(self) -> dict:
        """The batched kernel's schedule in this plan (gbs_batched_schedule)."""
        arr = (ctypes.c_int * 5)()
        _check(lib().gbs_batched_schedule(_vp(self.ws), arr))
        shape = {0: "512x1", 1: "256x2", 2: "640x1", 3: "256x3", 4: "768x1", 5: "384x2", 6: "256x4", 7: "256x4 clusters of 4", 8: "256x3 clusters of 3"}.get(arr[0], str(arr[0]))
        return {"cta_shape": shape, "threads": arr[1], "ctas": arr[2], "grain": arr[3], "children_per_batch": arr[4]}

    def run(self, check=False):
        st = torch.cuda.current_stream(self.ws.device)
        _check(lib().gbs_cumulants_batched(PRECISIONS[self.precision], _vp(self.ws), ctypes.c_void_p(st.cuda_stream)))
        if check:
            _check(lib().gbs_stream_status(_vp(self.ws), ctypes.c_void_p(st.cuda_stream)))
        return self.outputs

    def capture(self):
        """Capture run() in a CUDA graph (after one eager warm-up run)."""
        self.run()
        torch.cuda.synchronize(self.ws.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.ws.device)
        s.wait_stream(torch.cuda.current_stream(self.ws.device))
        with torch.cuda.stream(s):
            g.capture_begin()
            self.run()
            g.capture_end()
        torch.cuda.current_stream(self.ws.device).wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.outputs

    def status(self):
        st = torch.cuda.current_stream(self.ws.device)
        return int(lib().gbs_stream_status(_vp(self.ws), ctypes.c_void_p(st.cuda_stream)))


def autotune(V, kmax, precision="fp32r", workspace=None) -> float:
    """Tune the prefix-tree schedule for this shape (see gbs_autotune); returns the best ms."""
    V, M = _prep(V)
    out = torch.empty(table_size(M, kmax), dtype=torch.float64, device=V.device)
    ws = _workspace_for(workspace, M, kmax, precision, V.device)
    st = torch.cuda.current_stream(V.device)
    ms = ctypes.c_float(0.0)
    _check(lib().gbs_autotune(_vp(V), M, kmax, _vp(out), PRECISIONS[precision], ctypes.c_void_p(ws.ptr), ws.nbytes,
                              ctypes.c_void_p(st.cuda_stream), ctypes.byref(ms)))
    return float(ms.value)


def schedule(M: int, kmax: int, precision: str = "fp32r") -> dict:
    """Schedule the forward calls of this shape run on the current device (gbs_schedule)."""
    arr = (ctypes.c_int * 3)()
    _check(lib().gbs_schedule(M, kmax, PRECISIONS[precision], arr))
    return {"variant": arr[0], "grain": arr[1], "ccap": arr[2]}


def timing(on: bool) -> None:
    """Enable or disable per-order CUDA-event timing inside the library."""
    _check(lib().gbs_timing(1 if on else 0))


def timing_read() -> list[float]:
    """[pack, order 1, .., order 5] kernel milliseconds of the most recent timed call."""
    arr = (ctypes.c_float * 6)()
    _check(lib().gbs_timing_read(arr))
    return list(arr)


PIPE_PEAKS_SCRATCH = 65536


def pipe_peaks(device=None) -> dict:
    """Measured sustained FMA throughput of the FP64 and FP32 pipes (gbs_pipe_peaks)."""
    dev = torch.device(device or "cuda")
    scratch = torch.empty(PIPE_PEAKS_SCRATCH, dtype=torch.uint8, device=dev)
    out = (ctypes.c_double * 6)()
    st = torch.cuda.current_stream(dev)
    _check(lib().gbs_pipe_peaks(out, _vp(scratch), ctypes.c_void_p(st.cuda_stream)))
    return {"fp64_flops": out[0], "fp32_flops": out[1], "fp64_fma_per_clk_per_sm": out[2],
            "fp32_fma_per_clk_per_sm": out[3], "sm_mhz_fp64_probe": out[4], "sm_mhz_fp32_probe": out[5]}


def timing_read_backward() -> list[float]:
    """[P0 recomputation, h table, dL/dP0 gather, dL/dV scatter] milliseconds of the
    most recent timed gbs_cumulants_backward call."""
    arr = (ctypes.c_float * 4)()
    _check(lib().gbs_timing_read_backward(arr))
    return list(arr)


def n_subsets(M: int, kmax: int) -> int:
    return sum(comb(M, d) for d in range(1, kmax + 1))
