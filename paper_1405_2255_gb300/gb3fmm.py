"""Python binding of the C ABI in include/gb3fmm.h (argument marshalling only).

Every step of the force evaluation runs in the CUDA library libgb3fmm.so built
from ``csrc/``; this module only passes pointers and sizes.  It raises
``RuntimeError`` when the library is missing: there is no CPU fallback.

Device buffers are torch CUDA tensors (float64, contiguous); host buffers of the
``*_host`` calls are numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgb3fmm.so")

FMM_OK, FMM_E_INVALID, FMM_E_OOM, FMM_E_ADMISSION, FMM_E_CUDA = 0, -1, -2, -3, -4
FMM_E_TIMEOUT, FMM_E_OVERFLOW, FMM_E_NOTFOUND, FMM_E_BUSY = -5, -6, -7, -8
FMM_MAC_A, FMM_MAC_F, FMM_MAC_THETA = 0, 1, 2
FMM_PREC_FP64, FMM_PREC_MIXED = 0, 1
FMM_SCALE_ESTIMATE, FMM_SCALE_CALLER = 0, 1


class fmm_params(C.Structure):
    _fields_ = [("p", C.c_int), ("eps", C.c_double), ("mac", C.c_int), ("theta_crit", C.c_double),
                ("leaf_size", C.c_int), ("p2p_c", C.c_double), ("precision", C.c_int), ("scale_src", C.c_int),
                ("p2p_two_float", C.c_int), ("m2l_split", C.c_int), ("m2l_rot", C.c_int),
                ("adaptive_p", C.c_int)]


class fmm_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncells", C.c_int64), ("nleaves", C.c_int64), ("n_m2l", C.c_int64),
                ("n_p2p", C.c_int64), ("p2p_interactions", C.c_int64), ("coincident", C.c_int64),
                ("est_m2l", C.c_int64), ("est_p2p", C.c_int64), ("depth", C.c_int), ("p", C.c_int),
                ("eps", C.c_double), ("leaf_size", C.c_int),
                ("t_tree", C.c_float), ("t_estimate", C.c_float), ("t_up", C.c_float), ("t_walk", C.c_float),
                ("t_m2l", C.c_float), ("t_p2p", C.c_float), ("t_down", C.c_float), ("t_total", C.c_float),
                ("launches", C.c_int64), ("t_m2l_kernel", C.c_float), ("t_p2p_kernel", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol include/gb3fmm.h declares
EXPORTS = ["fmm_default_params", "fmm_create", "fmm_set_params", "fmm_evaluate", "fmm_evaluate_host",
           "fmm_direct", "fmm_evaluate_batch", "fmm_debug_dump", "fmm_last_stats", "fmm_destroy",
           "fmm_strerror", "fmm_last_error", "fmm_version", "fmm_alu_peaks", "fmm_evaluate_noalloc",
           "fmm_serve_config", "fmm_footprint_bytes", "fmm_system_register", "fmm_submit", "fmm_poll",
           "fmm_system_release", "fmm_workspace_bytes", "fmm_swap_matrix",
           "fmm_evaluate_active", "fmm_debug_m2l_orders", "fmm_swap_probe", "fmm_pair_peak"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libgb3fmm.so (build it first with ``paper_1405_2255_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgb3fmm.so not found at {path}: run __graft_entry__.build() first")
    L = C.CDLL(path)
    vp, i64, dbl, ci = C.c_void_p, C.c_int64, C.c_double, C.c_int
    L.fmm_default_params.argtypes = [C.POINTER(fmm_params)]
    L.fmm_default_params.restype = None
    L.fmm_create.argtypes = [C.POINTER(vp), C.POINTER(fmm_params), ci]
    L.fmm_set_params.argtypes = [vp, C.POINTER(fmm_params)]
    L.fmm_evaluate.argtypes = [vp, i64, vp, vp, dbl, vp, vp, vp, vp, C.POINTER(fmm_stats)]
    L.fmm_evaluate_host.argtypes = [vp, i64, vp, vp, dbl, vp, vp, vp, C.POINTER(fmm_stats)]
    L.fmm_direct.argtypes = [vp, i64, vp, vp, dbl, i64, vp, vp, vp, vp, vp]
    L.fmm_evaluate_batch.argtypes = [vp, ci, vp, vp, vp, vp, vp, vp, vp, C.POINTER(fmm_stats)]
    L.fmm_debug_dump.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fmm_last_stats.argtypes = [vp, C.POINTER(fmm_stats)]
    L.fmm_destroy.argtypes = [vp]
    L.fmm_strerror.argtypes = [ci]
    L.fmm_strerror.restype = C.c_char_p
    L.fmm_last_error.argtypes = [vp]
    L.fmm_last_error.restype = C.c_char_p
    L.fmm_alu_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.fmm_evaluate_noalloc.argtypes = [i64, vp, vp, dbl, C.POINTER(fmm_params), vp, vp, vp, C.c_char_p, ci]
    L.fmm_version.argtypes = []
    L.fmm_version.restype = C.c_char_p
    L.fmm_serve_config.argtypes = [vp, C.c_uint64, ci]
    L.fmm_footprint_bytes.argtypes = [C.POINTER(fmm_params), i64]
    L.fmm_footprint_bytes.restype = i64
    L.fmm_system_register.argtypes = [vp, i64, C.POINTER(ci)]
    L.fmm_submit.argtypes = [vp, ci, vp, vp, dbl, vp, vp, C.POINTER(C.c_uint64)]
    L.fmm_poll.argtypes = [vp, C.c_uint64, ci, C.POINTER(C.c_double)]
    L.fmm_system_release.argtypes = [vp, ci]
    L.fmm_workspace_bytes.argtypes = [vp]
    L.fmm_workspace_bytes.restype = C.c_uint64
    L.fmm_swap_matrix.argtypes = [ci, vp]
    L.fmm_debug_m2l_orders.argtypes = [vp, vp]
    L.fmm_swap_probe.argtypes = [ci, ci, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.fmm_pair_peak.argtypes = [ci, C.POINTER(C.c_double)]
    L.fmm_evaluate_active.argtypes = [vp, i64, vp, vp, dbl, vp, vp, vp, ci, vp, vp, vp, vp, C.POINTER(fmm_stats)]
    for name in EXPORTS:
        if name not in ("fmm_strerror", "fmm_last_error", "fmm_version", "fmm_default_params",
                        "fmm_footprint_bytes", "fmm_workspace_bytes"):
            getattr(L, name).restype = ci
    _lib = L
    return L


class FMMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _check(rc, ctx=None):
    if rc != 0:
        L = load()
        detail = L.fmm_last_error(ctx).decode() if ctx else ""
        raise FMMError(rc, f"{L.fmm_strerror(rc).decode()}: {detail}")


def fmm_default_params() -> fmm_params:
    p = fmm_params()
    load().fmm_default_params(C.byref(p))
    return p


def _ptr(t):
    if t is None:
        return None
    import torch
    assert t.is_cuda and t.is_contiguous(), "device buffers must be contiguous CUDA tensors"
    assert t.dtype in (torch.float64, torch.int64, torch.uint8), t.dtype
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Context:
    """Owns one fmm_ctx (device workspace); the methods are the C entry points."""

    def __init__(self, params: fmm_params | None = None, device: int = 0, **kw):
        self.L = load()
        if params is None:
            params = fmm_default_params()
        for k, v in kw.items():
            setattr(params, k, v)
        self.params = params
        h = C.c_void_p()
        _check(self.L.fmm_create(C.byref(h), C.byref(params), device))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        _check(self.L.fmm_set_params(self.h, C.byref(self.params)), self.h)

    def fmm_evaluate(self, x, mu, G=1.0, psi=None, acc=None, scale=None, stream=None, stats=False):
        """x: [n,3] float64 CUDA tensor, mu: [n]; returns (psi, acc[, stats dict])."""
        import torch
        n = mu.shape[0]
        if psi is None:
            psi = torch.empty(n, dtype=torch.float64, device=mu.device)
        if acc is None:
            acc = torch.empty((n, 3), dtype=torch.float64, device=mu.device)
        st = fmm_stats() if stats else None
        rc = self.L.fmm_evaluate(self.h, n, _ptr(x), _ptr(mu), float(G), _ptr(scale), _ptr(psi), _ptr(acc),
                                 _stream(stream), C.byref(st) if st is not None else None)
        _check(rc, self.h)
        return (psi, acc, st.as_dict()) if stats else (psi, acc)

    def fmm_evaluate_active(self, x, mu, active=None, G=1.0, psi=None, acc=None, scale=None, stream=None,
                            stats=False, reuse_tree=False, eps_b=None, tidal=None):
        """Forces for the active subset (Sec. 7.1): active is a [n] uint8/bool CUDA tensor or None
        (all); psi and acc (allocated here if None) are written for the active particles only.
        reuse_tree: keep the previous evaluation's tree (order, cells, centres) for the new
        positions.  eps_b: [n] float64 CUDA tensor of individual accuracy parameters (Sec. 7, opening).
        tidal: True or a [n,6] float64 CUDA tensor: also the tidal tensor (Sec. 7.4), returned last."""
        import torch
        n = mu.shape[0]
        if psi is None:
            psi = torch.full((n,), float("nan"), dtype=torch.float64, device=mu.device)
        if acc is None:
            acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device=mu.device)
        a = None if active is None else (active if active.dtype == torch.uint8 else active.to(torch.uint8))
        T = None
        if tidal is not None and tidal is not False:
            T = tidal if isinstance(tidal, torch.Tensor) else torch.full((n, 6), float("nan"), dtype=torch.float64,
                                                                         device=mu.device)
        st = fmm_stats() if stats else None
        rc = self.L.fmm_evaluate_active(self.h, n, _ptr(x), _ptr(mu), float(G), _ptr(scale), _ptr(a), _ptr(eps_b),
                                        1 if reuse_tree else 0, _ptr(psi), _ptr(acc), _ptr(T), _stream(stream),
                                        C.byref(st) if st is not None else None)
        _check(rc, self.h)
        out = (psi, acc) + ((T,) if T is not None else ())
        return out + (st.as_dict(),) if stats else out

    def fmm_evaluate_host(self, x: np.ndarray, mu: np.ndarray, G=1.0, psi=None, acc=None, stream=None, stats=False):
        """Host numpy in and out (the end-to-end call: copies inside)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        n = len(mu)
        psi = np.empty(n) if psi is None else psi
        acc = np.empty((n, 3)) if acc is None else acc
        st = fmm_stats() if stats else None
        s = 0 if stream is None else _stream(stream)
        rc = self.L.fmm_evaluate_host(self.h, n, x.ctypes.data, mu.ctypes.data, float(G), psi.ctypes.data,
                                      acc.ctypes.data, s, C.byref(st) if st is not None else None)
        _check(rc, self.h)
        return (psi, acc, st.as_dict()) if stats else (psi, acc)

    def fmm_direct(self, x, mu, G=1.0, sinks=None, want_f=False, stream=None):
        """GPU FP64 direct summation for the sinks (int64 CUDA tensor or None = all)."""
        import torch
        n = mu.shape[0]
        ns = n if sinks is None else sinks.shape[0]
        psi = torch.empty(ns, dtype=torch.float64, device=mu.device)
        acc = torch.empty((ns, 3), dtype=torch.float64, device=mu.device)
        f = torch.empty(ns, dtype=torch.float64, device=mu.device) if want_f else None
        _check(self.L.fmm_direct(self.h, n, _ptr(x), _ptr(mu), float(G), ns, _ptr(sinks), _ptr(psi), _ptr(acc),
                                 _ptr(f), _stream(stream)), self.h)
        return (psi, acc, f) if want_f else (psi, acc)

    def fmm_evaluate_batch(self, offsets: np.ndarray, x, mu, G, psi=None, acc=None, stream=None, stats=False):
        import torch
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        G = np.ascontiguousarray(np.broadcast_to(np.asarray(G, dtype=np.float64), (len(offsets) - 1,)))
        n = int(offsets[-1])
        if psi is None:
            psi = torch.empty(n, dtype=torch.float64, device=mu.device)
        if acc is None:
            acc = torch.empty((n, 3), dtype=torch.float64, device=mu.device)
        st = fmm_stats() if stats else None
        _check(self.L.fmm_evaluate_batch(self.h, len(offsets) - 1, offsets.ctypes.data, _ptr(x), _ptr(mu),
                                         G.ctypes.data, _ptr(psi), _ptr(acc), _stream(stream),
                                         C.byref(st) if st is not None else None), self.h)
        return (psi, acc, st.as_dict()) if stats else (psi, acc)

    # ---- serving: continuous batching of requests from many systems
    def fmm_serve_config(self, budget_bytes: int = 0, slots: int = 0):
        _check(self.L.fmm_serve_config(self.h, int(budget_bytes), int(slots)), self.h)

    def fmm_system_register(self, n: int) -> int:
        sid = C.c_int()
        _check(self.L.fmm_system_register(self.h, int(n), C.byref(sid)), self.h)
        return sid.value

    def fmm_submit(self, sys_id: int, x, mu, G, psi, acc) -> int:
        """Queue one force request (device tensors; x and mu must be ready, psi/acc
        are written before fmm_poll reports completion)."""
        t = C.c_uint64()
        _check(self.L.fmm_submit(self.h, int(sys_id), _ptr(x), _ptr(mu), float(G), _ptr(psi), _ptr(acc),
                                 C.byref(t)), self.h)
        return t.value

    def fmm_poll(self, ticket: int, timeout_ms: int = -1):
        """None while the request runs (after timeout_ms), else its latency in seconds;
        raises FMMError if its evaluation failed."""
        lat = C.c_double()
        rc = self.L.fmm_poll(self.h, int(ticket), int(timeout_ms), C.byref(lat))
        if rc == FMM_E_BUSY:
            return None
        _check(rc, self.h)
        return lat.value

    def fmm_system_release(self, sys_id: int):
        _check(self.L.fmm_system_release(self.h, int(sys_id)), self.h)

    def fmm_workspace_bytes(self) -> int:
        return int(self.L.fmm_workspace_bytes(self.h))

    def fmm_last_stats(self) -> dict:
        st = fmm_stats()
        _check(self.L.fmm_last_stats(self.h, C.byref(st)), self.h)
        return st.as_dict()

    def fmm_debug_m2l_orders(self) -> np.ndarray:
        """Order of every M2L interaction of the last evaluation (fmm_debug_dump's order)."""
        st = self.fmm_last_stats()
        q = np.zeros(max(int(st["n_m2l"]), 1), dtype=np.int32)
        _check(self.L.fmm_debug_m2l_orders(self.h, q.ctypes.data), self.h)
        return q[:int(st["n_m2l"])]

    def fmm_debug_dump(self) -> dict:
        st = self.fmm_last_stats()
        n, nc = int(st["n"]), int(st["ncells"])
        ci = np.zeros((max(nc, 1), 5), dtype=np.int64)
        cd = np.zeros((max(nc, 1), 6))
        m2l = np.zeros((max(st["n_m2l"], 1), 2), dtype=np.int64)
        p2p = np.zeros((max(st["n_p2p"], 1), 2), dtype=np.int64)
        perm = np.zeros(max(n, 1), dtype=np.int64)
        scale = np.zeros(max(n, 1))
        _check(self.L.fmm_debug_dump(self.h, ci.ctypes.data, cd.ctypes.data, m2l.ctypes.data, p2p.ctypes.data,
                                     perm.ctypes.data, scale.ctypes.data), self.h)
        return {"cells_int": ci[:nc], "cells_dbl": cd[:nc], "m2l": m2l[:st["n_m2l"]], "p2p": p2p[:st["n_p2p"]],
                "perm": perm[:n], "scale": scale[:n], "stats": st}


def fmm_evaluate_noalloc(x, mu, G=1.0, params: fmm_params | None = None, psi=None, acc=None, stream=None, **kw):
    """Allocation-free evaluation of a small system (n <= 8192): the library takes all
    scratch from a fixed array in device memory.  psi/acc may be passed in so that
    nothing is allocated on this side either."""
    import torch
    L = load()
    if params is None:
        params = fmm_default_params()
    for k, v in kw.items():
        setattr(params, k, v)
    n = mu.shape[0]
    if psi is None:
        psi = torch.empty(n, dtype=torch.float64, device=mu.device)
    if acc is None:
        acc = torch.empty((n, 3), dtype=torch.float64, device=mu.device)
    err = C.create_string_buffer(256)
    rc = L.fmm_evaluate_noalloc(n, _ptr(x), _ptr(mu), float(G), C.byref(params), _ptr(psi), _ptr(acc),
                                _stream(stream), err, 256)
    if rc != 0:
        raise FMMError(rc, f"{L.fmm_strerror(rc).decode()}: {err.value.decode()}")
    return psi, acc


def fmm_footprint_bytes(n: int, params: fmm_params | None = None, **kw) -> int:
    """The serving loop's workspace bound for a system of n particles."""
    if params is None:
        params = fmm_default_params()
    for k, v in kw.items():
        setattr(params, k, v)
    return int(load().fmm_footprint_bytes(C.byref(params), int(n)))


def fmm_swap_matrix(n: int) -> np.ndarray:
    """B_n (App. A.5.1) as built into the rotation-accelerated M2L, rows m / columns l = -n..n."""
    B = np.zeros((2 * n + 1, 2 * n + 1))
    _check(load().fmm_swap_matrix(int(n), B.ctypes.data))
    return B


def fmm_alu_peaks() -> tuple[float, float]:
    """Measured (FP64 DFMA, FP32 FFMA) throughput of the current device in TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(load().fmm_alu_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def fmm_pair_peak(warps_per_sm: int = 16) -> float:
    """The mixed P2P's pair arithmetic alone, in 10^9 pairs per second."""
    v = C.c_double()
    _check(load().fmm_pair_peak(int(warps_per_sm), C.byref(v)))
    return v.value


def fmm_swap_probe(npairs: int = 1 << 20, reps: int = 16) -> dict:
    """Swap stage of the rotated M2L, FMA immediates vs TF32 tensor cores (times in ms)."""
    L = load()
    ms = (C.c_double * 2)()
    md = C.c_double()
    _check(L.fmm_swap_probe(npairs, reps, ms, C.byref(md)))
    return {"fma_ms": ms[0], "mma_ms": ms[1], "maxdiff": md.value, "npairs": npairs, "reps": reps}


def fmm_version() -> str:
    return load().fmm_version().decode()


def fmm_strerror(code: int) -> str:
    return load().fmm_strerror(code).decode()
