"""CPU oracle for the FMM of Dehnen (arXiv 1405.2255): TEST INFRASTRUCTURE.

A plain serial FP64 C implementation (``fmm_oracle.c``) plus this ctypes
wrapper.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the GPU library and never
calls it; the product path must not import this package.

Parity status per function (the pins live in tests/test_oracle_*.py):
  harmonics     pinned: Table 3 closed forms, Upsilon/Theta relation (App. A.3),
                addition theorem (App. A.4) against 1/|r - x|.
  P2M/M2M       pinned: M2M(P2M) equals P2M at the new centre (exact shift);
                power bounds of eq. (14).
  M2L/L2L/L2P   pinned: against direct summation (converges as p grows), strict
                bound eq. (12), L2L exactness, L2P gradient vs finite differences.
  MEB           pinned: brute force over support sets on small point sets.
  estimate E~   pinned: eq. (17) equals 4 theta^p (equal radii) and 8 (rho/r)^p (one radius
                zero) for a point-mass source, where E = theta^p exactly (Sec. 4.2); a spread
                source lies strictly between the point-mass and all-at-the-centre values;
                Sec. 4's single-interaction statistics (relative errors above E~ <= 2 %,
                absolute <= 10 %, overestimates by > 10x <= 2 %, eq. 12 always).
  walk / FMM    pinned: reduction to direct summation (eps -> 0), N <= leaf size,
                whole-FMM error vs brute force, Plummer closed form, momentum.
  direct sum    pinned: two-body and symmetric closed forms, Plummer closed form.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class Params(C.Structure):
    _fields_ = [("p", C.c_int), ("eps", C.c_double), ("mac", C.c_int), ("theta_crit", C.c_double),
                ("leaf_size", C.c_int), ("p2p_c", C.c_double), ("scale_src", C.c_int), ("want_tidal", C.c_int),
                ("adaptive_p", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("ncells", C.c_long), ("nleaves", C.c_long), ("n_m2l", C.c_long), ("n_p2p", C.c_long),
                ("p2p_interactions", C.c_long), ("coincident", C.c_long), ("est_m2l", C.c_long),
                ("est_p2p", C.c_long), ("depth", C.c_int)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def _declare(L):
    L.orc_upsilon_re.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.orc_theta_re.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.orc_p2m.argtypes = [C.c_int, C.c_long, _dp, _dp, _dp, _dp, _dp]
    for f in (L.orc_m2m, L.orc_m2l, L.orc_l2l, L.orc_m2l_rot):
        f.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_swap_matrix.argtypes = [C.c_int, _dp]
    L.orc_direct_tidal.argtypes = [C.c_long, _dp, _dp, C.c_double, C.c_long, C.c_void_p, C.c_void_p]
    L.orc_run_tidal.argtypes = [C.c_void_p, _dp]
    L.orc_run_tidal.restype = C.c_int
    L.orc_run_m2l_orders.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_l2p.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.POINTER(C.c_double), _dp]
    L.orc_power.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_direct.argtypes = [C.c_long, _dp, _dp, C.c_double, C.c_long, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p]
    L.orc_direct.restype = C.c_long
    L.orc_meb_points.argtypes = [C.c_int, _dp, _dp, C.POINTER(C.c_double)]
    L.orc_meb_balls.argtypes = [C.c_int, _dp, _dp, _dp, C.POINTER(C.c_double)]
    L.orc_fmm.argtypes = [C.c_long, _dp, _dp, C.c_double, C.POINTER(Params), C.c_void_p]
    L.orc_fmm.restype = C.c_void_p
    L.orc_fmm_active.argtypes = [C.c_long, _dp, _dp, C.c_double, C.POINTER(Params), C.c_void_p, C.c_void_p,
                                 C.c_void_p]
    L.orc_fmm_active.restype = C.c_void_p
    L.orc_fmm_reuse.argtypes = [C.c_void_p, C.c_long, _dp, _dp, C.c_double, C.POINTER(Params), C.c_void_p,
                                C.c_void_p, C.c_void_p]
    L.orc_fmm_reuse.restype = C.c_void_p
    L.orc_run_free.argtypes = [C.c_void_p]
    L.orc_run_outputs.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_run_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    L.orc_run_ncells.argtypes = [C.c_void_p]
    L.orc_run_ncells.restype = C.c_long
    L.orc_run_cells.argtypes = [C.c_void_p, _lp, _dp]
    L.orc_run_lists.argtypes = [C.c_void_p, _lp, _lp]
    L.orc_run_perm.argtypes = [C.c_void_p, _lp]
    L.orc_run_scale.argtypes = [C.c_void_p, _dp]
    L.orc_mac_lhs.argtypes = [C.c_int, _dp, C.c_double, C.c_double, C.c_double]
    L.orc_mac_lhs.restype = C.c_double
    L.orc_interaction_errors.argtypes = [C.c_void_p, C.c_long, C.c_long, C.c_int, _dp]
    L.orc_interaction_errors.restype = C.c_int


def _c3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def ncoef(p):
    return (p + 1) * (p + 1)


def idx(n, m):
    """index of (n, m) in a full complex harmonic array"""
    return n * n + n + m


def upsilon(p, r):
    re, im = np.zeros(ncoef(p)), np.zeros(ncoef(p))
    lib().orc_upsilon_re(p, float(r[0]), float(r[1]), float(r[2]), re, im)
    return re + 1j * im


def theta(p, r):
    re, im = np.zeros(ncoef(p)), np.zeros(ncoef(p))
    lib().orc_theta_re(p, float(r[0]), float(r[1]), float(r[2]), re, im)
    return re + 1j * im


def _split(c):
    c = np.asarray(c, dtype=np.complex128)
    return np.ascontiguousarray(c.real), np.ascontiguousarray(c.imag)


def p2m(p, x, mu, z):
    x = np.ascontiguousarray(x, dtype=np.float64)
    re, im = np.zeros(ncoef(p)), np.zeros(ncoef(p))
    lib().orc_p2m(p, len(mu), x, np.ascontiguousarray(mu, dtype=np.float64), _c3(z), re, im)
    return re + 1j * im


def _shift(fn, p, X, a, b):
    xr, xi = _split(X)
    re, im = np.zeros(ncoef(p)), np.zeros(ncoef(p))
    fn(p, xr, xi, _c3(a), _c3(b), re, im)
    return re + 1j * im


def m2m(p, M, z, zp):
    return _shift(lib().orc_m2m, p, M, z, zp)


def m2l(p, M, zA, sB):
    return _shift(lib().orc_m2l, p, M, zA, sB)


def l2l(p, F, s, sp):
    return _shift(lib().orc_l2l, p, F, s, sp)


def m2l_rot(p, M, zA, sB):
    """eq. (3b) through the rotations of App. A.5.2 and the z-axis kernel eq. (A31)."""
    return _shift(lib().orc_m2l_rot, p, M, zA, sB)


def swap_matrix(n):
    """B_n of App. A.5.1, rows m and columns l = -n..n: Theta_n(z, y, x) = B_n Theta_n(x, y, z)."""
    B = np.zeros((2 * n + 1) * (2 * n + 1))
    lib().orc_swap_matrix(n, B)
    return B.reshape(2 * n + 1, 2 * n + 1)


def l2p(p, F, s, xb):
    fr, fi = _split(F)
    psi = C.c_double()
    a = np.zeros(3)
    lib().orc_l2p(p, fr, fi, _c3(s), _c3(xb), C.byref(psi), a)
    return psi.value, a


def power(p, M):
    mr, mi = _split(M)
    P = np.zeros(p + 1)
    lib().orc_power(p, mr, mi, P)
    return P


def error_estimate(P, r, rho_a, rho_b, mass, q=None):
    """E~_{A->B} of eq. (17) from the source cell's multipole powers P_0..P_q (eq. 14), the
    distance r = |s_B - z_A|, the radii rho_A, rho_B and the mass M_A: the quantity the
    oracle's walk compares, divided by M_A / r^2."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    q = len(P) - 1 if q is None else q
    return lib().orc_mac_lhs(q, P, float(r), float(rho_a), float(rho_b)) * r * r / mass


def interaction_errors(x, mu, p, theta_crit=0.7, leaf_size=32, p2p_c=1.0, sample=None, seed=0):
    """Sec. 4's single-interaction experiment: the cell pairs (A, B) that a walk with the
    geometric criterion theta < theta_crit (eq. 9) accepts, minus those with
    N_A N_B < p2p_c p^3, each evaluated alone at order p against direct summation.
    Returns an array [pairs, 4]: max delta a r^2 / M_A, max delta a / a, E~ (eq. 17), theta."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    prm = Params(p, 1.0, MAC_THETA, theta_crit, leaf_size, p2p_c, 0, 0, 0)
    L = lib()
    h = L.orc_fmm_active(len(mu), x, mu, 1.0, C.byref(prm), None, None, None)
    if not h:
        raise ValueError("oracle rejected the input")
    try:
        st = Stats()
        L.orc_run_stats(h, C.byref(st))
        m2 = np.zeros((max(st.n_m2l, 1), 2), dtype=np.int64)
        pp = np.zeros((max(st.n_p2p, 1), 2), dtype=np.int64)
        L.orc_run_lists(h, m2, pp)
        m2 = m2[:st.n_m2l]
        if sample is not None and sample < len(m2):
            m2 = m2[np.sort(np.random.default_rng(seed).choice(len(m2), sample, replace=False))]
        out, row = [], np.zeros(4)
        for a, b in m2:
            if L.orc_interaction_errors(h, int(a), int(b), p, row):
                out.append(row.copy())
        return np.array(out).reshape(-1, 4)
    finally:
        L.orc_run_free(h)


def direct(x, mu, G=1.0, sinks=None):
    """Direct FP64 sums of eqs. (1) and (6); returns psi, acc, f, coincident."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    n = len(mu)
    if sinks is None:
        ns, sp = n, None
    else:
        sinks = np.ascontiguousarray(sinks, dtype=np.int64)
        ns, sp = len(sinks), sinks.ctypes.data
    psi, acc, f = np.zeros(max(ns, 1)), np.zeros((max(ns, 1), 3)), np.zeros(max(ns, 1))
    coin = lib().orc_direct(n, x, mu, G, ns, sp, psi.ctypes.data, acc.ctypes.data, f.ctypes.data)
    return psi[:ns], acc[:ns], f[:ns], coin


def meb_points(pts):
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    c, r = np.zeros(3), C.c_double()
    lib().orc_meb_points(len(pts), pts, c, C.byref(r))
    return c, r.value


def meb_balls(cen, rad):
    cen = np.ascontiguousarray(cen, dtype=np.float64)
    rad = np.ascontiguousarray(rad, dtype=np.float64)
    c, r = np.zeros(3), C.c_double()
    ok = lib().orc_meb_balls(len(rad), cen, rad, c, C.byref(r))
    return (c, r.value) if ok else (None, None)


MAC_A, MAC_F, MAC_THETA = 0, 1, 2


@dataclass
class Run:
    psi: np.ndarray
    acc: np.ndarray
    stats: dict
    cells_int: np.ndarray   # [nc,5] level, leaf, first, count, nchild
    cells_dbl: np.ndarray   # [nc,6] s[3], rho, mass, minscale
    m2l: np.ndarray         # [n_m2l,2] (source cell, sink cell)
    p2p: np.ndarray         # [n_p2p,2]
    perm: np.ndarray
    scale: np.ndarray       # per sorted particle
    tidal: np.ndarray = None  # [n,6] (xx, xy, xz, yy, yz, zz) when asked for
    m2l_q: np.ndarray = None  # order of each M2L interaction (same order as m2l)


def fmm(x, mu, G=1.0, p=6, eps=1e-7, mac=MAC_A, theta_crit=0.5, leaf_size=32, p2p_c=1.0,
        scale=None, keep=True, active=None, eps_b=None, tidal=False, adaptive_p=False):
    """Run the oracle FMM; raises ValueError on invalid input.  active (bool/uint8 [n],
    caller order): forces for that subset only (Sec. 7.1), NaN for the others; eps_b [n]:
    individual accuracy parameters (Sec. 7, opening)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    prm = Params(p, eps, mac, theta_crit, leaf_size, p2p_c, 1 if scale is not None else 0, 1 if tidal else 0,
                 1 if adaptive_p else 0)
    sc = None if scale is None else np.ascontiguousarray(scale, dtype=np.float64)
    act = None if active is None else np.ascontiguousarray(np.asarray(active) != 0, dtype=np.uint8)
    L = lib()
    eb = None if eps_b is None else np.ascontiguousarray(eps_b, dtype=np.float64)
    h = L.orc_fmm_active(len(mu), x, mu, G, C.byref(prm), sc.ctypes.data if sc is not None else None,
                         act.ctypes.data if act is not None else None, eb.ctypes.data if eb is not None else None)
    if not h:
        raise ValueError("oracle rejected the input")
    try:
        return _collect(L, h, len(mu), keep)
    finally:
        L.orc_run_free(h)


def fmm_reused(x0, mu0, x, mu, G=1.0, p=6, eps=1e-7, mac=MAC_A, theta_crit=0.5, leaf_size=32, p2p_c=1.0,
               active=None, keep=True):
    """Sec. 7.1's re-cycled tree: build the tree for (x0, mu0), then evaluate (x, mu), the
    same particles in the same order, on that tree (order, cells and centres kept; radii,
    masses and centres of mass recomputed)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1, 3)
    mu0 = np.ascontiguousarray(mu0, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    prm = Params(p, eps, mac, theta_crit, leaf_size, p2p_c, 0, 0, 0)
    act = None if active is None else np.ascontiguousarray(np.asarray(active) != 0, dtype=np.uint8)
    L = lib()
    h0 = L.orc_fmm_active(len(mu0), x0, mu0, G, C.byref(prm), None, None, None)
    if not h0:
        raise ValueError("oracle rejected the first input")
    try:
        h = L.orc_fmm_reuse(h0, len(mu), x, mu, G, C.byref(prm), None, act.ctypes.data if act is not None else None,
                            None)
        if not h:
            raise ValueError("oracle rejected the second input")
        try:
            return _collect(L, h, len(mu), keep)
        finally:
            L.orc_run_free(h)
    finally:
        L.orc_run_free(h0)


def _collect(L, h, n, keep):
    psi, acc = np.zeros(max(n, 1)), np.zeros((max(n, 1), 3))
    L.orc_run_outputs(h, psi, acc)
    T = np.zeros((max(n, 1), 6))
    tid = T[:n] if n > 0 and L.orc_run_tidal(h, T) else None
    st = Stats()
    L.orc_run_stats(h, C.byref(st))
    stats = {k: getattr(st, k) for k, _ in Stats._fields_}
    if keep and n > 0:
        nc = L.orc_run_ncells(h)
        ci, cd = np.zeros((nc, 5), dtype=np.int64), np.zeros((nc, 6))
        L.orc_run_cells(h, ci, cd)
        m2 = np.zeros((max(st.n_m2l, 1), 2), dtype=np.int64)
        pp = np.zeros((max(st.n_p2p, 1), 2), dtype=np.int64)
        L.orc_run_lists(h, m2, pp)
        perm = np.zeros(n, dtype=np.int64)
        L.orc_run_perm(h, perm)
        scl = np.zeros(n)
        L.orc_run_scale(h, scl)
        q = np.zeros(max(st.n_m2l, 1), dtype=np.int32)
        L.orc_run_m2l_orders(h, q.ctypes.data)
        return Run(psi[:n], acc[:n], stats, ci, cd, m2[:st.n_m2l], pp[:st.n_p2p], perm, scl, tid, q[:st.n_m2l])
    return Run(psi[:n], acc[:n], stats, None, None, None, None, None, None, tid)


def direct_tidal(x, mu, G=1.0, sinks=None):
    """T = grad grad Psi by direct summation (Sec. 7.4), [ns,6] as (xx, xy, xz, yy, yz, zz)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    sk = None if sinks is None else np.ascontiguousarray(sinks, dtype=np.int64)
    ns = len(mu) if sk is None else len(sk)
    T = np.zeros((max(ns, 1), 6))
    lib().orc_direct_tidal(len(mu), x, mu, G, ns, sk.ctypes.data if sk is not None else None, T.ctypes.data)
    return T[:ns]
