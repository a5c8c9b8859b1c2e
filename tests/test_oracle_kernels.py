"""Pins for the oracle's FMM kernels (eqs. 3-8, 14, 12) against direct summation,
exact translation identities, the strict error bound of eq. (12) and the bounds
on the multipole power stated with eq. (14)."""
import math

import numpy as np
import pytest


def _cluster(rng, n, centre, radius):
    d = rng.normal(size=(n, 3))
    d *= (radius * rng.uniform(0, 1, size=n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    return centre + d, rng.uniform(0.5, 1.5, size=n) / n


def _direct_on(xs, ms, xt):
    d = xs[None, :, :] - xt[:, None, :]
    r = np.linalg.norm(d, axis=2)
    psi = np.sum(ms[None, :] / r, axis=1)
    acc = np.sum(ms[None, :, None] * d / r[:, :, None] ** 3, axis=1)
    return psi, acc


def test_p2m_then_m2m_is_p2m_at_new_centre(orc):
    """M2M (eq. 4) is an exact translation of P2M (eq. 3c)."""
    rng = np.random.default_rng(1)
    x, mu = _cluster(rng, 40, np.array([0.1, 0.2, -0.3]), 0.5)
    z, zp = np.array([0.1, 0.25, -0.3]), np.array([-0.4, 0.6, 0.1])
    for p in (1, 4, 10):
        M = orc.p2m(p, x, mu, z)
        Ms = orc.m2m(p, M, z, zp)
        Mp = orc.p2m(p, x, mu, zp)
        assert np.max(np.abs(Ms - Mp)) <= 1e-13 * np.max(np.abs(Mp))


def test_monopole_and_dipole(orc):
    """M_0^0 = total mass; about the centre of mass the dipole vanishes."""
    rng = np.random.default_rng(2)
    x, mu = _cluster(rng, 30, np.zeros(3), 1.0)
    com = (mu[:, None] * x).sum(0) / mu.sum()
    M = orc.p2m(3, x, mu, com)
    assert abs(M[0] - mu.sum()) < 1e-15
    assert np.max(np.abs(M[1:4])) < 1e-15


def test_multipole_power_bounds(orc):
    """P_0 = M, P_n <= M rho^n and |M_n^m| <= P_n / n! (eq. 14)."""
    rng = np.random.default_rng(3)
    p = 12
    for trial in range(5):
        x, mu = _cluster(rng, 25, np.zeros(3), 1.0)
        z = rng.normal(size=3) * 0.2
        M = orc.p2m(p, x, mu, z)
        P = orc.power(p, M)
        rho = np.max(np.linalg.norm(x - z, axis=1))
        assert abs(P[0] - mu.sum()) < 1e-14
        for n in range(p + 1):
            assert P[n] <= mu.sum() * rho ** n * (1 + 1e-12)
            for m in range(-n, n + 1):
                assert abs(M[orc.idx(n, m)]) <= P[n] / math.factorial(n) * (1 + 1e-12)
    # a single point mass saturates P_n = M rho^n
    x = np.array([[0.3, -0.4, 0.5]])
    mu = np.array([2.0])
    P = orc.power(p, orc.p2m(p, x, mu, np.zeros(3)))
    rho = np.linalg.norm(x[0])
    assert np.allclose(P, 2.0 * rho ** np.arange(p + 1), rtol=1e-12)


def test_m2l_l2p_converges_to_direct_within_strict_bound(orc):
    """M2L (eq. 3b) + L2P (eq. 7): the error of one interaction decreases with p and
    never exceeds the strict bound (M_A/r^2)(p+1)theta^p/(1-theta)^2 of eq. (12)."""
    rng = np.random.default_rng(4)
    xa, ma = _cluster(rng, 60, np.array([0.0, 0.0, 0.0]), 1.0)
    xb, _ = _cluster(rng, 30, np.array([3.2, 1.5, -1.0]), 0.8)
    zA = np.zeros(3)
    sB = np.array([3.2, 1.5, -1.0])
    rhoA = np.max(np.linalg.norm(xa - zA, axis=1))
    rhoB = np.max(np.linalg.norm(xb - sB, axis=1))
    r = np.linalg.norm(sB - zA)
    theta = (rhoA + rhoB) / r
    assert theta < 1
    psi_t, acc_t = _direct_on(xa, ma, xb)
    prev = first = None
    for p in (2, 4, 6, 8, 10, 12, 14):
        F = orc.m2l(p, orc.p2m(p, xa, ma, zA), zA, sB)
        errs = []
        for i, xt in enumerate(xb):
            psi, a = orc.l2p(p, F, sB, xt)
            errs.append(np.linalg.norm(a - acc_t[i]))
        emax = max(errs)
        bound = ma.sum() / r ** 2 * (p + 1) * theta ** p / (1 - theta) ** 2
        assert emax <= bound
        if prev is not None:
            assert emax < prev
        else:
            first = emax
        prev = emax
    assert prev < 1e-3 * first


def test_potential_sign_and_gradient(orc):
    """Psi is the negative potential (eq. 1): L2P's Psi is sum mu/r > 0 and a = grad Psi
    equals the central finite difference of the L2P potential."""
    rng = np.random.default_rng(5)
    xa, ma = _cluster(rng, 20, np.zeros(3), 0.5)
    sB = np.array([2.5, -1.0, 0.7])
    p = 10
    F = orc.m2l(p, orc.p2m(p, xa, ma, np.zeros(3)), np.zeros(3), sB)
    xt = sB + np.array([0.1, -0.15, 0.05])
    psi, a = orc.l2p(p, F, sB, xt)
    assert psi > 0
    h = 1e-5
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (orc.l2p(p, F, sB, xt + e)[0] - orc.l2p(p, F, sB, xt - e)[0]) / (2 * h)
        assert abs(fd - a[d]) < 1e-8 * np.linalg.norm(a)
    # acceleration points towards the source
    assert np.dot(a, -xt) > 0


def test_l2l_is_exact_on_the_truncated_expansion(orc):
    """L2L (eq. 5) re-expands the degree-p polynomial exactly: L2P after L2L equals L2P."""
    rng = np.random.default_rng(6)
    xa, ma = _cluster(rng, 20, np.zeros(3), 0.5)
    s = np.array([3.0, 0.5, -0.5])
    sp = s + np.array([0.2, -0.1, 0.15])
    for p in (2, 7, 12):
        F = orc.m2l(p, orc.p2m(p, xa, ma, np.zeros(3)), np.zeros(3), s)
        Fp = orc.l2l(p, F, s, sp)
        for _ in range(5):
            xt = sp + rng.normal(size=3) * 0.2
            psi1, a1 = orc.l2p(p, F, s, xt)
            psi2, a2 = orc.l2p(p, Fp, sp, xt)
            assert abs(psi1 - psi2) < 1e-13 * abs(psi1)
            assert np.linalg.norm(a1 - a2) < 1e-12 * np.linalg.norm(a1)


def test_m2l_of_point_mass_is_theta(orc):
    """A point mass mu at z_A has M = mu delta_{n0}; then F_n^m = mu Theta_n^m(s_B - z_A)
    (the P2L kernel of the Table 1 caption)."""
    p = 6
    M = np.zeros(orc.ncoef(p), dtype=complex)
    M[0] = 0.7
    zA, sB = np.array([0.1, 0.2, 0.3]), np.array([1.5, -0.7, 2.0])
    F = orc.m2l(p, M, zA, sB)
    T = orc.theta(p, sB - zA)
    assert np.max(np.abs(F - 0.7 * T)) < 1e-15 * np.max(np.abs(T))
