"""Pins of the rotation-accelerated M2L (App. A.5) in the oracle: the swap matrices of
App. A.5.1 against the matrix the paper prints, against swapping the coordinates of the
harmonics themselves, and the rotated M2L (eq. A31) against eq. (3b) term by term."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "swap_b4_x16.txt")


def _idx(n, m):
    return n * n + n + m


def test_swap_matrix_n4_as_printed(orc):
    want = np.loadtxt(GOLDEN)
    assert np.array_equal(16.0 * orc.swap_matrix(4), want)


@pytest.mark.parametrize("n", [1, 2, 5, 9, 16])
def test_swap_matrix_swaps_x_and_z(orc, n):
    """Theta_n(z, y, x) = B_n Theta_n(x, y, z) and Upsilon_n(z, y, x) = B_n^T Upsilon_n(x, y, z)."""
    B = orc.swap_matrix(n)
    rng = np.random.default_rng(n)
    sl = slice(n * n, (n + 1) * (n + 1))
    for _ in range(4):
        r = rng.normal(size=3)
        rs = r[[2, 1, 0]]
        t, ts = orc.theta(n, r)[sl], orc.theta(n, rs)[sl]
        assert np.max(np.abs(ts - B @ t)) <= 1e-11 * np.max(np.abs(ts))
        u, us = orc.upsilon(n, r)[sl], orc.upsilon(n, rs)[sl]
        assert np.max(np.abs(us - B.T @ u)) <= 1e-11 * np.max(np.abs(us))


@pytest.mark.parametrize("n", [3, 8, 16])
def test_swap_matrix_is_an_involution(orc, n):
    B = orc.swap_matrix(n)
    assert np.max(np.abs(B @ B - np.eye(2 * n + 1))) < 1e-9


def _l2p_field(orc, p, F, s, pts):
    out = []
    for x in pts:
        psi, a = orc.l2p(p, F, s, x)
        out.append([psi, *a])
    return np.array(out)


@pytest.mark.parametrize("p", [3, 8, 14, 16])
def test_rotated_m2l_equals_eq3b(orc, p):
    """The rotated M2L gives eq. (3b) up to rounding, for general directions and for
    interactions along +z and -z (no rotation about z needed): compared coefficient by
    coefficient on the scale of each order and through the potential and acceleration of
    the local expansion at points of the sink sphere."""
    rng = np.random.default_rng(100 + p)
    for direction in (None, (0.0, 0.0, 1.0), (0.0, 0.0, -1.0), (1.0, 0.0, 0.0)):
        zA = rng.normal(size=3)
        rhoA = 0.5
        xs = zA + rng.normal(size=(40, 3)) * 0.2
        xs = zA + (xs - zA) * np.minimum(1.0, rhoA / np.linalg.norm(xs - zA, axis=1))[:, None]
        M = orc.p2m(p, xs, rng.random(40), zA)
        u = rng.normal(size=3) if direction is None else np.array(direction)
        sB = zA + 2.5 * u / np.linalg.norm(u)
        Fd = orc.m2l(p, M, zA, sB)
        Fr = orc.m2l_rot(p, M, zA, sB)
        for n in range(p + 1):
            sl = slice(n * n, (n + 1) * (n + 1))
            nrm = np.array([math.sqrt(float(math.factorial(n - abs(m)) * math.factorial(n + abs(m))))
                            for m in range(-n, n + 1)])
            assert np.max(np.abs(Fr[sl] - Fd[sl]) / nrm) <= 1e-11 * np.max(np.abs(Fd[sl]) / nrm)
        pts = sB + rng.normal(size=(5, 3)) * 0.1
        fd, fr = _l2p_field(orc, p, Fd, sB, pts), _l2p_field(orc, p, Fr, sB, pts)
        assert np.max(np.abs(fr - fd)) <= 1e-12 * np.max(np.abs(fd))

