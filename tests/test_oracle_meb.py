"""Pins for the smallest enclosing balls that give the expansion centres z = s
(Sec. 5.1.1).  The oracle uses Welzl's recursion for points and an enumeration of
support sets for balls, in single precision relative to the first point (the
radius used by the method is recomputed exactly in FP64 afterwards); here both
are checked against an FP64 brute force and against an independent numerical
minimisation of max_i (|c - c_i| + r_i), to single-precision tolerances."""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize


def _brute_points(P):
    """Smallest ball whose boundary passes through some subset of <= 4 points
    (circumcentre in their affine hull) and contains all points."""
    best = None
    for k in range(1, 5):
        for sub in itertools.combinations(range(len(P)), k):
            Q = P[list(sub)]
            if k == 1:
                c, r = Q[0], 0.0
            else:
                D = Q[1:] - Q[0]
                G = D @ D.T
                if abs(np.linalg.det(G)) < 1e-12 * max(1.0, np.abs(G).max()) ** len(G):
                    continue
                lam = np.linalg.solve(G, 0.5 * np.diag(G))
                c = Q[0] + lam @ D
                r = np.linalg.norm(c - Q[0])
            if np.all(np.linalg.norm(P - c, axis=1) <= r * (1 + 1e-10) + 1e-15):
                if best is None or r < best[1]:
                    best = (c, r)
    return best


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9])
def test_meb_points_matches_brute_force(orc, n):
    rng = np.random.default_rng(n)
    for _ in range(6):
        P = rng.normal(size=(n, 3))
        c, r = orc.meb_points(P)
        cb, rb = _brute_points(P)
        scale = max(rb, 1e-300) + np.abs(P).max() * 1e-7
        assert abs(r - rb) <= 2e-5 * scale
        # the enclosing radius about the oracle's centre is the optimum to ~1e-5
        assert np.linalg.norm(P - c, axis=1).max() <= rb * (1 + 3e-5) + 1e-6 * scale
        if n > 1:
            assert np.linalg.norm(c - cb) <= 1e-2 * rb


def test_meb_points_special_cases(orc):
    # two points: the diametral ball
    c, r = orc.meb_points(np.array([[0.0, 0, 0], [2.0, 0, 0]]))
    assert np.allclose(c, [1, 0, 0], atol=1e-7) and abs(r - 1) < 1e-6
    # regular tetrahedron: centroid, circumradius sqrt(3/8) * edge
    T = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float)
    c, r = orc.meb_points(T)
    assert np.linalg.norm(c) < 1e-6 and abs(r - np.sqrt(3.0)) < 1e-6
    # an interior point does not move the ball
    c2, r2 = orc.meb_points(np.vstack([T, [[0.1, 0.2, -0.1]]]))
    assert np.allclose(c2, c, atol=1e-6) and abs(r2 - r) < 1e-6
    # obtuse triangle: the ball is the diametral ball of the longest side
    c, r = orc.meb_points(np.array([[0.0, 0, 0], [4.0, 0, 0], [2.0, 0.5, 0]]))
    assert np.allclose(c, [2, 0, 0], atol=1e-6) and abs(r - 2) < 1e-6
    # coincident points
    c, r = orc.meb_points(np.array([[0.5, 0.5, 0.5]] * 4))
    assert np.allclose(c, 0.5) and r == 0


def _numeric_balls(C, R):
    """epigraph form: minimise t subject to t >= |c - c_i| + r_i (SLSQP)"""
    c0 = C.mean(0)
    t0 = np.max(np.linalg.norm(C - c0, axis=1) + R)
    cons = [{"type": "ineq", "fun": (lambda v, i=i: v[3] - np.linalg.norm(C[i] - v[:3]) - R[i])}
            for i in range(len(R))]
    res = minimize(lambda v: v[3], np.r_[c0, t0], method="SLSQP", constraints=cons,
                   options={"ftol": 1e-14, "maxiter": 1000})
    c = res.x[:3]
    return c, np.max(np.linalg.norm(C - c, axis=1) + R)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_meb_balls_matches_numerical_minimum(orc, n):
    rng = np.random.default_rng(10 + n)
    for _ in range(4):
        C = rng.normal(size=(n, 3))
        R = rng.uniform(0.05, 0.8, size=n)
        c, r = orc.meb_balls(C, R)
        assert c is not None
        f = lambda q: np.max(np.linalg.norm(C - q, axis=1) + R)
        cn, rn = _numeric_balls(C, R)
        # the oracle's ball contains every ball and its centre is optimal to single precision
        assert f(c) <= r * (1 + 3e-5)
        assert abs(r - rn) <= 3e-5 * rn
        assert f(c) <= rn * (1 + 3e-5)


def test_meb_balls_with_zero_radii_equals_points(orc):
    rng = np.random.default_rng(99)
    for _ in range(5):
        P = rng.normal(size=(7, 3))
        c1, r1 = orc.meb_points(P)
        c2, r2 = orc.meb_balls(P, np.zeros(7))
        assert abs(r1 - r2) < 3e-5 * r1
        assert np.linalg.norm(c1 - c2) < 1e-2 * r1


def test_meb_balls_nested_and_equal(orc):
    # a ball containing the others is the answer
    C = np.array([[0.0, 0, 0], [0.1, 0, 0], [0, 0.2, 0]])
    R = np.array([1.0, 0.3, 0.2])
    c, r = orc.meb_balls(C, R)
    assert np.allclose(c, 0, atol=1e-6) and abs(r - 1) < 1e-6
    # two equal balls: centre midway, radius half the span plus r
    c, r = orc.meb_balls(np.array([[0.0, 0, 0], [2.0, 0, 0]]), np.array([0.5, 0.5]))
    assert np.allclose(c, [1, 0, 0], atol=1e-6) and abs(r - 1.5) < 1e-6
