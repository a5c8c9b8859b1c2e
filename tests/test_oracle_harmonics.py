"""Pins for the oracle's solid harmonics (eq. 2, App. A.3) against what the paper
and the mathematics fix: the printed closed forms of Table 3, the defining
relation between Upsilon and Theta, the addition theorem for 1/|r - x|
(App. A.4) and the shift theorem for Upsilon."""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_harmonics.txt")


def _table():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        n, m, c, poly = line.split(None, 3)
        rows.append((int(n), int(m), float(c), poly))
    return rows


def _points():
    rng = np.random.default_rng(7)
    return rng.normal(size=(12, 3)) * np.array([1.3, 0.7, 1.1])


def _real_part(Xc, n, m, idx):
    v = Xc[idx(n, abs(m))]
    return v.real if m >= 0 else v.imag


def test_table3_has_all_entries():
    rows = _table()
    assert len(rows) == 49
    assert {(n, m) for n, m, _, _ in rows} == {(n, m) for n in range(7) for m in range(-n, n + 1)}


@pytest.mark.parametrize("kind", ["upsilon", "theta"])
def test_table3_closed_forms(orc, kind):
    """(n-m)!(n+m)! U_n^m = r^{2n+1} T_n^m = coefficient * polynomial (Table 3)."""
    rows = _table()
    for pt in _points():
        x, y, z = pt
        r2 = x * x + y * y + z * z
        X = (orc.upsilon if kind == "upsilon" else orc.theta)(6, pt)
        for n, m, c, poly in rows:
            want = c * eval(poly, {}, {"x": x, "y": y, "z": z, "r2": r2})
            got = _real_part(X, n, m, orc.idx)
            if kind == "upsilon":
                got *= math.factorial(n - abs(m)) * math.factorial(n + abs(m))
            else:
                got *= r2 ** (n + 0.5)  # r^{2n+1}
            scale = max(1.0, abs(want))
            assert abs(got - want) <= 1e-12 * scale * (1 + r2) ** n, (kind, n, m, got, want)


def test_printed_20_entry_is_inconsistent(orc):
    """The printed (2,0) entry 3(z^2 - r^2) cannot be right: it is not harmonic."""
    pt = np.array([0.3, -0.4, 0.5])
    x, y, z = pt
    r2 = x * x + y * y + z * z
    Y = orc.upsilon(2, pt)
    got = 4.0 * Y[orc.idx(2, 0)].real
    assert abs(got - 3 * (z * z - r2)) > 1e-3
    assert abs(got - (3 * z * z - r2)) < 1e-14


def test_symmetry_negative_m(orc):
    """X_n^{-m} = (-1)^m X_n^{m*} for both families (eq. A.14)."""
    pt = np.array([0.7, -0.2, 0.4])
    for X in (orc.upsilon(10, pt), orc.theta(10, pt)):
        for n in range(11):
            for m in range(1, n + 1):
                assert np.allclose(X[orc.idx(n, -m)], (-1) ** m * np.conj(X[orc.idx(n, m)]), rtol=1e-14, atol=0)


def test_upsilon_theta_relation(orc):
    """Upsilon_n^m = r^{2n+1} Theta_n^m / ((n-m)!(n+m)!) (definition in App. A.3)."""
    pt = np.array([0.9, 0.35, -0.6])
    r = np.linalg.norm(pt)
    p = 14
    Y, T = orc.upsilon(p, pt), orc.theta(p, pt)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            want = r ** (2 * n + 1) * T[orc.idx(n, m)] / (math.factorial(n - m) * math.factorial(n + m))
            assert abs(Y[orc.idx(n, m)] - want) <= 1e-12 * max(abs(want), 1e-300)


def test_theta_is_derivative_of_inverse_r(orc):
    """Theta_1^0 = -d/dz (1/r) and Theta_1^1 = -(d/dx + i d/dy)... checked as the
    central finite difference of 1/r: Theta_1^0 = z/r^3, Re Theta_1^1 = x/r^3."""
    pt = np.array([0.4, -0.8, 0.3])
    h = 1e-5
    inv = lambda q: 1.0 / np.linalg.norm(q)
    T = orc.theta(1, pt)
    dz = (inv(pt + [0, 0, h]) - inv(pt - [0, 0, h])) / (2 * h)
    dx = (inv(pt + [h, 0, 0]) - inv(pt - [h, 0, 0])) / (2 * h)
    dy = (inv(pt + [0, h, 0]) - inv(pt - [0, h, 0])) / (2 * h)
    assert abs(T[orc.idx(1, 0)].real - (-dz)) < 1e-8
    assert abs(T[orc.idx(1, 1)].real - (-dx)) < 1e-8
    assert abs(T[orc.idx(1, 1)].imag - (-dy)) < 1e-8


def test_addition_theorem(orc):
    """1/|r - x| = sum_n sum_m Upsilon_n^m(x) Theta_n^{m*}(r) for |x| < |r| (App. A.4)."""
    rng = np.random.default_rng(3)
    p = 30
    for _ in range(5):
        r = rng.normal(size=3)
        r /= np.linalg.norm(r)
        x = rng.normal(size=3)
        x *= 0.3 / np.linalg.norm(x)
        Y, T = orc.upsilon(p, x), orc.theta(p, r)
        s = np.sum(Y * np.conj(T))
        assert abs(s.imag) < 1e-14
        assert abs(s.real - 1.0 / np.linalg.norm(r - x)) < 1e-12


def test_upsilon_shift_theorem(orc):
    """Upsilon_n^m(x + y) = sum_{k,l} Upsilon_k^l(x) Upsilon_{n-k}^{m-l}(y) (App. A.4)."""
    x = np.array([0.3, -0.5, 0.2])
    y = np.array([-0.1, 0.4, 0.6])
    p = 8
    Yx, Yy, Yxy = orc.upsilon(p, x), orc.upsilon(p, y), orc.upsilon(p, x + y)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            s = 0
            for k in range(n + 1):
                for l in range(-k, k + 1):
                    if abs(m - l) <= n - k:
                        s += Yx[orc.idx(k, l)] * Yy[orc.idx(n - k, m - l)]
            assert abs(s - Yxy[orc.idx(n, m)]) < 1e-14
