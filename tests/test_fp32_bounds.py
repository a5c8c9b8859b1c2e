"""Error bounds behind the single-precision pre-tests (host arithmetic, no GPU).

Two kernels decide in FP32 and fall back to FP64 near their thresholds: the walk's
acceptance test (theta < 1, eq. 9) and the selection of the particles whose FP64 distance
can be a cell's radius (Sec. 4).  Both rest on the error of a centre difference formed
from two-float values, (x_hi - s_hi) + (x_lo - s_lo).  These tests emulate the kernels'
FP32 operations in their order with numpy float32 (round to nearest, no contraction
except where the kernel uses an FMA) and check the bounds the kernels' margins are built
on, on inputs chosen to stress them: near-coincident points far from the origin, points
at the origin, mixed magnitudes over many decades.
"""
import numpy as np

F = np.float32


def split(v):
    """FP64 value as FP32 high part plus FP32 low part (the library's two-float form)."""
    h = np.asarray(v, dtype=np.float64).astype(F)
    l = (np.asarray(v, dtype=np.float64) - h.astype(np.float64)).astype(F)
    return h, l


def twofloat_diff(x, s):
    xh, xl = split(x)
    sh, sl = split(s)
    return (xh - sh) + (xl - sl)  # float32 throughout


def cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        kind = t % 6
        c = rng.normal(size=3) * 10.0 ** rng.uniform(-6, 12)
        scale = max(1.0, np.abs(c).max())
        if kind == 0:
            x = c + rng.normal(size=3) * 10.0 ** rng.uniform(-12, 2) * scale
        elif kind == 1:
            x = c + rng.normal(size=3) * scale * 10.0 ** rng.uniform(-16, -6)
        elif kind == 2:
            x = np.nextafter(c, c + 1)
        elif kind == 3:
            c = rng.normal(size=3) * 1e-5
            x = rng.normal(size=3) * 1e-5
        elif kind == 4:
            x = -c
        else:
            x = c * (1 + rng.normal(size=3) * 1e-7)
        out.append((x, c))
    return out


def test_twofloat_difference_error():
    """Per coordinate: |d_f - d| <= 2^-23 |d| + 2^-46 (|x| + |s|)."""
    for x, s in cases(30000, 11):
        d = x - s  # the FP64 difference (exact to 2^-53 relative)
        df = twofloat_diff(x, s).astype(np.float64)
        bound = 2.0 ** -23 * np.abs(d) + 2.0 ** -46 * (np.abs(x) + np.abs(s)) + 2.0 ** -52 * np.abs(d)
        assert np.all(np.abs(df - d) <= bound), (x, s, df, d)


def radius_bounds(x, s):
    """The radii kernel's FP32 lower and upper bounds of |x - s| (distance, not squared)."""
    xh, _ = split(x)
    sh, _ = split(s)
    dd = twofloat_diff(x, s)
    d2 = F(0)
    for k in range(3):  # fmaf: the exact product, one rounding
        d2 = F(np.float64(dd[k]) * np.float64(dd[k]) + np.float64(d2))
    mag = F(0)
    for k in range(3):
        mag = F(mag + F(abs(xh[k]) + abs(sh[k])))
    if not (mag >= F(2.0 ** -18) and mag <= F(2.0 ** 60)):
        return 0.0, np.inf
    df = np.sqrt(d2, dtype=F)
    e = F(mag * F(2.0 ** -44))
    lb = max(F(0), F(F(df * F(1 - 2.0 ** -20)) - e))
    ub = F(F(df * F(1 + 2.0 ** -20)) + e)
    return float(lb), float(ub)


def test_radius_candidate_bounds():
    """lb <= |x - s| <= ub for the FP64 distance the exact pass takes, so the particle at
    the largest distance always passes the candidate test ub >= max lb."""
    for x, s in cases(60000, 12):
        d = float(np.sqrt(((x - s) ** 2).sum()))
        lb, ub = radius_bounds(x, s)
        assert lb <= d * (1 + 1e-15) and d <= ub * (1 + 1e-15), (x, s, d, lb, ub)


def test_radius_candidates_contain_the_maximum():
    """Over a cell's particles the FP64 maximum is attained by a candidate."""
    rng = np.random.default_rng(13)
    for t in range(300):
        s = rng.normal(size=3) * 10.0 ** rng.uniform(-3, 8)
        k = rng.integers(2, 40)
        r = 10.0 ** rng.uniform(-9, 0) * max(1.0, np.abs(s).max())
        xs = s + rng.normal(size=(k, 3)) * r
        if t % 3 == 0:  # several particles at nearly the same largest distance
            u = rng.normal(size=(k, 3))
            u /= np.linalg.norm(u, axis=1)[:, None]
            xs = s + u * r * (1 + rng.normal(size=(k, 1)) * 1e-9)
        d = np.sqrt(((xs - s) ** 2).sum(axis=1))
        b = [radius_bounds(x, s) for x in xs]
        lb_max = max(v[0] for v in b)
        cand = [i for i in range(k) if b[i][1] >= lb_max]
        assert d[cand].max() == d.max()


def test_walk_distance_relative_error():
    """The walk's r from two-float centres: once (2^-24 sum|coords|)^2 < r^2 (the kernel's
    check), r_f is within 2^-19 of r, the basis of its 1e-5 theta margin."""
    checked = 0
    for x, s in cases(40000, 14):
        dd = twofloat_diff(x, s)
        r2 = F(F(F(dd[0] * dd[0]) + F(dd[1] * dd[1])) + F(dd[2] * dd[2]))
        xh, _ = split(x)
        sh, _ = split(s)
        e = F(F(np.abs(xh).sum() + np.abs(sh).sum()) * F(2.0 ** -24))
        if not (r2 >= F(2.0 ** -100)) or not (F(e * e) < r2):
            continue  # the kernel leaves these to FP64
        r = float(np.sqrt(((x - s) ** 2).sum()))
        rf = float(np.sqrt(np.float64(r2)))
        assert abs(rf - r) <= 2.0 ** -19 * r, (x, s, rf, r)
        checked += 1
    assert checked > 10000
