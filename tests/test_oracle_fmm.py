"""Pins for the oracle's direct sum and whole FMM against closed forms, invariants,
reductions to brute force and the paper's stated accuracy behaviour (Secs. 4-6)."""
import numpy as np
import pytest

from paper_1405_2255_gb300 import inputs


def _rel(acc, ref):
    return np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.fixture(scope="module")
def plummer4k(orc):
    x, mu = inputs.config_input(1)
    psi, acc, f, coin = orc.direct(x, mu)
    return x, mu, psi, acc, f


# ---------------------------------------------------------------- direct sum

def test_direct_two_body(orc):
    x = np.array([[0.0, 0, 0], [3.0, 4.0, 0]])
    mu = np.array([2.0, 5.0])
    psi, acc, f, coin = orc.direct(x, mu, G=0.5)
    assert np.allclose(psi, [0.5 * 5 / 5, 0.5 * 2 / 5], rtol=1e-15)
    assert np.allclose(acc[0], 0.5 * 5 * np.array([3, 4, 0]) / 125, rtol=1e-15)
    assert np.allclose(acc[1], -0.5 * 2 * np.array([3, 4, 0]) / 125, rtol=1e-15)
    assert np.allclose(f, [0.5 * 5 / 25, 0.5 * 2 / 25], rtol=1e-15)
    assert coin == 0


def test_direct_cube_vertices(orc):
    """Eight unit masses on the vertices of a cube of side 2: by symmetry each
    acceleration points at the centre with a known magnitude."""
    v = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], dtype=float)
    psi, acc, f, _ = orc.direct(v, np.ones(8))
    # distances from a vertex: 3 at 2, 3 at 2 sqrt 2, 1 at 2 sqrt 3
    want_psi = 3 / 2 + 3 / (2 * np.sqrt(2)) + 1 / (2 * np.sqrt(3))
    # radial component (towards the centre) of each pair force
    s3 = np.sqrt(3)
    want_a = 3 * (1 / 4) * (1 / s3) + 3 * (1 / 8) * (np.sqrt(2) / s3) + (1 / 12)
    assert np.allclose(psi, want_psi, rtol=1e-15)
    for i in range(8):
        assert np.allclose(acc[i], -want_a * v[i] / s3, rtol=1e-14)


def test_direct_coincident_pairs_are_skipped(orc):
    x = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    psi, acc, f, coin = orc.direct(x, np.ones(3))
    assert coin == 2
    assert np.allclose(psi, [1, 1, 2])


def test_plummer_closed_form(orc):
    """Binned medians of Psi_b and the radial acceleration against the truncated
    Plummer model: Psi(r) = [1/sqrt(r^2+1) - 1/sqrt(R^2+1) + M(R)/R] / M(R),
    a(r) = r (r^2+1)^{-3/2} / M(R), R = 30."""
    n = 20000
    x, mu = inputs.plummer(n, 77)
    run = orc.fmm(x, mu, p=8, eps=1e-7, leaf_size=32, keep=False)
    R = 30.0
    MR = inputs.plummer_mass(R)
    r = np.linalg.norm(x, axis=1)
    psi_m = (1 / np.sqrt(r * r + 1) - 1 / np.sqrt(R * R + 1) + MR / R) / MR
    a_m = r / (r * r + 1) ** 1.5 / MR
    ar = -np.sum(run.acc * x, axis=1) / np.maximum(r, 1e-300)
    edges = np.quantile(r, np.linspace(0.05, 0.95, 10))
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        assert abs(np.median(run.psi[sel] / psi_m[sel]) - 1) < 0.02
        assert abs(np.median(ar[sel] / a_m[sel]) - 1) < 0.05


# ---------------------------------------------------------------- FMM

def test_fmm_reduces_to_direct_when_nothing_is_accepted(orc, plummer4k):
    """With eps -> 0 the MAC (18a) never holds: the FMM is exactly direct summation."""
    x, mu, psi, acc, f = plummer4k
    run = orc.fmm(x, mu, p=4, eps=1e-300, leaf_size=16)
    assert run.stats["n_m2l"] == 0
    assert run.stats["p2p_interactions"] == len(mu) * (len(mu) - 1)
    assert np.max(np.abs(run.psi - psi) / psi) < 1e-13
    assert np.max(_rel(run.acc, acc)) < 1e-11


def test_fmm_single_leaf_is_direct(orc):
    x, mu = inputs.plummer(50, 5)
    psi, acc, _, _ = orc.direct(x, mu, G=2.0)
    run = orc.fmm(x, mu, G=2.0, p=3, eps=1e-6, leaf_size=64)
    assert run.stats["ncells"] == 1 and run.stats["n_m2l"] == 0
    assert np.allclose(run.psi, psi, rtol=1e-14)
    assert np.allclose(run.acc, acc, rtol=1e-13)


@pytest.mark.parametrize("eps", [1e-5, 1e-6, 1e-7])
def test_fmm_error_tracks_eps_18a(orc, plummer4k, eps):
    """MAC (18a) with the low-order a-estimate: rms relative error <~ eps, the 99.99th
    percentile within ~10x (Sec. 6.3)."""
    x, mu, psi, acc, f = plummer4k
    run = orc.fmm(x, mu, p=6, eps=eps, leaf_size=16)
    e = _rel(run.acc, acc)
    rms = np.sqrt(np.mean(e ** 2))
    assert rms <= eps
    assert np.percentile(e, 99.99) <= 10 * eps
    if eps >= 1e-6:
        assert run.stats["n_m2l"] > 0


def test_fmm_error_tracks_eps_18b(orc, plummer4k):
    """MAC (18b) with the low-order f-estimate controls the scaled error da/f."""
    x, mu, psi, acc, f = plummer4k
    eps = 1e-6
    run = orc.fmm(x, mu, p=6, eps=eps, mac=orc.MAC_F, leaf_size=16)
    e = np.linalg.norm(run.acc - acc, axis=1) / f
    assert run.stats["n_m2l"] > 0
    assert np.sqrt(np.mean(e ** 2)) <= eps
    assert np.percentile(e, 99.99) <= 10 * eps


def test_exact_scale_source(orc, plummer4k):
    """MAC (18a) fed the exact |a_b| (a caller-supplied scale) behaves like the estimate."""
    x, mu, psi, acc, f = plummer4k
    eps = 1e-6
    run = orc.fmm(x, mu, p=6, eps=eps, leaf_size=16, scale=np.linalg.norm(acc, axis=1))
    e = _rel(run.acc, acc)
    assert np.sqrt(np.mean(e ** 2)) <= eps
    assert np.allclose(run.scale, np.linalg.norm(acc, axis=1)[run.perm])


def test_geometric_mac_error_falls_with_p(orc, plummer4k):
    """theta < theta_crit (eq. 9): errors fall roughly like theta^p as p grows."""
    x, mu, psi, acc, f = plummer4k
    prev = None
    for p in (2, 4, 6, 8):
        run = orc.fmm(x, mu, p=p, mac=orc.MAC_THETA, theta_crit=0.5, leaf_size=16, p2p_c=0.0)
        rms = np.sqrt(np.mean(_rel(run.acc, acc) ** 2))
        if prev is not None:
            assert rms < 0.6 * prev
        prev = rms


def test_low_order_estimate_accuracy(orc, plummer4k):
    """The p = 1 (a) and p = 0 (f) low-order estimates have rms relative errors of ~15 %
    (Sec. 5.3.2): within [5 %, 30 %] and without a bias beyond a few per cent."""
    x, mu, psi, acc, f = plummer4k
    run = orc.fmm(x, mu, p=6, eps=1e-6, leaf_size=16)
    a_est = np.empty(len(mu))
    a_est[run.perm] = run.scale
    e = a_est / np.linalg.norm(acc, axis=1) - 1
    assert 0.05 <= np.sqrt(np.mean(e ** 2)) <= 0.3
    assert abs(np.mean(e)) < 0.05
    run = orc.fmm(x, mu, p=6, eps=1e-6, mac=orc.MAC_F, leaf_size=16)
    f_est = np.empty(len(mu))
    f_est[run.perm] = run.scale
    e = f_est / f - 1
    assert 0.05 <= np.sqrt(np.mean(e ** 2)) <= 0.3
    assert abs(np.mean(e)) < 0.05


def test_momentum(orc, plummer4k):
    """One-sided walk: sum mu a is not exactly 0, but its deviation is of the order of
    the force errors (Sec. 5.1); direct summation conserves it to rounding."""
    x, mu, psi, acc, f = plummer4k
    norm = np.sum(mu * np.linalg.norm(acc, axis=1))
    assert np.linalg.norm((mu[:, None] * acc).sum(0)) / norm < 1e-14
    eps = 1e-5
    run = orc.fmm(x, mu, p=6, eps=eps, leaf_size=16)
    assert np.linalg.norm((mu[:, None] * run.acc).sum(0)) / norm < 3 * eps


def test_tree_invariants(orc, plummer4k):
    x, mu, *_ = plummer4k
    leaf = 16
    run = orc.fmm(x, mu, p=4, eps=1e-6, leaf_size=leaf)
    ci = run.cells_int
    level, isleaf, first, count = ci[:, 0], ci[:, 1], ci[:, 2], ci[:, 3]
    assert count[0] == len(mu) and first[0] == 0 and level[0] == 0
    # leaves partition the particles
    L = np.where(isleaf == 1)[0]
    order = np.argsort(first[L])
    assert np.all(first[L][order][1:] == (first[L] + count[L])[order][:-1])
    assert np.all((count[L] <= leaf) | (level[L] == 21))
    assert np.all(count[isleaf == 0] > leaf)
    # every particle lies inside its leaf's ball
    s, rho = run.cells_dbl[:, :3], run.cells_dbl[:, 3]
    xs = x[run.perm]
    for c in L[:200]:
        d = np.linalg.norm(xs[first[c]:first[c] + count[c]] - s[c], axis=1)
        assert np.isclose(d.max(), rho[c], rtol=1e-14)


def test_cusp_with_point_mass(orc):
    """gamma = 1.5 Dehnen cusp with a 1 % central point mass (the cuspy workload)."""
    x, mu = inputs.dehnen(4000, 11)
    psi, acc, f, _ = orc.direct(x, mu)
    eps = 1e-6
    run = orc.fmm(x, mu, p=8, eps=eps, leaf_size=16)
    e = _rel(run.acc, acc)
    assert np.sqrt(np.mean(e ** 2)) <= eps


def test_edge_cases(orc):
    r = orc.fmm(np.zeros((0, 3)), np.zeros(0), p=4)
    assert len(r.psi) == 0
    r = orc.fmm(np.array([[1.0, 2, 3]]), np.array([1.0]), p=4)
    assert r.psi[0] == 0 and np.all(r.acc[0] == 0)
    # coincident particles contribute nothing and are counted
    x = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    r = orc.fmm(x, np.ones(3), p=3, leaf_size=1)
    assert r.stats["coincident"] == 2
    assert np.allclose(r.psi, [1, 1, 2])
    for bad_x, bad_mu in ((np.array([[np.nan, 0, 0]]), np.ones(1)), (np.zeros((2, 3)), np.array([1.0, -1.0]))):
        with pytest.raises(ValueError):
            orc.fmm(bad_x, bad_mu, p=3)
