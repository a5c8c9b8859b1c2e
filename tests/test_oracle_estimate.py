"""Pins for the oracle's error estimate E~_{A->B} (Sec. 4.2, eqs. 14-17), the quantity behind
every acceptance decision of the walk (eqs. 18a,b), and for the single-interaction
experiment of Sec. 4 that the paper uses to judge it.

Exact pins: for a source whose multipole power is P_n = M rho^n (a point mass at distance
rho from the expansion centre), E_{A->B} = theta^p (the binomial theorem; Sec. 4.2 states the
equality); E~ = 8 max(rho_A, rho_B) / (rho_A + rho_B) E, so E~ = 4 theta^p at rho_A = rho_B
and 8 (rho_A / r)^p at rho_B = 0.  Any spread of the mass lowers P_n and hence E~.
Statistical pins: the paper's Figs. 2-3 (relative errors hardly ever above E~, a small tail
of absolute errors above it, hardly any interaction overestimated by more than 10x, the
strict bound eq. 12 always)."""
import numpy as np
import pytest

from paper_1405_2255_gb300 import inputs


def _point_mass_power(orc, p, rho, mass=2.5):
    """P_0..P_p (eq. 14) of a single particle at distance rho from the centre, through the
    oracle's own P2M (eq. 3c) and power routines."""
    d = np.array([0.3, -0.5, 0.8])
    d *= rho / np.linalg.norm(d)
    M = orc.p2m(p, d[None, :], np.array([mass]), np.zeros(3))
    return orc.power(p, M)


@pytest.mark.parametrize("p", [1, 4, 10, 16])
def test_point_mass_power_is_maximal(orc, p):
    """P_n = M rho^n for a point mass (the equality case of Sec. 4.2's bound P_n <= M rho^n)."""
    rho, mass = 0.37, 2.5
    P = _point_mass_power(orc, p, rho, mass)
    np.testing.assert_allclose(P, mass * rho ** np.arange(p + 1), rtol=1e-13)


@pytest.mark.parametrize("p", [2, 5, 10, 14])
def test_estimate_equals_theta_p_for_a_point_mass(orc, p):
    """E = theta^p exactly when P_n = M rho^n: E~ = 4 theta^p for equal radii."""
    rho, mass, r = 0.4, 2.5, 1.9
    P = _point_mass_power(orc, p, rho, mass)
    theta = 2 * rho / r
    Et = orc.error_estimate(P, r, rho, rho, mass)
    assert Et == pytest.approx(4 * theta ** p, rel=1e-12)


@pytest.mark.parametrize("p", [3, 8, 12])
def test_estimate_factor_limits(orc, p):
    """The factor of eq. (17) is 4 at rho_A = rho_B and tends to 8 as either radius vanishes:
    a point source (rho_B = 0) gives E~ = 8 (rho_A / r)^p; all mass at the centre (P_k = 0 for
    k > 0, rho_A = 0) gives E~ = 8 (rho_B / r)^p."""
    rho, mass, r = 0.3, 1.7, 2.2
    P = _point_mass_power(orc, p, rho, mass)
    assert orc.error_estimate(P, r, rho, 0.0, mass) == pytest.approx(8 * (rho / r) ** p, rel=1e-12)
    P0 = np.zeros(p + 1)
    P0[0] = mass
    assert orc.error_estimate(P0, r, 0.0, rho, mass) == pytest.approx(8 * (rho / r) ** p, rel=1e-12)
    # a radius ratio near 0 approaches the limit continuously
    tiny = orc.error_estimate(P, r, rho, 1e-9 * rho, mass)
    assert tiny == pytest.approx(8 * (rho / r) ** p, rel=1e-7)


@pytest.mark.parametrize("p", [4, 8, 12])
def test_spread_source_lowers_the_estimate(orc, p):
    """A cell whose mass is spread inside rho has P_n < M rho^n for n >= 2, hence
    E_{A->B} < theta^p; it is never below the all-at-the-centre value (rho_B / r)^p."""
    rng = np.random.default_rng(p)
    pts = rng.normal(size=(200, 3))
    pts /= np.linalg.norm(pts, axis=1)[:, None]
    pts *= rng.uniform(0, 1, size=(200, 1)) ** (1 / 3)
    mu = rng.uniform(0.5, 1.5, 200)
    z = (mu[:, None] * pts).sum(0) / mu.sum()
    rho = np.linalg.norm(pts - z, axis=1).max()
    M = orc.p2m(p, pts, mu, z)
    P = orc.power(p, M)
    assert np.all(P[2:] < mu.sum() * rho ** np.arange(2, p + 1))
    r, rb = 3.1 * rho, 0.8 * rho
    spread = orc.error_estimate(P, r, rho, rb, mu.sum())
    point = orc.error_estimate(_point_mass_power(orc, p, rho, mu.sum()), r, rho, rb, mu.sum())
    P0 = np.zeros(p + 1)
    P0[0] = mu.sum()
    centre = orc.error_estimate(P0, r, rho, rb, mu.sum())
    assert centre < spread < point
    assert point == pytest.approx(8 * rho / (rho + rb) * ((rho + rb) / r) ** p, rel=1e-12)


@pytest.fixture(scope="module")
def interactions(orc):
    """Sec. 4's experiment on a Plummer sphere of 3e4: cell pairs accepted by theta < 0.7,
    pairs with N_A N_B < p^3 left out, 6000 sampled per order."""
    x, mu = inputs.plummer(30000, 99)
    return {p: orc.interaction_errors(x, mu, p, theta_crit=0.7, leaf_size=32, sample=6000, seed=p)
            for p in (4, 8)}


@pytest.mark.parametrize("p", [4, 8])
def test_single_interactions_against_the_estimate(interactions, p):
    """Figs. 2-3: the relative error of an interaction hardly ever exceeds E~ (eq. 16), the
    absolute error delta a r^2 / M_A exceeds it only in a small tail, and hardly any
    interaction is overestimated by more than a factor of ten."""
    e = interactions[p]
    assert len(e) > 3000
    rel, ab, Et = e[:, 1], e[:, 0], e[:, 2]
    assert np.mean(rel > Et) <= 0.02
    assert np.mean(ab > Et) <= 0.10
    assert np.mean(rel < 0.1 * Et) <= 0.02
    assert 0.1 < np.median(rel / Et) < 1.0


@pytest.mark.parametrize("p", [4, 8])
def test_single_interactions_within_strict_bound(interactions, p):
    """eq. (12): delta a <= M_A/r^2 (p+1) theta^p / (1 - theta)^2 for every interaction."""
    e = interactions[p]
    ab, theta = e[:, 0], e[:, 3]
    assert np.all(theta < 0.7)
    assert np.all(ab <= (p + 1) * theta ** p / (1 - theta) ** 2)
